"""The learned surrogate against the method without it: exact SLOS on the
same GPU.  Measures (and prints) held-out total variation, the fallback rate
of the checked inference, and evaluations per second of both paths.  Asserts
the inference's guarantee: every returned row is exact, or the batch passed
its spot check and the rows it returns exceed the TV bound at a rate no
higher than the stated one."""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_surrogate_gain_over_exact_path():
    from paper_2602_11092_gb300 import surrogate as S
    layer = S.SurrogateLayer(hidden=1024, n_hidden_layers=3, max_batch=4096)
    hist = layer.train(n_samples=4096 * 60, batch=4096, lr=1e-3)
    assert hist[-1][1] < hist[0][1]
    ev = layer.evaluate(count=2048)
    rng = np.random.default_rng(77)
    data = layer.sample_data(4096, rng)
    # exact path
    for _ in range(2):
        layer.exact(data)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        p = layer.exact(data)
    torch.cuda.synchronize()
    exact_rate = 5 * 4096 / (time.perf_counter() - t0)
    # checked surrogate: a spot check large enough that a clean batch can pass
    # (1 - 0.01^(1/n) <= 0.01 needs n >= 459 checks)
    rho = 1 / 8
    q, stats = layer.infer(data, rho=rho, tv_tol=0.02, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in range(5):
        q, stats = layer.infer(data, rho=rho, tv_tol=0.02, seed=r)
    torch.cuda.synchronize()
    surr_rate = 5 * 4096 / (time.perf_counter() - t0)
    print(f"\nheld-out TV {ev}; inference {stats}; exact {exact_rate:.0f}/s, checked surrogate {surr_rate:.0f}/s, "
          f"gain {surr_rate / exact_rate:.2f}x")
    tv = 0.5 * (q - p).abs().sum(dim=1).cpu().numpy()
    assert np.isfinite(tv).all()
    assert stats["checked"] == round(rho * 4096)
    if stats["batch_fallback"]:
        # the spot check could not bound the failure rate: every row is exact
        assert stats["fail_rate_ucb"] > stats["max_fail_rate"]
        assert stats["fallback"] == 4096
        assert tv.max() <= 1e-5
    else:
        assert stats["fail_rate_ucb"] <= stats["max_fail_rate"]
        # rows above the bound among those returned: within the stated rate
        # (the bound holds with 99 % confidence; a failing run is a 1 % event)
        assert (tv > 0.02).mean() <= stats["max_fail_rate"]
    # the held-out distribution says whether a batch could pass at all
    if ev["frac_gt_0.02"] > 0.5:
        assert stats["batch_fallback"]
