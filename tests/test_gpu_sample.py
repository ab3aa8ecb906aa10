"""Shot sampling (slos_sample) against the oracle's exact integer inversion
of the cumulative distribution: outcome indices must agree bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_11092_gb300 import workloads

pytestmark = pytest.mark.gpu


# (m, input, detection): output sizes 2, 6, 136, 330, 12376 and 490314 (1, 1,
# 1, 2, 49 and 1916 chunks of 256 weights, ragged tails)
PLANS = [(2, [1, 0], 0), (3, [1, 1, 0], 0), (16, [1, 1] + [0] * 14, 0), (8, [1, 0] * 4, 0),
         (12, [1, 0] * 6, 0), (16, [1, 0] * 8, 0)]


@pytest.mark.parametrize("m,s,det", PLANS)
def test_samples_match_oracle_bit_for_bit(slos, m, s, det):
    plan = slos.Plan(m, s, det)
    K = plan.n_outputs
    B = 5
    shots = 400 if K > 100000 else 3000
    p = workloads.random_distributions(B, K, seed=40 + m, zero_fraction=0.2)
    p[1] = 0.0
    p[1, K // 2] = 1.0                    # one outcome only
    if K > 3:
        p[2, :3] = [np.nan, -0.5, 0.0]    # weigh nothing
    u = workloads.uniforms(B, shots, seed=50 + m)
    u[0, :6] = [0.0, np.nextafter(np.float32(1.0), np.float32(0.0)), 1.0, -0.25, np.nan, 0.5]
    pt = torch.tensor(p, device="cuda")
    ut = torch.tensor(u, device="cuda")
    samples, counts = plan.sample(pt, ut, counts=True)
    samples = samples.cpu().numpy()
    for b in range(B):
        ref = oracle.sample_outcomes(p[b], u[b])
        assert np.array_equal(samples[b], ref), f"instance {b}: {np.nonzero(samples[b] != ref)[0][:5]}"
        assert np.array_equal(counts[b].cpu().numpy(), np.bincount(ref, minlength=K))
    assert np.all(samples[1] == K // 2)


def test_distribution_without_weight_gives_minus_one(slos):
    plan = slos.Plan(4, [1, 1, 0, 0])
    p = torch.zeros((2, plan.n_outputs), dtype=torch.float32, device="cuda")
    p[1, 3] = 0.5
    u = torch.tensor(workloads.uniforms(2, 50, seed=3), device="cuda")
    samples = plan.sample(p, u).cpu().numpy()
    assert np.all(samples[0] == -1) and np.all(samples[1] == 3)


def test_shots_from_simulated_distribution_follow_it(slos):
    """End to end: distributions from slos_forward, 200k shots each, every
    outcome frequency within 5 standard deviations of the oracle's p."""
    m, s, B, shots = 8, [1, 0] * 4, 3, 200_000
    rng = np.random.default_rng(61)
    U = workloads.haar_unitaries(m, B, rng)
    plan = slos.Plan(m, s)
    probs = plan.forward(torch.tensor(U, dtype=torch.complex64, device="cuda"))
    u = torch.tensor(workloads.uniforms(B, shots, seed=62), device="cuda")
    _, counts = plan.sample(probs, u, counts=True)
    outs = oracle.enumerate_fock(m, 4)
    for b in range(B):
        p = oracle.probabilities(U[b].astype(np.complex64).astype(np.complex128), s, outs)
        f = counts[b].double().cpu().numpy() / shots
        sd = np.sqrt(p * (1 - p) / shots)
        assert np.all(np.abs(f - p) <= 5 * sd + 2e-6)
