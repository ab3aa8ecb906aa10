"""Amplitude-encoded input (slos_encoded_forward): psi(t) = sum_s <t|U|s> x_s
against the oracle's transfer matrix (Ryser permanents)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_11092_gb300 import workloads

pytestmark = pytest.mark.gpu

P_TOL = 1e-5


def rand_states(rng, B, K):
    x = rng.standard_normal((B, K)) + 1j * rng.standard_normal((B, K))
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.complex64)


@pytest.mark.parametrize("m,n,space,B", [(4, 3, 0, 5), (6, 3, 0, 70), (5, 4, 0, 3), (8, 3, 1, 9), (7, 7, 0, 2),
                                         (9, 1, 0, 4)])
def test_encoded_amplitudes_match_oracle(slos, m, n, space, B):
    rng = np.random.default_rng(80 + m + n)
    s = [n] + [0] * (m - 1)  # any input: the plan only fixes (m, n, space)
    if space == 1:
        s = [1] * n + [0] * (m - n)
    plan = slos.Plan(m, s, space=space)
    basis = oracle.enumerate_unbunched(m, n) if space == 1 else oracle.enumerate_fock(m, n)
    K = plan.n_outputs
    assert K == len(basis)
    U = workloads.haar_unitaries(m, 1, rng)[0].astype(np.complex64)
    X = rand_states(rng, B, K)
    Ut, Xt = torch.tensor(U, device="cuda"), torch.tensor(X, device="cuda")
    amps = plan.encoded_forward(Ut, Xt, slos.AMPS).cpu().numpy()
    probs = plan.encoded_forward(Ut, Xt, slos.PROBS).cpu().numpy()
    ref = oracle.encoded_amplitudes(U.astype(np.complex128), X.astype(np.complex128), basis)
    assert np.abs(amps - ref).max() <= P_TOL
    assert np.abs(probs - np.abs(ref) ** 2).max() <= P_TOL
    if space == 0:  # the transfer matrix is unitary on the full Fock basis
        assert np.abs(probs.sum(axis=1) - 1.0).max() <= 1e-4


@pytest.mark.parametrize("m,n,B", [(8, 4, 4100), (10, 4, 130), (12, 2, 9000)])
def test_encoded_tensor_core_gemm_chunks_and_ragged_tiles(slos, m, n, B):
    """The GEMM runs on the tensor cores in TF32 with the three-product split
    (batch chunks of 4096 rows, 128 x 256 output tiles over (re, im)
    interleaved columns): batches past one chunk, output counts that leave a
    partial tile (2K = 660, 1430, 156 columns), every row and output against
    the oracle within the FP32 tolerance."""
    rng = np.random.default_rng(300 + m + n)
    plan = slos.Plan(m, [n] + [0] * (m - 1))
    basis = oracle.enumerate_fock(m, n)
    K = plan.n_outputs
    U = workloads.haar_unitaries(m, 1, rng)[0].astype(np.complex64)
    X = rand_states(rng, B, K)
    Ut, Xt = torch.tensor(U, device="cuda"), torch.tensor(X, device="cuda")
    amps = plan.encoded_forward(Ut, Xt, slos.AMPS)
    probs = plan.encoded_forward(Ut, Xt, slos.PROBS)
    plan.sync_status()
    ref = oracle.encoded_amplitudes(U.astype(np.complex128), X.astype(np.complex128), basis)
    assert np.abs(amps.cpu().numpy() - ref).max() <= P_TOL
    p = probs.cpu().numpy()
    assert np.abs(p - np.abs(ref) ** 2).max() <= P_TOL
    assert 0.5 * np.abs(p - np.abs(ref) ** 2).sum(axis=1).max() <= 1e-5
    assert torch.equal(probs, plan.encoded_forward(Ut, Xt, slos.PROBS))  # fixed summation order


def test_encoded_basis_state_equals_plain_forward(slos):
    """x = |s> reproduces slos_forward's amplitudes for input s."""
    m, s = 10, [1, 0, 2, 0, 1, 0, 0, 0, 0, 0]
    rng = np.random.default_rng(91)
    plan = slos.Plan(m, s)
    U = torch.tensor(workloads.haar_unitaries(m, 1, rng)[0].astype(np.complex64), device="cuda")
    basis = oracle.enumerate_fock(m, 4)
    idx = [i for i, t in enumerate(basis) if list(t) == s][0]
    X = torch.zeros((2, plan.n_outputs), dtype=torch.complex64, device="cuda")
    X[0, idx] = 1.0
    X[1, idx] = 1j
    amps = plan.encoded_forward(U, X, slos.AMPS)
    ref = plan.forward(U[None], slos.AMPS)[0]
    assert (amps[0] - ref).abs().max().item() <= P_TOL
    assert (amps[1] - 1j * ref).abs().max().item() <= P_TOL


def test_encoded_rejects_large_or_threshold_plans(slos):
    with pytest.raises(slos.SlosError):
        slos.Plan(16, [1, 0] * 8).encoded_forward(torch.eye(16, dtype=torch.complex64, device="cuda"),
                                                   torch.zeros((1, 490314), dtype=torch.complex64, device="cuda"))
    with pytest.raises(slos.SlosError):
        slos.Plan(4, [1, 1, 0, 0], slos.THRESHOLD).encoded_forward(
            torch.eye(4, dtype=torch.complex64, device="cuda"), torch.zeros((1, 10), dtype=torch.complex64,
                                                                            device="cuda"))
