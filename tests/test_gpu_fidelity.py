"""Fidelity kernel (slos_fidelity_kernel) against the oracle's Ryser
permanents: K[i][j] = |<s|Ua[i]^dag Ub[j]|s>|^2."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_11092_gb300 import workloads

pytestmark = pytest.mark.gpu

K_TOL = 1e-5


@pytest.mark.parametrize("m,s,Na,Nb", [
    (4, [0, 0, 1, 0], 5, 3),            # one photon
    (5, [1, 0, 2, 0, 1], 17, 9),        # bunched, ragged tiles
    (6, [1, 1, 1, 0, 0, 0], 20, 33),
    (12, [1, 0] * 6, 16, 16),
    (10, [2, 0, 0, 1, 0, 0, 2, 0, 1, 1], 7, 40),  # 7 photons
    (16, [1, 0] * 8, 6, 5),             # 8 photons
    (24, [1] * 4 + [0] * 20, 3, 18),    # 24 modes
])
def test_fidelity_kernel_matches_oracle(slos, m, s, Na, Nb):
    rng = np.random.default_rng(70 + m + Na)
    Ua = workloads.haar_unitaries(m, Na, rng).astype(np.complex64)
    Ub = workloads.haar_unitaries(m, Nb, rng).astype(np.complex64)
    K = slos.fidelity_kernel(s, torch.tensor(Ua, device="cuda"), torch.tensor(Ub, device="cuda")).cpu().numpy()
    ref = oracle.fidelity_kernel(Ua.astype(np.complex128), Ub.astype(np.complex128), s)
    assert K.shape == (Na, Nb)
    assert np.abs(K - ref).max() <= K_TOL


def test_gram_matrix_diagonal_and_symmetry(slos):
    from paper_2602_11092_gb300.functions import FidelityKernel
    m, s = 12, [1, 0] * 6
    mb = workloads.mesh_batch(m, 50, seed=1001)
    kern = FidelityKernel(m, s, theta=torch.tensor(mb.theta), w=torch.ones(m))
    X = torch.tensor(mb.data, dtype=torch.float32, device="cuda")
    G = kern(X).cpu().numpy()
    assert np.abs(np.diag(G) - 1.0).max() <= K_TOL
    assert np.abs(G - G.T).max() <= K_TOL
    C = kern(X[:7], X).cpu().numpy()
    assert np.abs(C - G[:7]).max() <= 1e-6
    # against the oracle on the mesh unitaries it builds itself
    U = np.stack([oracle.mesh_unitary(m, mb.theta, mb.data[b]) for b in range(8)])
    ref = oracle.fidelity_kernel(U, U, s)
    assert np.abs(G[:8, :8] - ref).max() <= 1e-4


def test_fidelity_kernel_rejects(slos):
    U = torch.zeros((2, 4, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(slos.SlosError):
        slos.fidelity_kernel([3, 3, 3, 0], U)   # 9 photons
    with pytest.raises(slos.SlosError):
        slos.fidelity_kernel([0, 0, 0, 0], U)   # no photon
