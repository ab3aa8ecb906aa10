"""The CPU SLOS baseline (oracle/slos_cpu.c) against the Ryser oracle: it is
timed as a CPU baseline, so it must compute the same distribution and the
same dL/dU as the plain definitions (Sec. II-A.1, II-A.3)."""
import numpy as np
import pytest

import oracle
from oracle import cpu_slos
from paper_2602_11092_gb300 import workloads


@pytest.mark.parametrize("m,s", [(2, [1, 1]), (3, [2, 0, 1]), (5, [1, 0, 1, 0, 1]), (6, [0, 3, 0, 1, 0, 0]),
                                 (4, [2, 2, 1, 0])])
def test_probabilities_and_gradient_match_ryser(m, s):
    rng = np.random.default_rng(71 + m)
    B = 3
    U = workloads.haar_unitaries(m, B, rng).astype(np.complex128)
    n = sum(s)
    K = workloads.fock_dim(m, n)
    g = rng.standard_normal(K)
    probs, dU = cpu_slos.train(U, s, g, nthreads=2)
    outs = oracle.enumerate_fock(m, n)
    for b in range(B):
        ref = oracle.probabilities(U[b], s, outs)
        assert np.abs(probs[b] - ref).max() < 1e-12
        ref_dU = oracle.grad_U_minors(U[b], s, g, outs)
        assert np.abs(dU[b] - ref_dU).max() < 1e-10 * max(1.0, np.abs(ref_dU).max())


def test_forward_only_and_normalisation():
    rng = np.random.default_rng(5)
    U = workloads.haar_unitaries(7, 2, rng)
    probs, dU = cpu_slos.train(U, [1, 0, 1, 0, 1, 0, 1], None)
    assert dU is None
    assert np.abs(probs.sum(axis=1) - 1.0).max() < 1e-12


def test_rejects_wrong_weight_length():
    U = np.eye(3, dtype=np.complex128)[None]
    with pytest.raises(ValueError):
        cpu_slos.train(U, [1, 1, 0], np.zeros(5))
