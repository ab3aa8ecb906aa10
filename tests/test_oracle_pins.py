"""Pins for the FP64 oracle against what physics and mathematics fix.

None of these re-types the oracle's own formula: each check compares the
oracle with an independent fact (a closed form, an invariant, a textbook
routine, or a different brute-force method on tiny inputs).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2602_11092_gb300 import workloads


def rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- permanents

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_ryser_matches_permutation_sum(n):
    rng = np.random.default_rng(n)
    A = rand_c(rng, n, n)
    assert abs(oracle.permanent(A) - oracle.permanent_naive(A)) <= 1e-13 * max(1.0, abs(oracle.permanent_naive(A)))


@pytest.mark.parametrize("n", range(1, 11))
def test_permanent_all_ones_is_factorial(n):
    assert oracle.permanent(np.ones((n, n))) == pytest.approx(math.factorial(n), rel=1e-14)


def test_permanent_of_diagonal_and_triangular():
    # Per(triangular) = product of the diagonal (only the identity permutation survives)
    rng = np.random.default_rng(7)
    A = np.triu(rand_c(rng, 6, 6))
    assert abs(oracle.permanent(A) - np.prod(np.diag(A))) < 1e-12


# ---------------------------------------------------------------- Fock space

@pytest.mark.parametrize("m,n", [(1, 3), (2, 4), (3, 3), (4, 2), (5, 4), (6, 3), (6, 5)])
def test_enumeration_order_and_count(m, n):
    out = oracle.enumerate_fock(m, n)
    assert out.shape == (math.comb(m + n - 1, n), m)
    assert np.all(out.sum(axis=1) == n)
    tuples = [tuple(r) for r in out]
    assert len(set(tuples)) == len(tuples)
    # descending lexicographic: Python tuple order reversed
    assert tuples == sorted(tuples, reverse=True)
    assert tuples == oracle.enumerate_fock_recursive(m, n)
    assert tuples[0] == (n,) + (0,) * (m - 1)
    assert tuples[-1] == (0,) * (m - 1) + (n,)


def test_enumeration_sampled_positions():
    m, n = 9, 5
    full = oracle.enumerate_fock(m, n)
    pos = np.array([0, 3, 17, 500, full.shape[0] - 1])
    assert np.array_equal(oracle.enumerate_fock(m, n, pos), full[pos])


# ---------------------------------------------------------------- physics pins

def test_hong_ou_mandel():
    # 50:50 beam splitter, one photon in each input: no coincidences.
    for B in (oracle.BS, np.array([[1, 1], [1, -1]]) / np.sqrt(2)):
        out = oracle.enumerate_fock(2, 2)          # (2,0), (1,1), (0,2)
        p = oracle.probabilities(B, [1, 1], out)
        assert p[1] <= 1e-15
        assert p[0] == pytest.approx(0.5, abs=1e-15)
        assert p[2] == pytest.approx(0.5, abs=1e-15)


def test_single_photon_is_column_modulus():
    rng = np.random.default_rng(3)
    U = workloads.haar_unitaries(7, 1, rng)[0]
    for i in range(7):
        s = [0] * 7
        s[i] = 1
        out = oracle.enumerate_fock(7, 1)
        p = oracle.probabilities(U, s, out)
        # output e_j has index j in descending-lex order
        assert np.allclose(p, np.abs(U[:, i]) ** 2, atol=1e-15)


def test_identity_and_permutation_give_delta():
    m, s = 5, [2, 0, 1, 0, 1]
    out = oracle.enumerate_fock(m, 4)
    tuples = [tuple(r) for r in out]
    p = oracle.probabilities(np.eye(m), s, out)
    assert p[tuples.index(tuple(s))] == pytest.approx(1.0, abs=1e-15)
    assert p.sum() == pytest.approx(1.0, abs=1e-15)
    perm = [3, 0, 4, 1, 2]           # input mode i -> output mode perm[i]
    P = np.zeros((m, m))
    for i, j in enumerate(perm):
        P[j, i] = 1.0
    target = [0] * m
    for i, si in enumerate(s):
        target[perm[i]] += si
    p = oracle.probabilities(P, s, out)
    assert p[tuples.index(tuple(target))] == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("m,n", [(6, 3), (5, 4), (8, 4), (8, 3)])
def test_haar_probabilities_sum_to_one(m, n):
    rng = np.random.default_rng(100 + m + n)
    U = workloads.haar_unitaries(m, 1, rng)[0]
    s = [1] * n + [0] * (m - n) if n <= m else None
    p = oracle.probabilities(U, s)
    assert abs(p.sum() - 1.0) <= 1e-12
    assert np.all(p >= 0)


@pytest.mark.parametrize("m,n", [(4, 4), (6, 3), (8, 4)])
def test_fourier_suppression_law(m, n):
    # U_jk = e^{2 pi i jk/m}/sqrt(m); photons in modes 0, m/n, 2m/n, ...:
    # p(t) = 0 whenever sum_j j t_j is not 0 mod n.
    F = np.exp(2j * np.pi * np.outer(np.arange(m), np.arange(m)) / m) / np.sqrt(m)
    s = [0] * m
    for l in range(n):
        s[l * m // n] = 1
    out = oracle.enumerate_fock(m, n)
    p = oracle.probabilities(F, s, out)
    weight = (out * np.arange(m)[None, :]).sum(axis=1)
    forbidden = (weight % n) != 0
    assert forbidden.any()
    assert np.all(p[forbidden] <= 1e-14)
    assert abs(p.sum() - 1.0) < 1e-12


def test_mean_photon_number_closed_form():
    rng = np.random.default_rng(11)
    m, s = 7, [1, 0, 2, 0, 1, 0, 0]
    U = workloads.haar_unitaries(m, 1, rng)[0]
    out = oracle.enumerate_fock(m, 4)
    p = oracle.probabilities(U, s, out)
    lhs = (out * p[:, None]).sum(axis=0)
    rhs = (np.abs(U) ** 2) @ np.array(s, dtype=float)
    assert np.allclose(lhs, rhs, atol=1e-13)


def _fock_amplitudes_by_expansion(U, s):
    """Independent brute force: expand prod_k (sum_j U[j, c_k] a_j^dag) |0> as a
    polynomial in the creation operators, then normalise the monomials."""
    m = U.shape[0]
    cols = [i for i in range(m) for _ in range(s[i])]
    poly = {tuple([0] * m): 1.0 + 0j}
    for c in cols:
        nxt = {}
        for mono, coef in poly.items():
            for j in range(m):
                t = list(mono)
                t[j] += 1
                t = tuple(t)
                nxt[t] = nxt.get(t, 0) + coef * U[j, c]
        poly = nxt
    sf = np.prod([math.factorial(x) for x in s])
    return {t: coef * math.sqrt(np.prod([math.factorial(x) for x in t])) / math.sqrt(sf) for t, coef in poly.items()}


@pytest.mark.parametrize("m,s", [(3, [1, 1, 1]), (4, [2, 0, 1, 0]), (5, [0, 3, 0, 0, 1])])
def test_amplitudes_match_operator_expansion(m, s):
    rng = np.random.default_rng(sum(s) + m)
    U = workloads.haar_unitaries(m, 1, rng)[0]
    out = oracle.enumerate_fock(m, sum(s))
    a = oracle.amplitudes(U, s, out)
    ref = _fock_amplitudes_by_expansion(U, s)
    for t, amp in zip(out, a):
        assert abs(amp - ref[tuple(t)]) < 1e-13


def test_photon_number_spectrum_of_one_data_phase():
    # Eq. (1): U(x) = W2 S(x) W1 with S(x) = e^{i x n_1}; every p(t) is a
    # trigonometric polynomial in x whose frequencies satisfy |w| <= n, and with
    # universal W1, W2 the top frequency n is present.
    m, n = 5, 3
    rng = np.random.default_rng(5)
    W1, W2 = workloads.haar_unitaries(m, 2, rng)
    s = [1, 1, 1, 0, 0]
    N = 4 * n + 2
    xs = 2 * np.pi * np.arange(N) / N
    out = oracle.enumerate_fock(m, n)
    freqs = np.fft.fftfreq(N, d=1.0 / N)

    def spectrum(Ufun):
        P = np.array([oracle.probabilities(Ufun(x), s, out) for x in xs])
        return np.fft.fft(P, axis=0) / N

    S = lambda x: np.diag([np.exp(1j * x)] + [1.0] * (m - 1))
    spec = spectrum(lambda x: W2 @ S(x) @ W1)
    assert np.abs(spec[np.abs(freqs) > n]).max() < 1e-12
    assert np.abs(spec[np.abs(freqs) == n]).max() > 1e-6
    # the same bound through the Clements mesh with one data phase
    theta = rng.uniform(0, 2 * np.pi, m * (m - 1))
    spec = spectrum(lambda x: oracle.mesh_unitary(m, theta, [x]))
    assert np.abs(spec[np.abs(freqs) > n]).max() < 1e-12


# ---------------------------------------------------------------- mesh

def test_mzi_closed_form():
    # B diag(e^{i th},1) B diag(e^{i ph},1) = i e^{i th/2} [[s, c],[c, -s]] diag(e^{i ph}, 1)
    for th, ph in [(0.3, 1.1), (2.0, -0.7), (np.pi, 0.2), (0.0, 3.0)]:
        sn, cs = np.sin(th / 2), np.cos(th / 2)
        closed = 1j * np.exp(1j * th / 2) * np.array([[sn, cs], [cs, -sn]]) @ np.diag([np.exp(1j * ph), 1])
        assert np.allclose(oracle.mzi(th, ph), closed, atol=1e-15)


def test_mzi_cross_and_bar():
    T0 = oracle.mzi(0.0, 0.4)
    assert abs(abs(T0[0, 1]) - 1) < 1e-15 and abs(T0[0, 0]) < 1e-15
    Tp = oracle.mzi(np.pi, 0.4)
    assert abs(abs(Tp[0, 0]) - 1) < 1e-15 and abs(Tp[0, 1]) < 1e-15


def test_mesh_m2_and_m3_brute_force():
    rng = np.random.default_rng(1)
    th2 = rng.uniform(0, 2 * np.pi, 2)
    # m=2: two columns, only column 0 holds an MZI (k=0); column 1 has k=1 > m-2
    assert oracle.mesh_layout(2) == [(0, 0)]
    assert np.allclose(oracle.mesh_unitary(2, th2), oracle.mzi(*th2))
    # with data phases the screen follows the first m//2 = 1 column, even
    # though column 1 holds no MZI
    d2 = rng.uniform(0, 2 * np.pi, 2)
    assert np.allclose(oracle.mesh_unitary(2, th2, d2), np.diag(np.exp(1j * d2)) @ oracle.mzi(*th2))
    assert np.allclose(oracle.mesh_unitary(2, th2, d2, data_col=0), oracle.mzi(*th2) @ np.diag(np.exp(1j * d2)))
    # m=3: columns 0 (k=0), 1 (k=1), 2 (k=0)
    th3 = rng.uniform(0, 2 * np.pi, 6)
    assert oracle.mesh_layout(3) == [(0, 0), (1, 1), (2, 0)]

    def e01(T):
        return np.array([[T[0, 0], T[0, 1], 0], [T[1, 0], T[1, 1], 0], [0, 0, 1]])

    def e12(T):
        return np.array([[1, 0, 0], [0, T[0, 0], T[0, 1]], [0, T[1, 0], T[1, 1]]])
    U = e01(oracle.mzi(th3[4], th3[5])) @ e12(oracle.mzi(th3[2], th3[3])) @ e01(oracle.mzi(th3[0], th3[1]))
    assert np.allclose(oracle.mesh_unitary(3, th3), U, atol=1e-15)
    # data screen after column m//2 = 1 (between MZI 0 and MZI 1)
    d = rng.uniform(0, 2 * np.pi, 3)
    S = np.diag(np.exp(1j * d))
    U = e01(oracle.mzi(th3[4], th3[5])) @ e12(oracle.mzi(th3[2], th3[3])) @ S @ e01(oracle.mzi(th3[0], th3[1]))
    assert np.allclose(oracle.mesh_unitary(3, th3, d), U, atol=1e-15)


@pytest.mark.parametrize("m", [2, 5, 12, 16])
def test_mesh_is_unitary_and_counts(m):
    rng = np.random.default_rng(m)
    th = rng.uniform(0, 2 * np.pi, m * (m - 1))
    assert len(oracle.mesh_layout(m)) == m * (m - 1) // 2
    U = oracle.mesh_unitary(m, th, rng.uniform(0, 1, m))
    assert np.abs(U @ U.conj().T - np.eye(m)).max() < 1e-14


# ---------------------------------------------------------------- threshold

def test_threshold_patterns_and_sum():
    m, n = 6, 3
    pats = oracle.threshold_patterns(m, n)
    assert len(pats) == sum(math.comb(m, k) for k in range(1, n + 1))
    assert pats[:m] == [(j,) for j in range(m)]
    assert pats[m:m + 3] == [(0, 1), (0, 2), (1, 2)]  # colex
    rng = np.random.default_rng(2)
    U = workloads.haar_unitaries(m, 1, rng)[0]
    out = oracle.enumerate_fock(m, n)
    p = oracle.probabilities(U, [1, 1, 1, 0, 0, 0], out)
    q = oracle.threshold_probs(p, out, m, n)
    assert abs(q.sum() - 1.0) < 1e-12
    # brute force: for each pattern, sum over outputs with exactly that support
    for idx, pat in enumerate(pats):
        mask = np.all((out > 0) == np.isin(np.arange(m), pat)[None, :], axis=1)
        assert abs(q[idx] - p[mask].sum()) < 1e-15
    # a single photon: threshold = PNR
    out1 = oracle.enumerate_fock(m, 1)
    p1 = oracle.probabilities(U, [0, 0, 1, 0, 0, 0], out1)
    assert np.allclose(oracle.threshold_probs(p1, out1, m, 1), p1)


def test_threshold_single_pattern_matches_aggregation():
    m, n = 7, 4
    rng = np.random.default_rng(17)
    U = workloads.haar_unitaries(m, 1, rng)[0]
    s = [1, 0, 1, 0, 1, 0, 1]
    out = oracle.enumerate_fock(m, n)
    q = oracle.threshold_probs(oracle.probabilities(U, s, out), out, m, n)
    pats = oracle.threshold_patterns(m, n)
    for idx in [0, 3, 10, 40, len(pats) - 1]:
        assert abs(oracle.threshold_prob_of_pattern(U, s, pats[idx]) - q[idx]) < 1e-15


# ---------------------------------------------------------------- gradients

@pytest.mark.parametrize("m,s", [(4, [1, 0, 1, 0]), (5, [1, 1, 0, 1, 0]), (6, [1, 0, 2, 0, 0, 0])])
def test_fd_gradient_matches_permanent_minor_gradient(m, s):
    rng = np.random.default_rng(40 + m)
    th = rng.uniform(0, 2 * np.pi, m * (m - 1))
    d = rng.uniform(0, np.pi, m) * rng.standard_normal(m)
    K = oracle.fock_dim(m, sum(s))
    c = rng.standard_normal(K)
    gt_fd, gd_fd = oracle.fd_grad_phases(m, th, d, s, c)
    gt_an, gd_an = oracle.analytic_grad_phases(m, th, d, s, c)
    scale = max(np.abs(gt_an).max(), 1e-3)
    assert np.abs(gt_fd - gt_an).max() < 1e-7 * scale * 100
    assert np.abs(gd_fd - gd_an).max() < 1e-7 * scale * 100


def test_grad_U_minors_against_wirtinger_fd():
    # dU = dL/dRe U + i dL/dIm U, checked entrywise by FD on Re and Im parts.
    rng = np.random.default_rng(9)
    m, s = 4, [1, 1, 0, 1]
    U = workloads.haar_unitaries(m, 1, rng)[0]
    out = oracle.enumerate_fock(m, 3)
    c = rng.standard_normal(out.shape[0])
    dU = oracle.grad_U_minors(U, s, c, out)
    h = 1e-6
    for j, i in itertools.product(range(m), range(m)):
        E = np.zeros((m, m)); E[j, i] = 1
        gr = (oracle.loss(U + h * E, s, c, out) - oracle.loss(U - h * E, s, c, out)) / (2 * h)
        gi = (oracle.loss(U + 1j * h * E, s, c, out) - oracle.loss(U - 1j * h * E, s, c, out)) / (2 * h)
        assert abs(dU[j, i] - (gr + 1j * gi)) < 1e-8


# ---------------------------------------------------------------- surrogate reference

def test_mlp_reference_gradients_match_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(12)
    sizes = [(6, 8), (6, 6), (5, 6)]  # (out, in): 4 phases -> 8 features -> 6 -> 6 -> 5
    params = [(rng.standard_normal(s) * 0.5, rng.standard_normal(s[0]) * 0.1) for s in sizes]
    phases = rng.uniform(0, 2 * np.pi, (3, 4))
    target = rng.dirichlet(np.ones(5), size=3)
    _, _, grads = mlp.loss_and_grads(params, phases, target, bf=False)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for idx in [(0, 0), (1, 2), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            fd = (mlp.loss_and_grads(pp, phases, target, bf=False)[0] -
                  mlp.loss_and_grads(pm, phases, target, bf=False)[0]) / (2 * h)
            assert abs(fd - grads[l][0][idx]) < 1e-7
        bp, bm = b.copy(), b.copy()
        bp[0] += h
        bm[0] -= h
        pp = list(params); pp[l] = (W, bp)
        pm = list(params); pm[l] = (W, bm)
        fd = (mlp.loss_and_grads(pp, phases, target, bf=False)[0] -
              mlp.loss_and_grads(pm, phases, target, bf=False)[0]) / (2 * h)
        assert abs(fd - grads[l][1][0]) < 1e-7


def _bf16_round_bits(x):
    """Round float32 values to bfloat16 (round to nearest, ties to even) by
    their bit patterns: keep the top 16 bits after adding 0x7FFF plus the
    lowest kept bit (finite inputs)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_mlp_bf16_rounding_is_round_to_nearest_even():
    """The BF16 mode's rounding against the bit-level definition, including
    halfway cases (ties go to the even neighbour) and representable values."""
    from oracle import mlp
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000), [0.0, -0.0, 1.0, -2.5]])
    x = x.astype(np.float32)
    assert np.array_equal(mlp.bf16(x), _bf16_round_bits(x))
    # halfway between 1 and 1 + 2^-7: ties to even (1); between 1 + 2^-7 and 1 + 2^-6: up
    half = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8], dtype=np.float32)
    assert np.array_equal(mlp.bf16(half), [1.0, 1.0 + 2.0 ** -6])
    assert np.abs(mlp.bf16(x) - x).max() <= np.abs(x).max() * 2.0 ** -8


def test_mlp_bf16_mode_within_its_rounding_bound_of_fp64():
    """The BF16 mode is the FP64 model with values rounded to bfloat16
    (unit roundoff u = 2^-9) at a fixed number of points per layer: features,
    weights, pre-activations and activations.  Each rounding perturbs a value
    by at most u relative, so with L hidden layers the logits and gradients
    stay within a few (4L + 4) u of the FP64 model, relative to their norm,
    and they do differ from it (the rounding is really applied)."""
    from oracle import mlp
    rng = np.random.default_rng(9)
    sizes = [(32, 16), (32, 32), (10, 32)]  # 8 phases -> 16 features -> 32 -> 32 -> 10
    params = [(rng.standard_normal(sz) / np.sqrt(sz[1]), rng.standard_normal(sz[0]) * 0.1) for sz in sizes]
    phases = rng.uniform(0, 2 * np.pi, (6, 8))
    target = rng.dirichlet(np.ones(10), size=6)
    u = 2.0 ** -9
    bound = (4 * (len(sizes) - 1) + 4) * u
    z64, _ = mlp.forward(params, phases, bf=False)
    zbf, _ = mlp.forward(params, phases, bf=True)
    rel = np.linalg.norm(zbf - z64) / np.linalg.norm(z64)
    assert 0.1 * u < rel <= bound, rel
    _, _, g64 = mlp.loss_and_grads(params, phases, target, bf=False)
    _, _, gbf = mlp.loss_and_grads(params, phases, target, bf=True)
    for (w64, b64), (wbf, bbf) in zip(g64, gbf):
        assert np.linalg.norm(wbf - w64) / np.linalg.norm(w64) <= 4 * bound
        assert np.linalg.norm(bbf - b64) / np.linalg.norm(b64) <= 4 * bound


def test_mlp_reference_invariants():
    from oracle import mlp
    z = np.array([[0.3, -1.0, 2.0], [5.0, 5.0, 5.0]])
    q = mlp.softmax(z)
    assert np.allclose(q.sum(axis=1), 1.0) and np.allclose(q[1], 1 / 3)
    # GELU: gelu(0) = 0, gelu(z) -> z for large z, gelu' by FD
    assert mlp.gelu(0.0) == 0.0 and abs(mlp.gelu(10.0) - 10.0) < 1e-12
    zz = np.linspace(-4, 4, 17)
    fd = (mlp.gelu(zz + 1e-6) - mlp.gelu(zz - 1e-6)) / 2e-6
    assert np.abs(fd - mlp.gelu_grad(zz)).max() < 1e-8
    # KL(p || softmax(log p)) = 0
    rng = np.random.default_rng(0)
    p = rng.dirichlet(np.ones(4), size=2)
    params = [(np.zeros((4, 2)), np.log(p[0]))]
    loss, _, _ = mlp.loss_and_grads(params, np.zeros((1, 1)), p[:1], bf=False)
    assert abs(loss) < 1e-12


# ---------------------------------------------------------------- spaces and measurements

@pytest.mark.parametrize("m,n", [(2, 2), (4, 2), (6, 3), (7, 7), (5, 1)])
def test_unbunched_outputs_are_the_fock_outputs_without_collisions(m, n):
    full = oracle.enumerate_fock(m, n)
    restricted = full[full.max(axis=1) <= 1]
    assert np.array_equal(oracle.enumerate_unbunched(m, n), restricted)
    assert len(restricted) == math.comb(m, n)


def test_unbunched_hong_ou_mandel_and_permutation():
    # |1,1> through a 50:50 beam splitter never leaves one photon per mode
    bs = np.array([[1, 1j], [1j, 1]]) / np.sqrt(2)
    assert oracle.probabilities(bs, [1, 1], oracle.enumerate_unbunched(2, 2))[0] <= 1e-15
    # a permutation sends |1,0,1,0> to one collision-free state with certainty
    perm = [2, 0, 3, 1]
    U = np.zeros((4, 4), dtype=np.complex128)
    for i, j in enumerate(perm):
        U[j, i] = 1.0
    outs = oracle.enumerate_unbunched(4, 2)
    p = oracle.probabilities(U, [1, 0, 1, 0], outs)
    target = np.zeros(4, dtype=np.int32)
    target[[perm[0], perm[2]]] = 1
    assert np.allclose(p, [1.0 if np.array_equal(t, target) else 0.0 for t in outs], atol=1e-15)


def test_mode_expectations_match_the_linear_closed_form():
    rng = np.random.default_rng(19)
    m, s = 6, [2, 0, 1, 0, 1, 0]
    U = workloads.haar_unitaries(m, 1, rng)[0]
    outs = oracle.enumerate_fock(m, 4)
    e = oracle.mode_expectations(oracle.probabilities(U, s, outs), outs)
    assert np.allclose(e, (np.abs(U) ** 2) @ np.array(s, dtype=float), atol=1e-13)


def test_click_probabilities_are_one_minus_no_photon():
    rng = np.random.default_rng(23)
    m, n, s = 5, 3, [1, 1, 0, 1, 0]
    U = workloads.haar_unitaries(m, 1, rng)[0]
    outs = oracle.enumerate_fock(m, n)
    p = oracle.probabilities(U, s, outs)
    clicks = oracle.click_probabilities(oracle.threshold_probs(p, outs, m, n), m, n)
    dark = np.array([p[outs[:, j] == 0].sum() for j in range(m)])
    assert np.allclose(clicks, 1.0 - dark, atol=1e-13)


def test_renormalise_sums_to_one_and_keeps_ratios():
    p = np.array([0.1, 0.0, 0.3, 0.05])
    q = oracle.renormalise(p)
    assert abs(q.sum() - 1.0) < 1e-15
    assert abs(q[2] / q[0] - 3.0) < 1e-12 and q[1] == 0.0


# ---------------------------------------------------------------- shot sampling

def test_sampling_dyadic_boundaries_are_exact():
    # p = (1/4, 3/4): draws below 1/4 give outcome 0, from 1/4 on outcome 1
    p = np.array([0.25, 0.75], dtype=np.float32)
    just_below = np.float32(np.nextafter(np.float32(0.25), np.float32(0.0)))
    u = np.array([0.0, just_below, 0.25, 0.5, np.nextafter(np.float32(1.0), np.float32(0.0))], dtype=np.float32)
    assert list(oracle.sample_outcomes(p, u)) == [0, 0, 1, 1, 1]


def test_sampling_never_draws_zero_weight_outcomes_and_follows_p():
    p = workloads.random_distributions(1, 40, seed=3, zero_fraction=0.3)[0]
    u = workloads.uniforms(1, 40000, seed=4)[0]
    s = oracle.sample_outcomes(p, u)
    counts = np.bincount(s, minlength=40)
    assert np.all(counts[p == 0] == 0)
    # every frequency within 5 standard deviations of its probability
    sd = np.sqrt(p * (1 - p) / len(u))
    assert np.all(np.abs(counts / len(u) - p) <= 5 * sd + 1e-9)


def test_sampling_one_hot_monotone_and_empty():
    p = np.zeros(7, dtype=np.float32)
    p[4] = 1.0
    assert set(oracle.sample_outcomes(p, workloads.uniforms(1, 200, seed=5)[0])) == {4}
    q = workloads.random_distributions(1, 30, seed=6)[0]
    u = np.sort(workloads.uniforms(1, 500, seed=7)[0])
    assert np.all(np.diff(oracle.sample_outcomes(q, u)) >= 0)
    assert set(oracle.sample_outcomes(np.zeros(5, np.float32), u[:10])) == {-1}


# ---------------------------------------------------------------- fidelity kernel

def test_fidelity_kernel_identity_symmetry_and_transition_probability():
    rng = np.random.default_rng(31)
    m, s = 5, [1, 0, 2, 0, 1]
    A = workloads.haar_unitaries(m, 3, rng)
    Bm = workloads.haar_unitaries(m, 4, rng)
    K = oracle.fidelity_kernel(A, Bm, s)
    assert np.allclose(np.diag(oracle.fidelity_kernel(A, A, s)), 1.0, atol=1e-13)
    assert np.allclose(K, oracle.fidelity_kernel(Bm, A, s).T, atol=1e-14)
    # the same number is the probability of output s for input s through Ua^dag Ub
    V = A[1].conj().T @ Bm[2]
    p = oracle.probabilities(V, s, np.array([s], dtype=np.int32))[0]
    assert abs(K[1, 2] - p) < 1e-13
    assert np.all((K >= 0) & (K <= 1 + 1e-12))


def test_fidelity_kernel_closed_forms():
    rng = np.random.default_rng(37)
    m = 4
    A = workloads.haar_unitaries(m, 2, rng)
    Bm = workloads.haar_unitaries(m, 3, rng)
    # one photon in mode 2: the squared overlap of the two columns
    K1 = oracle.fidelity_kernel(A, Bm, [0, 0, 1, 0])
    ref1 = np.abs(np.einsum("ij,kj->ik", A[:, :, 2].conj(), Bm[:, :, 2])) ** 2
    assert np.allclose(K1, ref1, atol=1e-14)
    # two photons in mode 1: <s|V|s> = V_11^2
    K2 = oracle.fidelity_kernel(A, Bm, [0, 2, 0, 0])
    v = np.einsum("ij,kj->ik", A[:, :, 1].conj(), Bm[:, :, 1])
    assert np.allclose(K2, np.abs(v) ** 4, atol=1e-14)


# ---------------------------------------------------------------- amplitude encoding

def test_transfer_matrix_is_a_unitary_representation():
    rng = np.random.default_rng(43)
    m, n = 4, 3
    basis = oracle.enumerate_fock(m, n)
    U1, U2 = workloads.haar_unitaries(m, 2, rng)
    P1, P2 = oracle.transfer_matrix(U1, basis), oracle.transfer_matrix(U2, basis)
    # a representation: Phi(U1 U2) = Phi(U1) Phi(U2), and unitary on the full Fock basis
    assert np.allclose(oracle.transfer_matrix(U1 @ U2, basis), P1 @ P2, atol=1e-12)
    assert np.allclose(P1.conj().T @ P1, np.eye(len(basis)), atol=1e-12)
    x = rng.standard_normal((3, len(basis))) + 1j * rng.standard_normal((3, len(basis)))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    assert np.allclose(np.linalg.norm(oracle.encoded_amplitudes(U1, x, basis), axis=1), 1.0, atol=1e-12)


def test_transfer_matrix_of_a_permutation_permutes_the_basis():
    m, n = 3, 2
    basis = oracle.enumerate_fock(m, n)
    perm = [2, 0, 1]  # input mode i -> output mode perm[i]
    U = np.zeros((m, m), dtype=np.complex128)
    for i, j in enumerate(perm):
        U[j, i] = 1.0
    P = oracle.transfer_matrix(U, basis)
    index = {tuple(t): i for i, t in enumerate(basis)}
    for si, s in enumerate(basis):
        t = [0] * m
        for i in range(m):
            t[perm[i]] = s[i]
        col = np.zeros(len(basis))
        col[index[tuple(t)]] = 1.0
        assert np.allclose(P[:, si], col, atol=1e-15)


@pytest.mark.parametrize("m,k", [(3, 5), (8, 4), (12, 6), (16, 7), (20, 3)])
def test_occupied_mode_counts_of_a_layer(m, k):
    """The uneven-batch planner sizes the sections of a layer (states with q
    occupied modes) in closed form: choose the q modes, then split k photons
    into q positive parts, C(m, q) C(k-1, q-1); the sizes sum to the layer,
    C(m+k-1, k) (Vandermonde).  Checked by counting the enumerated states."""
    states = oracle.enumerate_fock(m, k)
    counts = np.bincount((states > 0).sum(axis=1), minlength=min(m, k) + 1)
    assert counts[0] == 0
    for q in range(1, min(m, k) + 1):
        assert counts[q] == math.comb(m, q) * math.comb(k - 1, q - 1)
    assert counts.sum() == math.comb(m + k - 1, k) == oracle.fock_dim(m, k)
