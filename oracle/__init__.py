"""FP64 CPU oracle for the batched linear-optics layer (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library: it has
its own Fock-state enumeration, its own permanent (Ryser, in ``oracle.c``),
its own interferometer-mesh builder and its own gradients.

Every function computes a plain definition:

* output distribution of an n-photon Fock input through an m-mode unitary,
  p(t) = |Per(U[rows(t), cols(s)])|^2 / (prod t! prod s!)   (Sec. II-A.1);
* threshold-detector outcome probabilities, the sum of p(t) over outputs with
  the same set of occupied modes (Sec. II-B, detector models);
* the trainable interferometer U(x, theta) = W2(theta2) S(x) W1(theta1), built
  from Mach-Zehnder interferometers whose parameters are physical phases
  (Sec. II-A.3 and the angle-encoding circuit of Sec. II-C.1);
* gradients of L = sum_t c_t p(t) with respect to the phases, by FP64 central
  finite differences and analytically through permanent minors (Sec. II-A.3,
  differentiable simulation);
* a small FP32/FP64 MLP forward/backward used to check the learned surrogate.

Parity status: every function here is pinned by tests/test_oracle_pins.py
against physics or mathematics that does not use the function itself.
"""
from __future__ import annotations

import bisect
import ctypes
import itertools
import math
import os
import subprocess
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (and the CPU SLOS baseline,
    slos_cpu.c) with gcc (OpenMP)."""
    from . import cpu_slos
    cpu_slos.build(force)
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


@lru_cache(maxsize=1)
def _lib():
    build()
    lib = ctypes.CDLL(_SO)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.oracle_permanent.argtypes = [ctypes.c_int, dp, dp]
    lib.oracle_amplitudes.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, ctypes.c_int64, ip, dp, ctypes.c_int]
    lib.oracle_grad_U.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, ctypes.c_int64, ip, dp, dp, ctypes.c_int]
    lib.oracle_enumerate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint8)]
    lib.oracle_enumerate.restype = ctypes.c_int64
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def default_threads() -> int:
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


# --------------------------------------------------------------------------
# Fock space (Sec. II-A.1): compositions of n photons into m modes,
# N_Fock = C(m+n-1, n), listed in descending lexicographic order.
# --------------------------------------------------------------------------

def fock_dim(m: int, n: int) -> int:
    return math.comb(m + n - 1, n)


def enumerate_fock(m: int, n: int, positions=None) -> np.ndarray:
    """Compositions of n into m parts in descending lexicographic order.

    With ``positions`` (sorted ascending int array) only those entries of the
    walk are returned.  Shape [K, m], dtype int32.
    """
    total = fock_dim(m, n)
    if positions is None:
        positions = np.arange(total, dtype=np.int64)
    positions = np.ascontiguousarray(positions, dtype=np.int64)
    if positions.size and (np.any(np.diff(positions) < 0) or positions[-1] >= total or positions[0] < 0):
        raise ValueError("positions must be sorted and inside the Fock space")
    out = np.zeros((positions.size, m), dtype=np.uint8)
    got = _lib().oracle_enumerate(
        m, n, positions.size,
        positions.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
    )
    assert got == total
    return out.astype(np.int32)


def enumerate_fock_recursive(m: int, n: int):
    """Pure-Python recursion (small cases): t_0 from n down to 0, then the rest."""
    if m == 1:
        return [(n,)]
    res = []
    for t0 in range(n, -1, -1):
        for rest in enumerate_fock_recursive(m - 1, n - t0):
            res.append((t0,) + rest)
    return res


# --------------------------------------------------------------------------
# Permanents (Sec. II-A.1: probabilities are permanents of submatrices of U)
# --------------------------------------------------------------------------

def permanent(A: np.ndarray) -> complex:
    """Ryser permanent (C, FP64)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    out = np.zeros(2)
    _lib().oracle_permanent(n, _dptr(A.view(np.float64)), _dptr(out))
    return complex(out[0], out[1])


def permanent_naive(A: np.ndarray) -> complex:
    """Sum over all n! permutations of prod_i A[i, sigma(i)] (tiny n only)."""
    n = A.shape[0]
    tot = 0j
    for sigma in itertools.permutations(range(n)):
        prod = 1 + 0j
        for i in range(n):
            prod *= A[i, sigma[i]]
        tot += prod
    return tot


def amplitudes(U: np.ndarray, s, outputs: np.ndarray | None = None, nthreads: int | None = None) -> np.ndarray:
    """<t|U|s> = Per(U[rows(t), cols(s)]) / sqrt(prod t! prod s!) for each output t."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    m = U.shape[0]
    s = np.ascontiguousarray(s, dtype=np.int32)
    n = int(s.sum())
    if outputs is None:
        outputs = enumerate_fock(m, n)
    outputs = np.ascontiguousarray(outputs, dtype=np.int32)
    K = outputs.shape[0]
    amps = np.zeros(K, dtype=np.complex128)
    _lib().oracle_amplitudes(m, n, _dptr(U.view(np.float64)), _iptr(s), K, _iptr(outputs),
                             _dptr(amps.view(np.float64)), nthreads or default_threads())
    return amps


def probabilities(U: np.ndarray, s, outputs=None, nthreads=None) -> np.ndarray:
    a = amplitudes(U, s, outputs, nthreads)
    return a.real ** 2 + a.imag ** 2


# --------------------------------------------------------------------------
# Threshold detectors (Sec. II-B): each mode reports only "click" / "no click".
# Outcome = set b of occupied modes, 1 <= |b| <= min(n, m); q(b) = sum of p(t)
# over outputs t whose occupied-mode set is b.  Outcome order: by |b|
# ascending, then by colex rank of the subset.
# --------------------------------------------------------------------------

def threshold_patterns(m: int, n: int):
    pats = []
    for k in range(1, min(n, m) + 1):
        subsets = list(itertools.combinations(range(m), k))
        subsets.sort(key=lambda c: tuple(reversed(c)))  # colex
        pats.extend(subsets)
    return pats


def threshold_probs(p: np.ndarray, outputs: np.ndarray, m: int, n: int) -> np.ndarray:
    pats = threshold_patterns(m, n)
    index = {pat: i for i, pat in enumerate(pats)}
    q = np.zeros(len(pats), dtype=np.float64)
    for prob, t in zip(p, outputs):
        key = tuple(int(j) for j in np.nonzero(t)[0])
        q[index[key]] += prob
    return q


def threshold_prob_of_pattern(U: np.ndarray, s, pattern, nthreads=None) -> float:
    """q(b) for one occupied-mode set b: the sum of p(t) over every output t
    whose occupied modes are exactly b (all compositions of n into |b|
    positive parts, placed on b)."""
    U = np.asarray(U)
    m = U.shape[0]
    n = int(np.sum(s))
    b = list(pattern)

    def positive_parts(total, parts):
        if parts == 1:
            yield (total,)
            return
        for first in range(1, total - parts + 2):
            for rest in positive_parts(total - first, parts - 1):
                yield (first,) + rest

    outs = []
    for occ in positive_parts(n, len(b)):
        t = [0] * m
        for mode, c in zip(b, occ):
            t[mode] = c
        outs.append(t)
    return float(probabilities(U, s, np.array(outs, dtype=np.int32), nthreads).sum())


# --------------------------------------------------------------------------
# Computation spaces and measurement strategies (Sec. II-A.3, QuantumLayer:
# the Hilbert subspace the state is represented on; full distribution or
# per-mode photon-number expectations).
# --------------------------------------------------------------------------

def enumerate_unbunched(m: int, n: int) -> np.ndarray:
    """Collision-free outputs (every t_j <= 1), one row per output, in the
    library's order: the Fock order (descending lexicographic over occupation
    vectors) restricted to them, which lists the occupied-mode tuples in
    ascending lexicographic order."""
    rows = []
    for S in itertools.combinations(range(m), n):
        t = np.zeros(m, dtype=np.int32)
        t[list(S)] = 1
        rows.append(t)
    return np.array(rows, dtype=np.int32).reshape(-1, m)


def mode_expectations(p: np.ndarray, outputs: np.ndarray) -> np.ndarray:
    """<n_j> = sum_t t_j p(t) over the listed outputs (plain sums, FP64)."""
    p = np.asarray(p, dtype=np.float64)
    outputs = np.asarray(outputs)
    e = np.zeros(outputs.shape[1], dtype=np.float64)
    for prob, t in zip(p, outputs):
        e += prob * t
    return e


def click_probabilities(q: np.ndarray, m: int, n: int) -> np.ndarray:
    """P(detector j clicks) = sum of q(b) over threshold outcomes b with j in b."""
    e = np.zeros(m, dtype=np.float64)
    for prob, b in zip(q, threshold_patterns(m, n)):
        for j in b:
            e[j] += prob
    return e


def renormalise(p: np.ndarray) -> np.ndarray:
    """The distribution conditioned on the listed outputs: p / sum p."""
    p = np.asarray(p, dtype=np.float64)
    return p / p.sum()


# --------------------------------------------------------------------------
# Shot sampling (hardware-aware design section, MerlinProcessor: outputs as
# they come from a photonic processor, a finite number of shots).  A shot maps
# one uniform draw u in [0, 1) to an outcome by inverting the cumulative
# distribution.  To make the decision exact (the same on any machine and in
# any summation order) the weights are fixed-point integers:
# P(t) = floor(p(t) 2^32), C(t) = P(0) + ... + P(t) (exact integers),
# T = C(K-1); the shot's target is floor(floor(u 2^32) T / 2^32) and its
# outcome is the first t with C(t) > target.  Outcomes whose weight rounds to
# zero are never drawn.
# --------------------------------------------------------------------------

def sample_outcomes(p: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Outcome index of every draw in u (1-D) for the distribution p (1-D,
    float32 values as given); plain Python integers for the arithmetic.
    NaN or negative weights weigh nothing; draws outside [0, 1) are clamped
    into it (NaN counts as 0); a distribution with no weight gives -1."""
    P = [int(math.floor(float(x) * 2.0 ** 32)) if float(x) > 0.0 else 0 for x in np.asarray(p, dtype=np.float32)]
    C = list(itertools.accumulate(P))
    T = C[-1]
    out = np.empty(len(u), dtype=np.int64)
    for i, x in enumerate(np.asarray(u, dtype=np.float32)):
        U32 = 0 if not float(x) > 0.0 else min(int(math.floor(float(x) * 2.0 ** 32)), 2 ** 32 - 1)
        if T == 0:
            out[i] = -1
            continue
        target = (U32 * T) >> 32
        out[i] = bisect.bisect_right(C, target)
    return out


# --------------------------------------------------------------------------
# Fidelity kernel (kernel-methods section): |phi(x)> = U(x)|s>,
# k(x1, x2) = |<phi(x1)|phi(x2)>|^2 = |<s|U(x1)^dag U(x2)|s>|^2, and for a
# Fock state <s|V|s> = Per(V[cols(s), cols(s)]) / prod_i s_i!.
# --------------------------------------------------------------------------

def fidelity_kernel(Ua, Ub, s) -> np.ndarray:
    """k[i][j] = |<s|Ua[i]^dag Ub[j]|s>|^2 (FP64, Ryser permanents)."""
    s = [int(x) for x in s]
    cols = [i for i in range(len(s)) for _ in range(s[i])]
    sf = float(np.prod([math.factorial(x) for x in s]))
    Ua = np.asarray(Ua, dtype=np.complex128)
    Ub = np.asarray(Ub, dtype=np.complex128)
    K = np.empty((len(Ua), len(Ub)), dtype=np.float64)
    for i in range(len(Ua)):
        for j in range(len(Ub)):
            V = Ua[i].conj().T @ Ub[j]
            K[i, j] = abs(permanent(V[np.ix_(cols, cols)]) / sf) ** 2
    return K


# --------------------------------------------------------------------------
# Amplitude encoding (Sec. II-C): |x> = sum_s x_s |s> over a basis of n-photon
# Fock states; output amplitudes psi(t) = sum_s <t|U|s> x_s.
# --------------------------------------------------------------------------

def transfer_matrix(U: np.ndarray, basis: np.ndarray) -> np.ndarray:
    """Phi[t][s] = <t|U|s> for t, s in the basis (rows of occupations)."""
    basis = np.asarray(basis, dtype=np.int32)
    return np.stack([amplitudes(U, list(s), basis) for s in basis], axis=1)


def encoded_amplitudes(U: np.ndarray, X: np.ndarray, basis: np.ndarray) -> np.ndarray:
    """psi[b][t] = sum_s <t|U|s> X[b][s]."""
    Phi = transfer_matrix(U, basis)
    return np.asarray(X, dtype=np.complex128) @ Phi.T


# --------------------------------------------------------------------------
# Interferometer mesh (Sec. II-A.3: trainable parameters are the phases of the
# physical components; Sec. II-C.1: U(x, theta) = W2(theta2) S(x) W1(theta1)).
# MZI on modes (k, k+1): T = B diag(e^{i theta}, 1) B diag(e^{i phi}, 1) with
# the 50:50 beam splitter B = [[1, i], [i, 1]] / sqrt(2).  Rectangular layout:
# m columns, column c holds MZIs on (k, k+1) for k = c mod 2, c mod 2 + 2, ...
# k <= m-2; phases are ordered column by column, k ascending, (theta, phi) per
# MZI; U = T_last ... T_first.  Data screen diag(e^{i phi_d}) on modes
# 0..n_data-1 after the first `data_col` columns (default m // 2).
# --------------------------------------------------------------------------

BS = np.array([[1.0, 1.0j], [1.0j, 1.0]], dtype=np.complex128) / np.sqrt(2.0)


def mzi(theta: float, phi: float) -> np.ndarray:
    return BS @ np.diag([np.exp(1j * theta), 1.0]) @ BS @ np.diag([np.exp(1j * phi), 1.0])


def mesh_layout(m: int):
    """List of (column, k) in application order."""
    out = []
    for c in range(m):
        for k in range(c % 2, m - 1, 2):
            out.append((c, k))
    return out


def embed(m: int, k: int, T2: np.ndarray) -> np.ndarray:
    E = np.eye(m, dtype=np.complex128)
    E[k:k + 2, k:k + 2] = T2
    return E


def mesh_factors(m: int, theta, data=None, data_col=None):
    """Ordered list of (kind, index, m x m matrix), first applied first.

    kind is "mzi" (index = MZI number in phase order) or "data" (index None).
    """
    theta = np.asarray(theta, dtype=np.float64)
    layout = mesh_layout(m)
    assert theta.size == 2 * len(layout)
    if data_col is None:
        data_col = m // 2
    has_data = data is not None and len(data) > 0
    facs = []

    def screen():
        d = np.ones(m, dtype=np.complex128)
        d[: len(data)] = np.exp(1j * np.asarray(data, dtype=np.float64))
        return ("data", None, np.diag(d))

    idx = 0
    for c in range(m + 1):
        if has_data and c == data_col:
            facs.append(screen())
        while idx < len(layout) and layout[idx][0] == c:
            k = layout[idx][1]
            facs.append(("mzi", idx, embed(m, k, mzi(theta[2 * idx], theta[2 * idx + 1]))))
            idx += 1
    return facs


def mesh_unitary(m: int, theta, data=None, data_col=None) -> np.ndarray:
    U = np.eye(m, dtype=np.complex128)
    for _, _, F in mesh_factors(m, theta, data, data_col):
        U = F @ U
    return U


# --------------------------------------------------------------------------
# Gradients of L = sum_t c_t p(t) (Sec. II-A.3, differentiable simulation)
# --------------------------------------------------------------------------

def loss(U, s, c, outputs=None):
    return float(np.dot(c, probabilities(U, s, outputs)))


def fd_grad_phases(m, theta, data, s, c, h=1e-6, data_col=None, outputs=None):
    """FP64 central finite differences of L w.r.t. (theta, data)."""
    theta = np.array(theta, dtype=np.float64)
    data = np.array(data if data is not None else [], dtype=np.float64)
    if outputs is None:
        outputs = enumerate_fock(m, int(np.sum(s)))

    def L(th, da):
        return loss(mesh_unitary(m, th, da, data_col), s, c, outputs)

    gt = np.zeros_like(theta)
    for i in range(theta.size):
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        gt[i] = (L(tp, data) - L(tm, data)) / (2 * h)
    gd = np.zeros_like(data)
    for i in range(data.size):
        dp = data.copy(); dp[i] += h
        dm = data.copy(); dm[i] -= h
        gd[i] = (L(theta, dp) - L(theta, dm)) / (2 * h)
    return gt, gd


def grad_U_minors(U, s, c, outputs=None, nthreads=None) -> np.ndarray:
    """dL/dRe U + i dL/dIm U through permanent minors (C, FP64)."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    m = U.shape[0]
    s = np.ascontiguousarray(s, dtype=np.int32)
    n = int(s.sum())
    if outputs is None:
        outputs = enumerate_fock(m, n)
    outputs = np.ascontiguousarray(outputs, dtype=np.int32)
    c = np.ascontiguousarray(c, dtype=np.float64)
    dU = np.zeros((m, m), dtype=np.complex128)
    _lib().oracle_grad_U(m, n, _dptr(U.view(np.float64)), _iptr(s), outputs.shape[0], _iptr(outputs),
                         _dptr(c), _dptr(dU.view(np.float64)), nthreads or default_threads())
    return dU


def dmzi(theta: float, phi: float):
    """Derivatives of the 2x2 MZI matrix w.r.t. theta and phi, from the product form."""
    Dth = BS @ np.diag([1j * np.exp(1j * theta), 0.0]) @ BS @ np.diag([np.exp(1j * phi), 1.0])
    Dph = BS @ np.diag([np.exp(1j * theta), 1.0]) @ BS @ np.diag([1j * np.exp(1j * phi), 0.0])
    return Dth, Dph


def phase_grad_from_dU(m, theta, data, dU, data_col=None):
    """Chain dU (PyTorch convention) to the phases: dL/dx = Re sum conj(dU) * dU/dx.

    dU/dx is formed explicitly as the product of all factors with the one
    factor that depends on x replaced by its derivative.
    """
    theta = np.asarray(theta, dtype=np.float64)
    data = np.asarray(data if data is not None else [], dtype=np.float64)
    facs = mesh_factors(m, theta, data, data_col)
    layout = mesh_layout(m)
    mats = [F for _, _, F in facs]
    n_f = len(mats)
    # prefix[i] = F_{i-1} ... F_0 ; suffix[i] = F_{n-1} ... F_{i+1}
    prefix = [np.eye(m, dtype=np.complex128)]
    for F in mats:
        prefix.append(F @ prefix[-1])
    suffix = [None] * n_f
    acc = np.eye(m, dtype=np.complex128)
    for i in range(n_f - 1, -1, -1):
        suffix[i] = acc
        acc = acc @ mats[i]
    gt = np.zeros_like(theta)
    gd = np.zeros_like(data)
    for i, (kind, idx, _) in enumerate(facs):
        if kind == "mzi":
            k = layout[idx][1]
            Dth, Dph = dmzi(theta[2 * idx], theta[2 * idx + 1])
            for which, D2 in ((0, Dth), (1, Dph)):
                D = np.zeros((m, m), dtype=np.complex128)
                D[k:k + 2, k:k + 2] = D2
                dUdx = suffix[i] @ D @ prefix[i]
                gt[2 * idx + which] = np.real(np.sum(np.conj(dU) * dUdx))
        else:
            for j in range(data.size):
                D = np.zeros((m, m), dtype=np.complex128)
                D[j, j] = 1j * np.exp(1j * data[j])
                dUdx = suffix[i] @ D @ prefix[i]
                gd[j] = np.real(np.sum(np.conj(dU) * dUdx))
    return gt, gd


def analytic_grad_phases(m, theta, data, s, c, data_col=None, outputs=None):
    U = mesh_unitary(m, theta, data, data_col)
    dU = grad_U_minors(U, s, c, outputs)
    return phase_grad_from_dU(m, theta, data, dU, data_col)
