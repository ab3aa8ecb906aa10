"""Seeded synthetic inputs shaped like the paper's quantum-layer workloads.

This module only draws random numbers (numpy ``default_rng``); it holds none
of the simulation arithmetic and imports nothing from the CUDA binding or the
oracle, so the tests can feed the same inputs to both.

Workloads (seed = 1000 + workload index unless overridden):

* ``tiny``      m=6,  n=3, input |1,1,1,0,0,0>, one Haar unitary, PNR.
* ``layer12``   m=12, n=6, photons in even modes, batch 4096 Clements meshes:
                132 trainable phases U[0, 2pi) shared by the batch, 12 data
                phases x*w with x ~ N(0,1)^12 per sample, w ~ U(0, pi)^12 once.
* ``train16``   m=16, n=8, photons in even modes, batch 256 meshes with 240
                trainable phases + 16 data phases drawn the same way;
                loss weights c ~ N(0,1) over the 490314 outputs.
* ``uneven``    1024 instances, m ~ U{8..20}, n ~ U{2..min(10, m//2)},
                photons in the first n even modes, Haar unitaries,
                threshold detection for m >= 16, PNR otherwise.
* ``surrogate`` the ``layer12`` phase distribution (144 phase inputs).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 1000


def fock_dim(m: int, n: int) -> int:
    return math.comb(m + n - 1, n)


def even_mode_input(m: int, n: int) -> list[int]:
    """n photons in modes 0, 2, ..., 2(n-1)."""
    s = [0] * m
    for i in range(n):
        s[2 * i] = 1
    return s


def haar_unitaries(m: int, count: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random unitaries: QR of (A + iB)/sqrt(2) with A, B standard normal
    (row-major fill, real part then imaginary part), R's diagonal phase-fixed.
    Returns complex128 [count, m, m]."""
    out = np.empty((count, m, m), dtype=np.complex128)
    for b in range(count):
        A = rng.standard_normal((m, m))
        B = rng.standard_normal((m, m))
        Z = (A + 1j * B) / np.sqrt(2.0)
        Q, R = np.linalg.qr(Z)
        d = np.diag(R)
        out[b] = Q * (d / np.abs(d))[None, :]
    return out


def n_mesh_phases(m: int) -> int:
    """Two phases per MZI, m(m-1)/2 MZIs in the rectangular mesh."""
    return m * (m - 1)


@dataclass
class MeshBatch:
    m: int
    theta: np.ndarray      # float64 [P] shared trainable phases
    w: np.ndarray          # float64 [m] data-phase weights
    x: np.ndarray          # float64 [B, m] features
    data: np.ndarray       # float64 [B, m] data phases x * w

    @property
    def batch(self) -> int:
        return self.x.shape[0]


def mesh_batch(m: int, batch: int, seed: int) -> MeshBatch:
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2.0 * np.pi, size=n_mesh_phases(m))
    w = rng.uniform(0.0, np.pi, size=m)
    x = rng.standard_normal((batch, m))
    return MeshBatch(m=m, theta=theta, w=w, x=x, data=x * w[None, :])


def tiny(seed: int = SEED_BASE + 0):
    rng = np.random.default_rng(seed)
    U = haar_unitaries(6, 1, rng)
    return dict(m=6, n=3, s=[1, 1, 1, 0, 0, 0], U=U)


def layer12(batch: int = 4096, seed: int = SEED_BASE + 1):
    m, n = 12, 6
    return dict(m=m, n=n, s=even_mode_input(m, n), mesh=mesh_batch(m, batch, seed))


def train16(batch: int = 256, seed: int = SEED_BASE + 2):
    m, n = 16, 8
    mb = mesh_batch(m, batch, seed)
    rng = np.random.default_rng(seed + 10_000)
    c = rng.standard_normal(fock_dim(m, n))
    return dict(m=m, n=n, s=even_mode_input(m, n), mesh=mb, c=c)


@dataclass
class UnevenInstance:
    m: int
    n: int
    s: list
    threshold: bool


def uneven(count: int = 1024, seed: int = SEED_BASE + 3, with_unitaries: bool = True):
    rng = np.random.default_rng(seed)
    inst = []
    for _ in range(count):
        m = int(rng.integers(8, 21))
        n = int(rng.integers(2, min(10, m // 2) + 1))
        inst.append(UnevenInstance(m=m, n=n, s=even_mode_input(m, n), threshold=m >= 16))
    Us = None
    if with_unitaries:
        Us = [haar_unitaries(it.m, 1, rng)[0] for it in inst]
    return inst, Us


def surrogate_phases(count: int, seed: int):
    """Phase vectors for the m=12 layer: shared theta (seed 1001) + data phases."""
    base = layer12(batch=1)
    mb = base["mesh"]
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((count, 12))
    return mb.theta, x * mb.w[None, :]


def random_distributions(batch: int, K: int, seed: int, zero_fraction: float = 0.1) -> np.ndarray:
    """float32 [batch, K] rows of non-negative weights summing to about one
    (exponential draws, a seeded fraction set to zero), for sampling tests."""
    rng = np.random.default_rng(seed)
    w = rng.exponential(size=(batch, K))
    w[rng.random((batch, K)) < zero_fraction] = 0.0
    w /= np.maximum(w.sum(axis=1, keepdims=True), 1e-300)
    return w.astype(np.float32)


def uniforms(batch: int, shots: int, seed: int) -> np.ndarray:
    """float32 [batch, shots] draws in [0, 1): the random numbers shot
    sampling consumes, passed in so that every side sees the same ones."""
    rng = np.random.default_rng(seed)
    u = rng.random((batch, shots)).astype(np.float32)
    return np.minimum(u, np.float32(np.nextafter(np.float32(1.0), np.float32(0.0))))
