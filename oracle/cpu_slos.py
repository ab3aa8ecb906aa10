"""CPU SLOS recursion (slos_cpu.c): a timed CPU baseline, not a parity
reference (TEST INFRASTRUCTURE; only tests/ and bench.py's CPU-baseline leg
use it).  Its outputs are pinned against the Ryser oracle in
tests/test_cpu_slos.py."""
from __future__ import annotations

import ctypes
import os
import subprocess
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libslos_cpu.so")


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "slos_cpu.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


@lru_cache(maxsize=1)
def _lib():
    build()
    lib = ctypes.CDLL(_SO)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.slos_cpu_train.argtypes = [ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int]
    lib.slos_cpu_dim.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.slos_cpu_dim.restype = ctypes.c_int64
    lib.slos_cpu_plan_create.argtypes = [ctypes.c_int, ctypes.c_int, ip]
    lib.slos_cpu_plan_create.restype = ctypes.c_void_p
    lib.slos_cpu_plan_destroy.argtypes = [ctypes.c_void_p]
    lib.slos_cpu_plan_train.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int]
    return lib


class Plan:
    """Transition tables for (m, input state), built once; train() then runs
    the forward and reverse recursion for a batch of unitaries."""

    def __init__(self, m: int, s):
        self.m = m
        self.s = np.ascontiguousarray(s, dtype=np.int32)
        self.n = int(self.s.sum())
        self.K = int(_lib().slos_cpu_dim(m, self.n))
        self._p = _lib().slos_cpu_plan_create(m, self.n, self.s.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        if not self._p:
            raise ValueError("slos_cpu_plan_create failed (m, n up to 64; input must hold n photons)")

    def __del__(self):
        if getattr(self, "_p", None):
            _lib().slos_cpu_plan_destroy(self._p)
            self._p = None

    def train(self, U: np.ndarray, g: np.ndarray | None = None, nthreads: int = 0):
        U = np.ascontiguousarray(U, dtype=np.complex128)
        B = U.shape[0]
        if U.shape[1:] != (self.m, self.m):
            raise ValueError("U must be [B][m][m]")
        probs = np.empty((B, self.K), dtype=np.float64)
        dU = np.empty((B, self.m, self.m), dtype=np.complex128) if g is not None else None
        gp = None
        if g is not None:
            gp = np.ascontiguousarray(g, dtype=np.float64)
            if gp.shape != (self.K,):
                raise ValueError("g must have one weight per output state")
        dpt = ctypes.POINTER(ctypes.c_double)
        rc = _lib().slos_cpu_plan_train(self._p, B, U.ctypes.data_as(dpt),
                                        gp.ctypes.data_as(dpt) if gp is not None else None,
                                        probs.ctypes.data_as(dpt), dU.ctypes.data_as(dpt) if dU is not None else None,
                                        int(nthreads))
        if rc != 0:
            raise MemoryError("slos_cpu_plan_train: out of memory")
        return probs, dU


def train(U: np.ndarray, s, g: np.ndarray | None = None, nthreads: int = 0):
    """U: complex [B][m][m]; s: input occupations; g: [K] weights of
    L = sum_t g(t) p(t) (None: forward only).  Returns (probs [B][K], dU [B][m][m]
    or None) in FP64."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    B, m, _ = U.shape
    s = np.ascontiguousarray(s, dtype=np.int32)
    n = int(s.sum())
    if m > 64 or n > 64:
        raise ValueError("slos_cpu: m and n up to 64")
    lib = _lib()
    K = int(lib.slos_cpu_dim(m, n))
    probs = np.empty((B, K), dtype=np.float64)
    dU = np.empty((B, m, m), dtype=np.complex128) if g is not None else None
    gp = None
    if g is not None:
        gp = np.ascontiguousarray(g, dtype=np.float64)
        if gp.shape != (K,):
            raise ValueError("g must have one weight per output state")
    dpt = ctypes.POINTER(ctypes.c_double)
    rc = lib.slos_cpu_train(m, n, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), B,
                            U.ctypes.data_as(dpt), gp.ctypes.data_as(dpt) if gp is not None else None,
                            probs.ctypes.data_as(dpt), dU.ctypes.data_as(dpt) if dU is not None else None,
                            int(nthreads))
    if rc != 0:
        raise MemoryError("slos_cpu_train: out of memory")
    return probs, dU
