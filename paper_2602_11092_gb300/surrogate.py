"""ctypes binding of include/surrogate.h (argument marshalling only) and the
surrogate driver: tensor-core MLP inference with an exact SLOS spot check and
exact fallback (the exact path judges the surrogate's total variation)."""
from __future__ import annotations

import ctypes

import torch

from . import binding as B

_vp, _i64, _int, _f = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float

_SIG = {
    "surr_gemm_bf16": ([_int, _int, _int, _int, _vp, _i64, _vp, _i64, _vp, _int, _vp, _vp, _vp], _int),
    "surr_sync_status": ([_vp], _int),
    "surr_create": ([_int, _int, _int, _int, _int, ctypes.c_ulonglong, ctypes.POINTER(_vp)], _int),
    "surr_destroy": ([_vp], _int),
    "surr_forward": ([_vp, _vp, _int, _vp, _vp], _int),
    "surr_train_step": ([_vp, _vp, _vp, _int, _f, _vp, _vp], _int),
    "surr_get_param": ([_vp, _int, _vp, _vp], _int),
    "surr_set_param": ([_vp, _int, _vp, _vp], _int),
    "surr_get_grad": ([_vp, _int, _vp, _vp], _int),
}

_done = False


def lib():
    global _done
    L = B.load()
    if not _done:
        for name, (args, res) in _SIG.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _done = True
    return L


def symbols():
    return list(_SIG)


GEMM_F32, GEMM_F32_BIAS, GEMM_GELU, GEMM_GELU_BWD, GEMM_F32_ACCUM = 0, 1, 2, 3, 4


def gemm(A: torch.Tensor, Bm: torch.Tensor, epi: int = GEMM_F32, C: torch.Tensor | None = None,
         bias: torch.Tensor | None = None, aux: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """C = A . B^T on the tensor cores (A [M][K], B [N][K] bf16)."""
    M, K = A.shape
    N = Bm.shape[0]
    if C is None:
        dt = torch.bfloat16 if epi in (GEMM_GELU, GEMM_GELU_BWD) else torch.float32
        C = torch.empty((M, N), dtype=dt, device=A.device)
    B._check(lib().surr_gemm_bf16(epi, M, N, K, B._ptr(A), A.stride(0), B._ptr(Bm), Bm.stride(0), B._ptr(C),
                                  C.stride(0), B._ptr(bias), B._ptr(aux), B._stream(stream)))
    return C


def sync_status(stream=None):
    B._check(lib().surr_sync_status(B._stream(stream)))


class Surrogate:
    def __init__(self, n_phases=144, hidden=2048, n_hidden_layers=4, n_outputs=12376, max_batch=4096, seed=1004):
        h = ctypes.c_void_p()
        B._check(lib().surr_create(n_phases, hidden, n_hidden_layers, n_outputs, max_batch, seed, ctypes.byref(h)))
        self._h = h
        self.n_phases, self.hidden, self.n_layers, self.K = n_phases, hidden, n_hidden_layers, n_outputs
        self.max_batch = max_batch

    def forward(self, phases: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        Bn = phases.shape[0]
        if out is None:
            out = torch.empty((Bn, self.K), dtype=torch.float32, device=phases.device)
        B._check(lib().surr_forward(self._h, B._ptr(phases), Bn, B._ptr(out), B._stream(stream)))
        return out

    def train_step(self, phases, target, lr, loss_rows=None, stream=None):
        B._check(lib().surr_train_step(self._h, B._ptr(phases), B._ptr(target), phases.shape[0], float(lr),
                                       B._ptr(loss_rows), B._stream(stream)))

    def _shape(self, layer):
        fi = 2 * self.n_phases if layer == 0 else self.hidden
        fo = self.K if layer == self.n_layers else self.hidden
        return fo, fi

    def get_param(self, layer):
        import numpy as np
        fo, fi = self._shape(layer)
        w = np.zeros((fo, fi), dtype=np.float32)
        b = np.zeros(fo, dtype=np.float32)
        B._check(lib().surr_get_param(self._h, layer, w.ctypes.data, b.ctypes.data))
        return w, b

    def set_param(self, layer, w, b):
        import numpy as np
        w = np.ascontiguousarray(w, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        B._check(lib().surr_set_param(self._h, layer, w.ctypes.data, b.ctypes.data))

    def get_grad(self, layer):
        import numpy as np
        fo, fi = self._shape(layer)
        w = np.zeros((fo, fi), dtype=np.float32)
        b = np.zeros(fo, dtype=np.float32)
        B._check(lib().surr_get_grad(self._h, layer, w.ctypes.data, b.ctypes.data))
        return w, b

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and B._lib is not None:
            B._lib.surr_destroy(h)
            self._h = None
