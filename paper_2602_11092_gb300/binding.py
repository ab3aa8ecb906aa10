"""ctypes binding of libslos.so (include/slos.h): argument marshalling only.

Every computation happens inside the CUDA library; this module turns torch
tensors into device pointers and the current torch stream into a
cudaStream_t.  There is no CPU fallback: if the library is missing or a call
fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libslos.so")

PNR, THRESHOLD = 0, 1
PROBS, AMPS = 0, 1
FOCK, UNBUNCHED = 0, 1  # computation spaces (slos_space_t)

_status_names = {0: "SLOS_OK", 1: "SLOS_ERR_INVALID_ARG", 2: "SLOS_ERR_UNSUPPORTED", 3: "SLOS_ERR_OOM",
                 4: "SLOS_ERR_CUDA", 5: "SLOS_ERR_TIMEOUT", 6: "SLOS_ERR_INTERNAL"}


class SlosError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_names.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n_data", ctypes.c_int), ("data_col", ctypes.c_int)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t
_int = ctypes.c_int

# name -> argtypes (restype slos_status_t = int unless noted)
_SIGNATURES = {
    "slos_last_error": ([], ctypes.c_char_p),
    "slos_version": ([], ctypes.c_char_p),
    "mesh_unitary": ([ctypes.POINTER(MeshDesc), _vp, _i64, _vp, _i64, _int, _vp, _vp], _int),
    "mesh_unitary_backward_workspace": ([ctypes.POINTER(MeshDesc), _int, _i64, ctypes.POINTER(_sz)], _int),
    "mesh_unitary_backward": ([ctypes.POINTER(MeshDesc), _vp, _i64, _vp, _i64, _int, _vp, _vp, _vp, _vp, _sz, _vp],
                              _int),
    "mesh_unitary_weighted": ([ctypes.POINTER(MeshDesc), _vp, _i64, _vp, _i64, _vp, _int, _vp, _vp], _int),
    "slos_autotune": ([_vp, _vp, _int, _vp, _vp, _vp, _vp, _sz, ctypes.c_char_p, _vp], _int),
    "slos_plan_tuning": ([_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_int),
                          ctypes.POINTER(_int)], _int),
    "mesh_sum_rows": ([_vp, _int, _int, _vp, _vp], _int),
    "mesh_unitary_weighted_backward": ([ctypes.POINTER(MeshDesc), _vp, _i64, _vp, _i64, _vp, _int, _vp, _vp, _vp,
                                        _vp, _vp, _sz, _vp], _int),
    "slos_plan": ([_int, _int, ctypes.POINTER(_int), _int, _sz, ctypes.POINTER(_vp)], _int),
    "slos_plan_space": ([_int, _int, ctypes.POINTER(_int), _int, _int, _sz, ctypes.POINTER(_vp)], _int),
    "slos_plan_query": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_int)], _int),
    "slos_expectations": ([_vp, _vp, _int, _vp, _vp], _int),
    "slos_expectations_backward": ([_vp, _vp, _int, _vp, _vp], _int),
    "slos_renormalise": ([_vp, _vp, _int, _vp, _vp, _vp], _int),
    "slos_renormalise_backward": ([_vp, _vp, _vp, _vp, _int, _vp, _vp], _int),
    "slos_sample_workspace_bytes": ([_vp, _int, ctypes.POINTER(_sz)], _int),
    "slos_sample": ([_vp, _vp, _int, _int, _vp, _vp, _vp, _vp, _sz, _vp], _int),
    "slos_fidelity_kernel": ([_int, ctypes.POINTER(_int), _vp, _int, _vp, _int, _vp, _vp], _int),
    "slos_encoded_workspace_bytes": ([_vp, ctypes.POINTER(_sz)], _int),
    "slos_encoded_forward": ([_vp, _vp, _vp, _int, _int, _vp, _vp, _sz, _vp], _int),
    "slos_workspace_bytes": ([_vp, _int, _int, ctypes.POINTER(_sz)], _int),
    "slos_forward": ([_vp, _vp, _int, _int, _vp, _int, _vp, _sz, _vp], _int),
    "slos_backward": ([_vp, _vp, _int, _int, _vp, _i64, _vp, _vp, _sz, _vp], _int),
    "slos_sync_status": ([_vp, _vp], _int),
    "slos_plan_destroy": ([_vp], _int),
    "slos_batched_plan": ([_int, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(ctypes.POINTER(_int)),
                           ctypes.POINTER(_int), ctypes.POINTER(_vp)], _int),
    "slos_batched_query": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_sz)], _int),
    "slos_batched_forward": ([_vp, _vp, _vp, _vp, _sz, _vp], _int),
    "slos_batched_autotune": ([_vp, _vp, _vp, _vp, _sz, ctypes.c_char_p, _vp], _int),
    "slos_batched_inject_stall": ([_vp, _int], _int),
    "slos_host_rank": ([_int, ctypes.POINTER(_int)], _i64),
    "slos_host_unrank": ([_int, _int, _i64, ctypes.POINTER(_int)], _int),
    "slos_device_index_table": ([_int, _int, _i64, _i64, _vp, _vp, _vp], _int),
    "slos_host_transition_table": ([_int, _int, _vp, _vp, _vp], _int),
    "slos_host_validate_tables": ([_int, _int, _int, _vp, _vp], _int),
    "slos_inject_fault": ([_int, _int], _int),
    "slos_host_split_layer": ([_int, _int, _int, ctypes.POINTER(_int), _vp, _vp, _vp, _vp], _int),
    "slos_host_split_tail": ([_int, _int, ctypes.POINTER(_int), _vp, _vp, _vp], _int),
    "slos_noalloc_scratch_bytes": ([], _sz),
    "slos_forward_noalloc": ([_vp, _vp, _int, _int, _vp, _vp], _int),
    "slos_profile_enable": ([_int], _int),
    "slos_profile_reset": ([], _int),
    "slos_launch_count": ([], _i64),
    "slos_profile_collect": ([], _int),
    "slos_profile_entry": ([_int, ctypes.c_char_p, _sz, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double)], _int),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libslos.so (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libslos.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGNATURES)


def _check(status: int):
    if status != 0:
        raise SlosError(status, load().slos_last_error().decode())


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t: torch.Tensor, dtype, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


# ------------------------------------------------------------------ mesh

def mesh_unitary(m: int, theta: torch.Tensor, data: torch.Tensor | None, batch: int, data_col: int | None = None,
                 out: torch.Tensor | None = None, stream=None, w: torch.Tensor | None = None) -> torch.Tensor:
    """theta: float32 [P] (shared) or [B, P]; data: float32 [B, n_data] or
    None.  With w (float32 [n_data]) the data phases are data * w, formed in
    the kernel (mesh_unitary_weighted)."""
    lib = load()
    _need(theta, torch.float32, "theta")
    n_data = 0 if data is None else data.shape[-1]
    if data is not None:
        _need(data, torch.float32, "data")
    if w is not None:
        _need(w, torch.float32, "w")
        if data is None or w.numel() < n_data:
            raise ValueError("w needs one weight per data phase")
    desc = MeshDesc(m, n_data, m // 2 if data_col is None else data_col)
    if out is None:
        out = torch.empty((batch, m, m), dtype=torch.complex64, device=theta.device)
    ts = 0 if theta.dim() == 1 else theta.shape[-1]
    ds = 0 if data is None else data.shape[-1]
    if w is None:
        _check(lib.mesh_unitary(ctypes.byref(desc), _ptr(theta), ts, _ptr(data), ds, batch, _ptr(out),
                                _stream(stream)))
    else:
        _check(lib.mesh_unitary_weighted(ctypes.byref(desc), _ptr(theta), ts, _ptr(data), ds, _ptr(w), batch,
                                         _ptr(out), _stream(stream)))
    return out


def mesh_unitary_backward(m: int, theta, data, batch: int, dU: torch.Tensor, data_col=None, stream=None,
                          w: torch.Tensor | None = None, need_dw: bool = False):
    """(dtheta, ddata) or, with need_dw, (dtheta, ddata, dw per instance)."""
    lib = load()
    _need(dU, torch.complex64, "dU")
    n_data = 0 if data is None else data.shape[-1]
    desc = MeshDesc(m, n_data, m // 2 if data_col is None else data_col)
    shared = theta.dim() == 1
    ts = 0 if shared else theta.shape[-1]
    P = m * (m - 1)
    dtheta = torch.empty((P,) if shared else (batch, P), dtype=torch.float32, device=dU.device)
    ddata = torch.empty((batch, n_data), dtype=torch.float32, device=dU.device) if n_data else None
    dw = torch.empty((batch, n_data), dtype=torch.float32, device=dU.device) if (n_data and need_dw) else None
    nbytes = ctypes.c_size_t()
    _check(lib.mesh_unitary_backward_workspace(ctypes.byref(desc), batch, ts, ctypes.byref(nbytes)))
    ws = torch.empty(max(1, nbytes.value), dtype=torch.uint8, device=dU.device)
    ds = 0 if data is None else data.shape[-1]
    if w is None:
        _check(lib.mesh_unitary_backward(ctypes.byref(desc), _ptr(theta), ts, _ptr(data), ds, batch, _ptr(dU),
                                         _ptr(dtheta), _ptr(ddata), _ptr(ws), nbytes.value, _stream(stream)))
    else:
        _check(lib.mesh_unitary_weighted_backward(ctypes.byref(desc), _ptr(theta), ts, _ptr(data), ds, _ptr(w), batch,
                                                  _ptr(dU), _ptr(dtheta), _ptr(ddata), _ptr(dw), _ptr(ws),
                                                  nbytes.value, _stream(stream)))
    return (dtheta, ddata, dw) if need_dw else (dtheta, ddata)


def mesh_sum_rows(rows: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """mesh_sum_rows: float32 [batch, width] -> [width], the batch sum in a fixed order."""
    _need(rows, torch.float32, "rows")
    if rows.dim() != 2:
        raise ValueError("rows must be [batch, width]")
    batch, width = rows.shape
    if out is None:
        out = torch.empty(width, dtype=torch.float32, device=rows.device)
    _check(load().mesh_sum_rows(_ptr(rows), batch, width, _ptr(out), _stream(stream)))
    return out


def fidelity_kernel(input_state, Ua: torch.Tensor, Ub: torch.Tensor | None = None, out=None, stream=None):
    """K[i][j] = |<s|Ua[i]^dag Ub[j]|s>|^2 for unitaries [Na, m, m] and
    [Nb, m, m] (Ub = Ua: the Gram matrix)."""
    _need(Ua, torch.complex64, "Ua")
    Ub = Ua if Ub is None else Ub
    _need(Ub, torch.complex64, "Ub")
    m = Ua.shape[-1]
    s = [int(x) for x in input_state]
    if len(s) != m:
        raise ValueError("input_state needs one occupation per mode")
    K = torch.empty((Ua.shape[0], Ub.shape[0]), dtype=torch.float32, device=Ua.device) if out is None else out
    arr = (ctypes.c_int * m)(*s)
    _check(load().slos_fidelity_kernel(m, arr, _ptr(Ua), Ua.shape[0], _ptr(Ub), Ub.shape[0], _ptr(K),
                                       _stream(stream)))
    return K


# ------------------------------------------------------------------ plans

class Plan:
    """Owns a slos_plan_t for one (m, n, input state, detection, computation
    space)."""

    def __init__(self, m: int, input_state, detection: int = PNR, mem_budget_bytes: int = 0, space: int = FOCK):
        lib = load()
        s = [int(x) for x in input_state]
        assert len(s) == m
        self.m, self.n, self.input_state, self.detection, self.space = m, sum(s), s, detection, space
        arr = (ctypes.c_int * m)(*s)
        h = ctypes.c_void_p()
        _check(lib.slos_plan_space(m, self.n, arr, detection, space, mem_budget_bytes, ctypes.byref(h)))
        self._h = h
        K, F, st = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib.slos_plan_query(h, ctypes.byref(K), ctypes.byref(F), ctypes.byref(st)))
        self.n_outputs, self.fock_dim, self.checkpoint_stride = K.value, F.value, st.value

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self, batch: int, training: bool) -> int:
        b = ctypes.c_size_t()
        _check(load().slos_workspace_bytes(self._h, batch, 1 if training else 0, ctypes.byref(b)))
        return b.value

    def workspace(self, batch: int, training: bool, device="cuda") -> torch.Tensor:
        return torch.empty(max(1, self.workspace_bytes(batch, training)), dtype=torch.uint8, device=device)

    def _check_io(self, U: torch.Tensor, out: torch.Tensor | None, output: int):
        """U complex64 [B, m, m]; out (if given) float32 (probabilities) or
        complex64 (amplitudes) [B, n_outputs], contiguous, on U's device."""
        _need(U, torch.complex64, "U")
        if U.dim() != 3 or U.shape[1] != self.m or U.shape[2] != self.m:
            raise ValueError(f"U must be [B, {self.m}, {self.m}], got {tuple(U.shape)}")
        if out is not None:
            _need(out, torch.complex64 if output == AMPS else torch.float32, "out")
            if tuple(out.shape) != (U.shape[0], self.n_outputs):
                raise ValueError(f"out must be [{U.shape[0]}, {self.n_outputs}], got {tuple(out.shape)}")
            if out.device != U.device:
                raise ValueError("U and out must be on the same device")

    def forward(self, U: torch.Tensor, output: int = PROBS, save_for_backward: bool = False,
                workspace: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None):
        self._check_io(U, out, output)
        B = U.shape[0]
        if workspace is None:
            workspace = self.workspace(B, save_for_backward, U.device)
        if out is None:
            dt = torch.complex64 if output == AMPS else torch.float32
            out = torch.empty((B, self.n_outputs), dtype=dt, device=U.device)
        _check(load().slos_forward(self._h, _ptr(U), B, output, _ptr(out), 1 if save_for_backward else 0,
                                   _ptr(workspace), workspace.numel(), _stream(stream)))
        return out

    def expectations(self, probs: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Per-mode photon-number expectations (PNR) or click probabilities
        (threshold) of an output distribution [B, n_outputs] -> [B, m]."""
        _need(probs, torch.float32, "probs")
        B = probs.shape[0]
        if out is None:
            out = torch.empty((B, self.m), dtype=torch.float32, device=probs.device)
        _check(load().slos_expectations(self._h, _ptr(probs), B, _ptr(out), _stream(stream)))
        return out

    def expectations_backward(self, dout: torch.Tensor, dprobs: torch.Tensor | None = None, stream=None):
        _need(dout, torch.float32, "dout")
        B = dout.shape[0]
        if dprobs is None:
            dprobs = torch.empty((B, self.n_outputs), dtype=torch.float32, device=dout.device)
        _check(load().slos_expectations_backward(self._h, _ptr(dout), B, _ptr(dprobs), _stream(stream)))
        return dprobs

    def renormalise(self, p: torch.Tensor, q: torch.Tensor | None = None, Z: torch.Tensor | None = None,
                    stream=None):
        """q = p / sum_t p (per instance) and the sums Z."""
        _need(p, torch.float32, "p")
        B = p.shape[0]
        q = torch.empty_like(p) if q is None else q
        Z = torch.empty(B, dtype=torch.float32, device=p.device) if Z is None else Z
        _check(load().slos_renormalise(self._h, _ptr(p), B, _ptr(q), _ptr(Z), _stream(stream)))
        return q, Z

    def renormalise_backward(self, q: torch.Tensor, Z: torch.Tensor, dq: torch.Tensor,
                             dp: torch.Tensor | None = None, stream=None):
        for t, nm in ((q, "q"), (Z, "Z"), (dq, "dq")):
            _need(t, torch.float32, nm)
        dp = torch.empty_like(dq) if dp is None else dp
        _check(load().slos_renormalise_backward(self._h, _ptr(q), _ptr(Z), _ptr(dq), q.shape[0], _ptr(dp),
                                                _stream(stream)))
        return dp

    def sample(self, probs: torch.Tensor, uniforms: torch.Tensor, counts: bool = False, stream=None):
        """Shots from distributions [B, n_outputs] driven by draws [B, shots]
        in [0, 1): returns int32 outcome indices [B, shots] (and int32
        counts [B, n_outputs] when counts=True)."""
        _need(probs, torch.float32, "probs")
        _need(uniforms, torch.float32, "uniforms")
        B, S = uniforms.shape
        if probs.shape[0] != B:
            raise ValueError("probs and uniforms need the same batch")
        nb = ctypes.c_size_t()
        _check(load().slos_sample_workspace_bytes(self._h, B, ctypes.byref(nb)))
        ws = torch.empty(max(1, nb.value), dtype=torch.uint8, device=probs.device)
        samples = torch.empty((B, S), dtype=torch.int32, device=probs.device)
        cnt = torch.empty((B, self.n_outputs), dtype=torch.int32, device=probs.device) if counts else None
        _check(load().slos_sample(self._h, _ptr(probs), B, S, _ptr(uniforms), _ptr(samples), _ptr(cnt), _ptr(ws),
                                  ws.numel(), _stream(stream)))
        return (samples, cnt) if counts else samples

    def encoded_workspace_bytes(self) -> int:
        nb = ctypes.c_size_t()
        _check(load().slos_encoded_workspace_bytes(self._h, ctypes.byref(nb)))
        return nb.value

    def encoded_forward(self, U: torch.Tensor, X: torch.Tensor, output: int = PROBS, out=None, workspace=None,
                        stream=None):
        """Amplitude-encoded inputs X [B, n_outputs] (complex64 state vectors
        over this plan's basis) through one unitary U [m, m]."""
        _need(U, torch.complex64, "U")
        _need(X, torch.complex64, "X")
        Bn = X.shape[0]
        if workspace is None:
            nb = ctypes.c_size_t()
            _check(load().slos_encoded_workspace_bytes(self._h, ctypes.byref(nb)))
            workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=X.device)
        if out is None:
            dt = torch.complex64 if output == AMPS else torch.float32
            out = torch.empty((Bn, self.n_outputs), dtype=dt, device=X.device)
        _check(load().slos_encoded_forward(self._h, _ptr(U), _ptr(X), Bn, output, _ptr(out), _ptr(workspace),
                                           workspace.numel(), _stream(stream)))
        return out

    def forward_noalloc(self, U: torch.Tensor, out: torch.Tensor, output: int = PROBS, stream=None):
        """slos_forward_noalloc: the library's built-in scratch, no workspace."""
        self._check_io(U, out, output)
        _check(load().slos_forward_noalloc(self._h, _ptr(U), U.shape[0], output, _ptr(out), _stream(stream)))
        return out

    def backward(self, U: torch.Tensor, dout: torch.Tensor, workspace: torch.Tensor, output: int = PROBS,
                 dU: torch.Tensor | None = None, stream=None):
        """dout: [B, K] or [K] (shared by the batch, stride 0)."""
        B = U.shape[0]
        stride = 0 if dout.dim() == 1 else dout.shape[-1]
        if not dout.is_contiguous():
            raise ValueError("dout must be contiguous")
        if dU is None:
            dU = torch.empty_like(U)
        _check(load().slos_backward(self._h, _ptr(U), B, output, _ptr(dout), stride, _ptr(dU), _ptr(workspace),
                                    workspace.numel(), _stream(stream)))
        return dU

    def sync_status(self, stream=None):
        _check(load().slos_sync_status(self._h, _stream(stream)))

    def autotune(self, U: torch.Tensor, cache_path: str | None = None, stream=None) -> dict:
        """slos_autotune for U's batch: times forward(save) + backward over the
        candidate launch shapes (buffers allocated here) and keeps the fastest."""
        _need(U, torch.complex64, "U")
        B = U.shape[0]
        ws = self.workspace(B, training=True, device=U.device)
        out = torch.empty((B, self.n_outputs), dtype=torch.float32, device=U.device)
        dout = torch.ones(self.n_outputs, dtype=torch.float32, device=U.device)
        dU = torch.empty_like(U)
        path = cache_path.encode() if cache_path else None
        _check(load().slos_autotune(self._h, _ptr(U), B, _ptr(out), _ptr(dout), _ptr(dU), _ptr(ws), ws.numel(), path,
                                    _stream(stream)))
        return self.tuning()

    def tuning(self) -> dict:
        v = [_int() for _ in range(4)]
        _check(load().slos_plan_tuning(self._h, *[ctypes.byref(x) for x in v]))
        return {"prefix_layers": v[0].value, "prefix_ni": v[1].value, "fwd_blocks_per_sm": v[2].value,
                "bwd_blocks_per_sm": v[3].value}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.slos_plan_destroy(h)
            self._h = None


class BatchedPlan:
    """Uneven batch of (m_i, n_i, input_i, detection_i) instances."""

    def __init__(self, ms, ns, inputs, detections):
        lib = load()
        cnt = len(ms)
        self.count = cnt
        m_arr = (ctypes.c_int * cnt)(*ms)
        n_arr = (ctypes.c_int * cnt)(*ns)
        d_arr = (ctypes.c_int * cnt)(*detections)
        self._rows = [(ctypes.c_int * len(s))(*s) for s in inputs]
        rows = (ctypes.POINTER(ctypes.c_int) * cnt)(*[ctypes.cast(r, ctypes.POINTER(ctypes.c_int)) for r in self._rows])
        h = ctypes.c_void_p()
        _check(lib.slos_batched_plan(cnt, m_arr, n_arr, rows, d_arr, ctypes.byref(h)))
        self._h = h
        uo = (ctypes.c_int64 * (cnt + 1))()
        oo = (ctypes.c_int64 * (cnt + 1))()
        wb = ctypes.c_size_t()
        _check(lib.slos_batched_query(h, uo, oo, ctypes.byref(wb)))
        self.u_offsets = list(uo)
        self.out_offsets = list(oo)
        self.workspace_bytes = wb.value

    def forward(self, U_packed, out_packed, workspace, stream=None):
        _check(load().slos_batched_forward(self._h, _ptr(U_packed), _ptr(out_packed), _ptr(workspace),
                                           workspace.numel(), _stream(stream)))
        return out_packed

    def autotune(self, U_packed, out_packed, workspace, cache_path=None, stream=None):
        cp = cache_path.encode() if cache_path else None
        _check(load().slos_batched_autotune(self._h, _ptr(U_packed), _ptr(out_packed), _ptr(workspace),
                                            workspace.numel(), cp, _stream(stream)))

    def sync_status(self, stream=None):
        _check(load().slos_sync_status(self._h, _stream(stream)))

    def inject_stall(self, enable: bool):
        _check(load().slos_batched_inject_stall(self._h, 1 if enable else 0))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.slos_plan_destroy(h)
            self._h = None


# ------------------------------------------------------------------ index tables

def host_rank(m: int, t) -> int:
    arr = (ctypes.c_int * m)(*[int(x) for x in t])
    return load().slos_host_rank(m, arr)


def host_unrank(m: int, k: int, rank: int):
    arr = (ctypes.c_int * m)()
    _check(load().slos_host_unrank(m, k, rank, arr))
    return list(arr)


def host_transition_table(m: int, k: int):
    """(rowptr, entries, ctab) numpy arrays of layer k, built by the library."""
    import math
    import numpy as np
    Fk, Fp = math.comb(m + k - 1, k), math.comb(m + k - 2, k - 1)
    rowptr = np.zeros(Fk + 1, dtype=np.int32)
    entries = np.zeros(m * Fp, dtype=np.uint32)
    ctab = np.zeros(Fp * m, dtype=np.int32)
    _check(load().slos_host_transition_table(m, k, rowptr.ctypes.data, entries.ctypes.data, ctab.ctypes.data))
    return rowptr, entries, ctab.reshape(Fp, m)


def host_split_layer(m: int, n: int, k: int):
    """Backward split-lattice tables of layer k (parents in layer k-1) as
    numpy arrays (dict), built by the library."""
    import numpy as np
    lib = load()
    h = _int()
    counts = np.zeros(2, dtype=np.int64)
    _check(lib.slos_host_split_layer(m, n, k, ctypes.byref(h), counts.ctypes.data, None, None, None))
    nb, nbc = (int(x) for x in counts)
    out = {"h": h.value, "bdesc": np.zeros((nb, 4), dtype=np.int32), "bhead": np.zeros((nb, 8), dtype=np.int32),
           "bchunk": np.zeros(nbc, dtype=np.int32)}
    _check(lib.slos_host_split_layer(m, n, k, ctypes.byref(h), counts.ctypes.data,
                                     *(out[key].ctypes.data for key in ("bdesc", "bhead", "bchunk"))))
    return out


def host_split_tail(m: int, n: int):
    """Tail child table of the split lattice (dict of numpy arrays), built by the library."""
    import numpy as np
    lib = load()
    h = _int()
    offsets = np.zeros(n + 1, dtype=np.int32)
    count = np.zeros(1, dtype=np.int64)
    _check(lib.slos_host_split_tail(m, n, ctypes.byref(h), offsets.ctypes.data, count.ctypes.data, None))
    ctab = np.zeros(int(count[0]), dtype=np.uint16)
    _check(lib.slos_host_split_tail(m, n, ctypes.byref(h), offsets.ctypes.data, count.ctypes.data,
                                    ctab.ctypes.data))
    return {"h": h.value, "coff": offsets, "ctab": ctab}


def device_index_table(m: int, k: int, first: int, count: int, device="cuda", stream=None):
    comp = torch.empty((count, m), dtype=torch.uint8, device=device)
    par = torch.empty((count, m), dtype=torch.int32, device=device)
    _check(load().slos_device_index_table(m, k, first, count, _ptr(comp), _ptr(par), _stream(stream)))
    return comp, par


# ------------------------------------------------------------------ tracing

def profile_enable(on: bool = True):
    _check(load().slos_profile_enable(1 if on else 0))


def profile_reset():
    _check(load().slos_profile_reset())


def launch_count() -> int:
    return int(load().slos_launch_count())


def profile_collect() -> dict:
    """{kernel name: (launches, total_ms, total_algorithmic_bytes)}"""
    lib = load()
    n = lib.slos_profile_collect()
    out = {}
    buf = ctypes.create_string_buffer(128)
    for i in range(n):
        L, ms, by = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(lib.slos_profile_entry(i, buf, 128, ctypes.byref(L), ctypes.byref(ms), ctypes.byref(by)))
        out[buf.value.decode()] = (L.value, ms.value, by.value)
    return out
