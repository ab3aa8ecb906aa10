"""ctypes binding of include/surrogate.h (argument marshalling only) and the
surrogate driver: tensor-core MLP inference with an exact SLOS spot check and
exact fallback (the exact path checks the surrogate's total variation)."""
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
    "surr_set_input_harmonics": ([_vp, _int], _int),
    "surr_forward": ([_vp, _vp, _int, _vp, _vp], _int),
    "surr_train_step": ([_vp, _vp, _vp, _int, _f, _vp, _vp], _int),
    "surr_get_param": ([_vp, _int, _vp, _vp], _int),
    "surr_set_param": ([_vp, _int, _vp, _vp], _int),
    "surr_get_grad": ([_vp, _int, _vp, _vp], _int),
    "surr_save": ([_vp, ctypes.c_char_p, _i64], _int),
    "surr_load": ([_vp, ctypes.c_char_p, ctypes.POINTER(_i64)], _int),
    "surr_tv_rows": ([_vp, _vp, _vp, _int, _int, _vp, _vp], _int),
    "surr_screen": ([_vp, _int, _int, _vp, _int, _vp, ctypes.POINTER(_int), _f, _vp, _vp, _vp], _int),
    "surr_scatter_rows": ([_vp, _vp, _int, _int, _vp, _vp], _int),
    "surr_gather_rows": ([_vp, _vp, _int, _int, _vp, _vp], _int),
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

    def set_input_harmonics(self, harmonics: int):
        """Inputs become n_phases / harmonics values x per row; the model's
        phases h * x (h = 1..harmonics) are formed in its feature kernel."""
        B._check(lib().surr_set_input_harmonics(self._h, int(harmonics)))

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

    def save(self, path: str, stream_index: int = 0):
        """Checkpoint weights, Adam state and the caller's data-stream position."""
        B._check(lib().surr_save(self._h, str(path).encode(), int(stream_index)))

    def load(self, path: str) -> int:
        """Restore a checkpoint; returns the data-stream position saved with it."""
        idx = ctypes.c_int64()
        B._check(lib().surr_load(self._h, str(path).encode(), ctypes.byref(idx)))
        return idx.value

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


# ---------------------------------------------------------------------- driver

class SurrogateLayer:
    """Surrogate of the m=12, n=6 layer (132 shared trainable phases + 12
    data phases x*w), trained on exact SLOS distributions; at inference the
    exact path screens every sample, spot-checks a seeded fraction and
    replaces every sample that fails (total variation > tv_tol)."""

    def __init__(self, hidden=2048, n_hidden_layers=4, max_batch=4096, seed=1004, device="cuda"):
        import numpy as np

        from . import workloads
        w = workloads.layer12(batch=1)
        self.m, self.n, self.s = 12, 6, w["s"]
        mb = w["mesh"]
        self.device = torch.device(device)
        self.theta = torch.tensor(mb.theta, dtype=torch.float32, device=self.device)
        self.wdata = mb.w
        self.plan = B.Plan(self.m, self.s)
        self.K = self.plan.n_outputs
        self.harmonics = 12
        self.model = Surrogate(n_phases=self.harmonics * self.m, hidden=hidden,
                               n_hidden_layers=n_hidden_layers, n_outputs=self.K, max_batch=max_batch, seed=seed)
        self.model.set_input_harmonics(self.harmonics)
        self.max_batch = max_batch
        occ, _ = B.device_index_table(self.m, self.n, 0, self.K, device=self.device)
        self.occ = occ
        self._np = np

    # data phases x*w for a seeded stream of samples
    def sample_data(self, count: int, rng):
        x = rng.standard_normal((count, self.m))
        return torch.tensor(x * self.wdata[None, :], dtype=torch.float32, device=self.device)

    # The model's 144 phase inputs are h * x_j for the harmonics h = 1..12 of
    # the 12 data phases x_j (it takes sin and cos of each), formed by the
    # model's feature kernel from the data phases.  The 132 trainable phases
    # are the same for every sample and carry nothing; the data phases sit in
    # one column between the two halves of the mesh, so every amplitude is a
    # homogeneous polynomial of degree n = 6 in the e^{i x_j} and each
    # probability a trigonometric polynomial of degree <= 6 in every x_j: its
    # harmonics are the natural inputs.

    def exact(self, data: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        U = B.mesh_unitary(self.m, self.theta, data.contiguous(), data.shape[0])
        return self.plan.forward(U, out=out)

    def train(self, n_samples: int, batch: int = 4096, lr: float = 1e-3, seed: int = 1004, lr_min: float = 1e-5):
        import math
        rng = self._np.random.default_rng(seed)
        steps = max(1, n_samples // batch)
        losses = torch.zeros(batch, dtype=torch.float32, device=self.device)
        hist = []
        for it in range(steps):
            data = self.sample_data(batch, rng)
            p = self.exact(data)
            cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * it / steps))
            self.model.train_step(data, p, cur, losses)
            if it % max(1, steps // 20) == 0 or it == steps - 1:
                hist.append((it, float(losses.mean().item())))
        sync_status()
        return hist

    def evaluate(self, count: int = 10000, seed: int = 1005, batch: int = 2048):
        """Held-out total variation of the bare surrogate against exact SLOS."""
        rng = self._np.random.default_rng(seed)
        tvs = []
        L = lib()
        for off in range(0, count, batch):
            nb = min(batch, count - off)
            nb8 = (nb + 7) // 8 * 8
            data = self.sample_data(nb8, rng)
            q = self.model.forward(data)
            p = self.exact(data)
            rows = torch.arange(nb8, dtype=torch.int32, device=self.device)
            tv = torch.empty(nb8, dtype=torch.float32, device=self.device)
            B._check(L.surr_tv_rows(B._ptr(q), B._ptr(rows), B._ptr(p), nb8, self.K, B._ptr(tv), B._stream()))
            tvs.append(tv[:nb].cpu().numpy())
        tv = self._np.concatenate(tvs)
        return {"p50": float(self._np.median(tv)), "p99": float(self._np.percentile(tv, 99)), "max": float(tv.max()),
                "frac_gt_0.02": float((tv > 0.02).mean()), "count": int(tv.size)}

    @staticmethod
    def failure_rate_bound(failures: int, checked: int, confidence: float = 0.99) -> float:
        """One-sided exact (Clopper-Pearson) upper confidence bound on a
        binomial rate: the largest rate under which observing at most
        `failures` in `checked` independent draws still has probability
        >= 1 - confidence (bisection on the binomial distribution function)."""
        import math
        if checked <= 0 or failures >= checked:
            return 1.0
        alpha = 1.0 - confidence

        def cdf(r):
            return sum(math.comb(checked, k) * r ** k * (1.0 - r) ** (checked - k) for k in range(failures + 1))

        lo, hi = failures / checked, 1.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if cdf(mid) > alpha:
                lo = mid
            else:
                hi = mid
        return hi

    def infer(self, data: torch.Tensor, rho: float = 1 / 64, tv_tol: float = 0.02, seed: int = 0,
              max_fail_rate: float = 0.01, confidence: float = 0.99):
        """Surrogate outputs with the exact path as arbiter.

        1. Spot-check first: a seeded fraction rho of the samples runs through
           both the surrogate and the exact path, and the batch's failure
           rate (TV > tv_tol) is bounded from above at the given confidence.
        2. If that bound exceeds max_fail_rate, the whole batch takes the exact
           path; the surrogate never runs on the rest.
        3. Otherwise the surrogate runs on every sample, and every sample is
           screened: its per-mode mean photon numbers against the exact ones
           (closed form); a screened-out sample provably has TV > tv_tol.
           Screened-out and failed samples take the exact path (a failed
           checked sample keeps its exact row), the rest keep the surrogate.

        Every returned row is therefore exact, or belongs to a batch whose
        unchecked rows exceed tv_tol at a rate <= max_fail_rate (with
        probability >= confidence).  When the surrogate cannot meet the bound
        the call costs the exact path plus the checked fraction."""
        L = lib()
        Bn = data.shape[0]
        rng = self._np.random.default_rng(seed)
        n_chk = max(1, int(round(rho * Bn)))
        chk = torch.tensor(self._np.sort(rng.choice(Bn, size=n_chk, replace=False)), dtype=torch.int32,
                           device=self.device)
        dchk = torch.empty((n_chk, self.m), dtype=torch.float32, device=self.device)
        B._check(L.surr_gather_rows(B._ptr(data), B._ptr(chk), n_chk, self.m, B._ptr(dchk), B._stream()))
        qchk = self.model.forward(dchk)
        pchk = self.exact(dchk)
        ident = torch.arange(n_chk, dtype=torch.int32, device=self.device)
        tv = torch.empty(n_chk, dtype=torch.float32, device=self.device)
        B._check(L.surr_tv_rows(B._ptr(qchk), B._ptr(ident), B._ptr(pchk), n_chk, self.K, B._ptr(tv), B._stream()))
        # decisions on the host
        tvh = tv.cpu().numpy()
        ch = chk.cpu().numpy()
        failed = int((tvh > tv_tol).sum())
        ucb = self.failure_rate_bound(failed, n_chk, confidence)
        batch_fallback = ucb > max_fail_rate
        screened = None
        if batch_fallback:
            q = self.exact(data)
            bad = self._np.arange(Bn)
        else:
            q = self.model.forward(data)
            U = B.mesh_unitary(self.m, self.theta, data, Bn)
            flag = torch.zeros(Bn, dtype=torch.int32, device=self.device)
            marg = torch.empty((Bn, self.m), dtype=torch.float32, device=self.device)
            s_host = (ctypes.c_int * self.m)(*self.s)
            B._check(L.surr_screen(B._ptr(q), Bn, self.K, B._ptr(self.occ), self.m, B._ptr(U), s_host,
                                   2.0 * self.n * tv_tol, B._ptr(marg), B._ptr(flag), B._stream()))
            fl = flag.cpu().numpy().astype(bool)
            screened = int(fl.sum())
            # checked samples keep their exact rows; screened-out ones are recomputed
            B._check(L.surr_scatter_rows(B._ptr(pchk), B._ptr(chk), n_chk, self.K, B._ptr(q), B._stream()))
            fl[ch] = False
            redo = self._np.nonzero(fl)[0]
            if redo.size:
                rows = torch.tensor(redo, dtype=torch.int32, device=self.device)
                dbad = torch.empty((redo.size, self.m), dtype=torch.float32, device=self.device)
                B._check(L.surr_gather_rows(B._ptr(data), B._ptr(rows), redo.size, self.m, B._ptr(dbad),
                                            B._stream()))
                pbad = self.exact(dbad)
                B._check(L.surr_scatter_rows(B._ptr(pbad), B._ptr(rows), redo.size, self.K, B._ptr(q), B._stream()))
            bad = self._np.union1d(redo, ch[tvh > tv_tol])
        stats = {"batch": Bn, "screen_flagged": screened, "checked": n_chk, "check_failed": failed,
                 "fail_rate_ucb": ucb, "max_fail_rate": max_fail_rate, "confidence": confidence,
                 "batch_fallback": bool(batch_fallback), "fallback": int(bad.size),
                 "fallback_rate": float(bad.size / Bn), "checked_tv_max": float(tvh.max()),
                 "surrogate_rows": n_chk + (0 if batch_fallback else Bn)}
        return q, stats
