"""torch.autograd.Functions over the C ABI (Sec. II-A.3: differentiable
simulation; Sec. II-B: the quantum layer as a composable module).

MeshFn  : (theta, data) -> U           via mesh_unitary / mesh_unitary_backward
SlosFn  : U -> probabilities or amps   via slos_forward / slos_backward
QuantumLayer: theta (trainable) and data phases x*w (formed in the mesh kernel)
-> output distribution.

The Functions only marshal arguments; all arithmetic is in libslos.so.
"""
from __future__ import annotations

import torch

from . import binding as B


class MeshFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, data, m, batch, data_col, w=None):
        theta = theta.contiguous()
        data = data.contiguous() if data is not None else None
        w = w.contiguous() if w is not None else None
        U = B.mesh_unitary(m, theta, data, batch, data_col, w=w)
        empty = torch.empty(0, device=theta.device)
        ctx.save_for_backward(theta, data if data is not None else empty, w if w is not None else empty)
        ctx.m, ctx.batch, ctx.data_col = m, batch, data_col
        ctx.has_data, ctx.has_w = data is not None, w is not None
        return U

    @staticmethod
    def backward(ctx, dU):
        theta, data, w = ctx.saved_tensors
        data = data if ctx.has_data else None
        w = w if ctx.has_w else None
        need_dw = w is not None and ctx.needs_input_grad[5]
        res = B.mesh_unitary_backward(ctx.m, theta, data, ctx.batch, dU.contiguous(), ctx.data_col, w=w,
                                      need_dw=need_dw)
        dw = B.mesh_sum_rows(res[2]) if need_dw else None  # per-instance rows, summed over the batch by the library
        return res[0], res[1], None, None, None, dw


class SlosFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, plan: B.Plan, output: int):
        U = U.contiguous()
        ws = plan.workspace(U.shape[0], training=True, device=U.device)
        out = plan.forward(U, output, save_for_backward=True, workspace=ws)
        ctx.save_for_backward(U)
        ctx.plan, ctx.ws, ctx.output = plan, ws, output
        return out

    @staticmethod
    def backward(ctx, dout):
        (U,) = ctx.saved_tensors
        if dout.dim() == 2 and dout.stride(0) == 0 and dout.stride(1) == 1:
            d = dout[0]  # the same gradient row for every instance (stride 0)
        else:
            d = dout.contiguous()
        if ctx.ws is None:
            raise RuntimeError("SlosFn: a second backward through the same forward is not supported (its activations "
                               "were released by the first backward); run the forward again")
        dU = ctx.plan.backward(U, d, ctx.ws, ctx.output)
        ctx.ws = None
        return dU, None, None


class ExpectationFn(torch.autograd.Function):
    """probabilities [B, K] -> per-mode expectations [B, m]."""

    @staticmethod
    def forward(ctx, probs, plan: B.Plan):
        ctx.plan = plan
        return plan.expectations(probs.contiguous())

    @staticmethod
    def backward(ctx, dout):
        return ctx.plan.expectations_backward(dout.contiguous()), None


class RenormaliseFn(torch.autograd.Function):
    """p [B, K] -> p / sum_t p: the distribution conditioned on the plan's space."""

    @staticmethod
    def forward(ctx, p, plan: B.Plan):
        q, Z = plan.renormalise(p.contiguous())
        ctx.save_for_backward(q, Z)
        ctx.plan = plan
        return q

    @staticmethod
    def backward(ctx, dq):
        q, Z = ctx.saved_tensors
        return ctx.plan.renormalise_backward(q, Z, dq.contiguous()), None


def mesh_unitary(theta, data, m: int, batch: int, data_col: int | None = None, w=None):
    """U(theta, data) with data phases data (or data * w, formed in the kernel)."""
    return MeshFn.apply(theta, data, m, batch, m // 2 if data_col is None else data_col, w)


def slos(U, plan: B.Plan, output: int = B.PROBS):
    return SlosFn.apply(U, plan, output)


class QuantumLayer(torch.nn.Module):
    """U(x, theta) = W2(theta2) S(x) W1(theta1) followed by the SLOS output
    of a fixed Fock input (Sec. II-B, Sec. II-C.1).

    space: FOCK or UNBUNCHED (collision-free outputs only); renormalise:
    condition the distribution on the space (divide by its total);
    measurement: "probs" (the distribution), "expectations" (per-mode photon
    numbers, or click probabilities under threshold detection) or "amps"."""

    def __init__(self, m: int, input_state, detection: int = B.PNR, output: int = B.PROBS,
                 mem_budget_bytes: int = 0, theta: torch.Tensor | None = None, w: torch.Tensor | None = None,
                 device="cuda", space: int = B.FOCK, renormalise: bool = False, measurement: str | None = None):
        super().__init__()
        self.m = m
        self.plan = B.Plan(m, input_state, detection, mem_budget_bytes, space)
        if measurement is None:
            measurement = "amps" if output == B.AMPS else "probs"
        if measurement not in ("probs", "expectations", "amps"):
            raise ValueError("measurement must be 'probs', 'expectations' or 'amps'")
        if measurement == "amps" and renormalise:
            raise ValueError("renormalisation applies to distributions")
        self.measurement, self.renormalise = measurement, renormalise
        self.output = B.AMPS if measurement == "amps" else B.PROBS
        P = m * (m - 1)
        if theta is None:
            theta = torch.rand(P, device=device) * 2 * torch.pi
        self.theta = torch.nn.Parameter(theta.to(device=device, dtype=torch.float32))
        if w is None:
            w = torch.ones(m, device=device)
        self.register_buffer("w", w.to(device=device, dtype=torch.float32))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        x = x.to(torch.float32).contiguous()
        U = mesh_unitary(self.theta, x, self.m, x.shape[0], w=self.w[: x.shape[-1]].contiguous())
        y = slos(U, self.plan, self.output)
        if self.renormalise:
            y = RenormaliseFn.apply(y, self.plan)
        if self.measurement == "expectations":
            y = ExpectationFn.apply(y, self.plan)
        return y


class FidelityKernel(torch.nn.Module):
    """k(x1, x2) = |<s|U(x1)^dag U(x2)|s>|^2 with U(x) = W2(theta) S(x w)
    W1(theta) (the angle-encoding circuit): kernel(X) gives the Gram matrix,
    kernel(X1, X2) the cross kernel (kernel-methods section)."""

    def __init__(self, m: int, input_state, theta: torch.Tensor | None = None, w: torch.Tensor | None = None,
                 device="cuda"):
        super().__init__()
        self.m, self.input_state = m, [int(x) for x in input_state]
        P = m * (m - 1)
        if theta is None:
            theta = torch.rand(P, device=device) * 2 * torch.pi
        self.register_buffer("theta", theta.to(device=device, dtype=torch.float32))
        if w is None:
            w = torch.ones(m, device=device)
        self.register_buffer("w", w.to(device=device, dtype=torch.float32))

    def unitaries(self, x: torch.Tensor) -> torch.Tensor:
        x = x.to(torch.float32).contiguous()
        return B.mesh_unitary(self.m, self.theta, x, x.shape[0], w=self.w[: x.shape[-1]].contiguous())

    @torch.no_grad()
    def forward(self, x1: torch.Tensor, x2: torch.Tensor | None = None) -> torch.Tensor:
        U1 = self.unitaries(x1)
        U2 = U1 if x2 is None else self.unitaries(x2)
        return B.fidelity_kernel(self.input_state, U1, U2)
