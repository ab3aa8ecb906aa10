"""torch.autograd.Functions over the C ABI (Sec. II-A.3: differentiable
simulation; Sec. II-B: the quantum layer as a composable module).

MeshFn  : (theta, data) -> U           via mesh_unitary / mesh_unitary_backward
SlosFn  : U -> probabilities or amps   via slos_forward / slos_backward
QuantumLayer: theta (trainable) and data phases x*w -> output distribution.

The Functions only marshal arguments; all arithmetic is in libslos.so.
"""
from __future__ import annotations

import torch

from . import binding as B


class MeshFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, data, m, batch, data_col):
        theta = theta.contiguous()
        data = data.contiguous() if data is not None else None
        U = B.mesh_unitary(m, theta, data, batch, data_col)
        ctx.save_for_backward(theta, data if data is not None else torch.empty(0, device=theta.device))
        ctx.m, ctx.batch, ctx.data_col, ctx.has_data = m, batch, data_col, data is not None
        return U

    @staticmethod
    def backward(ctx, dU):
        theta, data = ctx.saved_tensors
        data = data if ctx.has_data else None
        dtheta, ddata = B.mesh_unitary_backward(ctx.m, theta, data, ctx.batch, dU.contiguous(), ctx.data_col)
        return dtheta, ddata, None, None, None


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
        dU = ctx.plan.backward(U, d, ctx.ws, ctx.output)
        ctx.ws = None
        return dU, None, None


def mesh_unitary(theta, data, m: int, batch: int, data_col: int | None = None):
    return MeshFn.apply(theta, data, m, batch, m // 2 if data_col is None else data_col)


def slos(U, plan: B.Plan, output: int = B.PROBS):
    return SlosFn.apply(U, plan, output)


class QuantumLayer(torch.nn.Module):
    """U(x, theta) = W2(theta2) S(x) W1(theta1) followed by the SLOS output
    distribution of a fixed Fock input (Sec. II-B, Sec. II-C.1)."""

    def __init__(self, m: int, input_state, detection: int = B.PNR, output: int = B.PROBS,
                 mem_budget_bytes: int = 0, theta: torch.Tensor | None = None, w: torch.Tensor | None = None,
                 device="cuda"):
        super().__init__()
        self.m = m
        self.plan = B.Plan(m, input_state, detection, mem_budget_bytes)
        self.output = output
        P = m * (m - 1)
        if theta is None:
            theta = torch.rand(P, device=device) * 2 * torch.pi
        self.theta = torch.nn.Parameter(theta.to(device=device, dtype=torch.float32))
        if w is None:
            w = torch.ones(m, device=device)
        self.register_buffer("w", w.to(device=device, dtype=torch.float32))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        data = (x * self.w[None, : x.shape[-1]]).to(torch.float32)
        U = mesh_unitary(self.theta, data, self.m, x.shape[0])
        return slos(U, self.plan, self.output)
