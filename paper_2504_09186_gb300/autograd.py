"""torch.autograd support: amplitudes as a differentiable function of the gate matrices.

Forward runs the planned contraction (complex64 path) with the given gate values; backward
runs the adjoint contraction (tnc_adjoint), which returns E_g = sum_b w_b d amp_b / dU_g
(holomorphic derivative).  PyTorch's gradient of a real loss with respect to a complex
input is conj(dL/dz) for holomorphic maps, so with the upstream gradient g (grad_output)
the weights are w = conj(g) and the returned gradient is conj(E).  Gradients through gate
parameters (e.g. fSim angles) follow from building the matrices with torch operations.
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np
import torch

from .tnc import Context, Plan


class Amplitudes(torch.autograd.Function):
    """amps = Amplitudes.apply(plan, ctx, bitstrings, arities, *gates)

    gates: one complex128 tensor per gate, d x d (U[out, in]); returns (batch, 2^n_open)
    complex128 amplitudes summed over every slice.
    """

    @staticmethod
    def forward(fctx, plan: Plan, ctx: Context, bitstrings: Optional[np.ndarray], arities: List[int], *gates):
        plan.update_gates([g.detach().cpu().numpy() for g in gates])
        amps = ctx.amplitudes(plan, bitstrings, "c64")
        fctx.plan, fctx.ctx, fctx.bits, fctx.arities = plan, ctx, bitstrings, list(arities)
        fctx.devices = [g.device for g in gates]
        return torch.from_numpy(amps)

    @staticmethod
    def backward(fctx, grad_out):
        w = np.conj(grad_out.detach().cpu().numpy())
        env, _ = fctx.ctx.adjoint(fctx.plan, fctx.bits, w, fctx.arities)
        grads = [torch.from_numpy(np.conj(e)).to(dev) for e, dev in zip(env, fctx.devices)]
        return (None, None, None, None, *grads)


def amplitudes(plan: Plan, ctx: Context, bitstrings, arities, gates) -> torch.Tensor:
    return Amplitudes.apply(plan, ctx, bitstrings, arities, *gates)


def fsim_torch(theta: torch.Tensor, phi: torch.Tensor) -> torch.Tensor:
    """fSim(theta, phi) built from torch ops (differentiable in the angles)."""
    c = torch.cos(theta).to(torch.complex128)
    s = torch.sin(theta).to(torch.complex128)
    one = torch.ones((), dtype=torch.complex128)
    zero = torch.zeros((), dtype=torch.complex128)
    e = torch.exp(-1j * phi.to(torch.complex128))
    rows = [
        torch.stack([one, zero, zero, zero]),
        torch.stack([zero, c, -1j * s, zero]),
        torch.stack([zero, -1j * s, c, zero]),
        torch.stack([zero, zero, zero, e]),
    ]
    return torch.stack(rows)
