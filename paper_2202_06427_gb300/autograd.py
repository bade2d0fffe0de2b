"""torch.autograd wrapper: the shifted-force pair energy and its hand-written
adjoint (Sec. 3.3, Code 9 differentiates a pair sum; here the backward is a
CUDA kernel, not tracing).

    E(x, H) = sum over pair-images within rc of u(r),
    u(r) = 1/r - 1/rc + (r - rc)/rc^2.

Forward runs the half-shell energy sweep. Backward runs the full-shell force
sweep: dL/dx = dL/dE * dE/dx = -dL/dE * F, and dL/dH at fixed Cartesian
positions = dL/dE * H^-T (X - W) with X = sum_i x_i (x) F_i and W the virial.
"""
import numpy as np
import torch

from .api import cl_backward, cl_build, cl_map, cl_update


class _Holder:
    def __init__(self, cutoff, lcell):
        self.cutoff = float(cutoff)
        self.lcell = int(lcell)
        self.cl = None


class ShiftedForceEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, h, holder):
        hnp = h.detach().cpu().numpy() if torch.is_tensor(h) else np.asarray(h, dtype=np.float64)
        if holder.cl is None or holder.cl.n != pos.shape[0]:
            holder.cl = cl_build(pos, hnp, holder.cutoff, holder.lcell)
        else:
            cl_update(holder.cl, pos, h=hnp)
        e = cl_map(holder.cl, "energy")["energy"]
        ctx.holder = holder
        ctx.h_meta = (h.device, h.dtype) if torch.is_tensor(h) else None
        return e.reshape(())

    @staticmethod
    def backward(ctx, g):
        want_box = bool(ctx.needs_input_grad[1]) and ctx.h_meta is not None
        gp, gb, _ = cl_backward(ctx.holder.cl, g.detach(), want_box=want_box, want_virial=False)
        if want_box:
            gb = gb.to(device=ctx.h_meta[0], dtype=ctx.h_meta[1])
        return gp, gb, None


class PairEnergy:
    """Reusable energy function: keeps one cell list resident and updates it
    for new positions (Sec. 4.2: lists are reused between steps)."""

    def __init__(self, cutoff, lcell=2):
        self.holder = _Holder(cutoff, lcell)

    def __call__(self, pos, h):
        return ShiftedForceEnergy.apply(pos, h, self.holder)


def energy(pos, h, cutoff, lcell=2):
    """One-shot differentiable shifted-force energy of (n, dim) float64 CUDA
    positions in the box h (rows = lattice vectors; a tensor for dL/dH)."""
    return ShiftedForceEnergy.apply(pos, h, _Holder(cutoff, lcell))
