"""torch.autograd wrapper: the shifted-force pair energy and its hand-written
adjoint (Sec. 3.3, Code 9 differentiates a pair sum; here the backward is a
CUDA kernel, not tracing).

    E(x, H) = sum over pair-images within rc of u(r),
    u(r) = 1/r - 1/rc + (r - rc)/rc^2.

When a gradient will be needed, forward runs one full-shell sweep that gives
the energy together with dE/dx = -F and dE/dH at fixed Cartesian positions,
H^-T (X - W) with X = sum_i x_i (x) F_i and W the virial (cl_energy_grad), and
backward only scales them by dL/dE (cl_scale). Otherwise forward runs the
half-shell energy sweep alone.
"""
import numpy as np
import torch

from .api import cl_build, cl_energy_grad, cl_map, cl_scale, cl_update


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
        ctx.h_meta = (h.device, h.dtype) if torch.is_tensor(h) else None
        want_box = bool(ctx.needs_input_grad[1]) and ctx.h_meta is not None
        if ctx.needs_input_grad[0] or want_box:
            e, dedx, dedh, _ = cl_energy_grad(holder.cl, want_box=want_box)
            ctx.save_for_backward(dedx, dedh if want_box else None)
        else:
            e = cl_map(holder.cl, "energy")["energy"]
        return e.reshape(())

    @staticmethod
    def backward(ctx, g):
        dedx, dedh = ctx.saved_tensors
        g = g.detach()
        gp = cl_scale(g, dedx) if ctx.needs_input_grad[0] else None
        gb = None
        if dedh is not None:
            gb = cl_scale(g, dedh).to(device=ctx.h_meta[0], dtype=ctx.h_meta[1])
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
