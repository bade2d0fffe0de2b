"""torch.autograd through the hand-written adjoint: the forward that a gradient
follows runs the fused energy-and-gradient sweep, the backward applies the
chain rule with cl_scale; both against the FP64 oracle's analytic gradient."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import BAND, TOL_GB, check_energy, check_forces, check_matrix

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tric", [False, True])
def test_energy_grad_through_autograd(cuda_ok, tric):
    from paper_2202_06427_gb300 import autograd as AG
    rng = np.random.default_rng(510 + tric)
    L = 24.0
    h = np.eye(3) * L
    if tric:
        h[1, 0], h[2, 0], h[2, 1] = 0.2 * L, -0.15 * L, 0.1 * L
    x = synth.jittered_fractional(h, 24, 24 ** 3 - 100, 0.4, 511 + tric)
    x = x + rng.integers(-2, 3, size=x.shape).astype(np.float64) @ h  # unwrapped inputs
    rc = 3.0
    ref = oracle.pair_map(x, h, rc, band=BAND)
    pos = torch.from_numpy(x).cuda().requires_grad_(True)
    hb = torch.from_numpy(h.copy()).cuda().requires_grad_(True)
    f = AG.PairEnergy(rc, lcell=2)
    e = f(pos, hb)
    check_energy(e.item(), ref["energy"])
    (2.5 * e).backward()
    check_forces(pos.grad.cpu().numpy(), -2.5 * ref["forces"])
    check_matrix(hb.grad.cpu().numpy(), 2.5 * ref["dedh"], TOL_GB)
    # positions only, and no gradient at all
    pos2 = torch.from_numpy(x).cuda().requires_grad_(True)
    e2 = f(pos2, h)
    e2.backward()
    check_forces(pos2.grad.cpu().numpy(), -ref["forces"])
    with torch.no_grad():
        check_energy(f(torch.from_numpy(x).cuda(), h).item(), ref["energy"])
