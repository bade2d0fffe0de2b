"""The mapped functions of the paper's examples, as C entry points built on the
functor hook: Code 5 (mass-weighted 1/r), Code 6/7 (Lennard-Jones energy and
forces), Code 10 (pairwise-velocity histogram), against the FP64 oracle's sums
over every pair-image."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import BAND

pytestmark = pytest.mark.gpu

REGIMES = [(3, False, 3.0, 1), (3, True, 3.0, 2), (2, True, 4.0, 2), (3, True, 0.6, 2)]


def _set(dim, tric, rc_or_frac, seed):
    rng = np.random.default_rng(seed)
    if rc_or_frac < 1:  # small box: pairs with several images inside the cutoff
        h = np.eye(dim) * 9.0
        if tric:
            h[1, 0] = 2.0
        n_side = 9
        rc = rc_or_frac * oracle.geom_info(h, 1.0)["w"].min()
    else:
        L = 22.0 if dim == 3 else 50.0
        h = np.eye(dim) * L
        if tric:
            for a in range(1, dim):
                for b in range(a):
                    h[a, b] = rng.uniform(-0.25 * L, 0.25 * L)
        n_side = int(L)
        rc = rc_or_frac
    x = synth.jittered_fractional(h, n_side, n_side ** dim - 3, 0.4, seed + 1)
    x = x + rng.integers(-2, 3, size=x.shape).astype(np.float64) @ h
    return np.ascontiguousarray(x), h, rc


@pytest.mark.parametrize("dim,tric,rc,lcell", REGIMES)
def test_lj_energy_and_forces(cuda_ok, dim, tric, rc, lcell):
    import paper_2202_06427_gb300 as P
    x, h, rc = _set(dim, tric, rc, 300 + dim + 10 * tric + lcell)
    eps, sigma = 0.0442, 0.8
    ref = oracle.lj(x, h, rc, eps, sigma, band=BAND)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, lcell)
    e, f = P.cl_map_lj(cl, eps, sigma)
    e0, _ = P.cl_map_lj(cl, eps, sigma, forces=False)
    slack = ref["band_abs_energy"]
    for got in (e.item(), e0.item()):
        assert abs(got - ref["energy"]) <= 1e-5 * ref["abs_energy"] + slack, (got, ref["energy"])
    fg = f.cpu().numpy().astype(np.float64)
    scale = np.abs(ref["forces"]).max()
    assert np.abs(fg - ref["forces"]).max() <= 1e-4 * scale + np.abs(ref["band_forces"]).max()


@pytest.mark.parametrize("dim,tric,rc,lcell", REGIMES)
def test_mass_potential(cuda_ok, dim, tric, rc, lcell):
    import paper_2202_06427_gb300 as P
    x, h, rc = _set(dim, tric, rc, 400 + dim + 10 * tric + lcell)
    m = np.random.default_rng(5).uniform(0.5, 2.0, size=x.shape[0]).astype(np.float32)
    ref = oracle.mass_potential(x, h, rc, m.astype(np.float64), band=BAND)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, lcell)
    got = P.cl_map_mass(cl, torch.from_numpy(m).cuda()).item()
    assert abs(got - ref["value"]) <= 1e-5 * abs(ref["value"]) + ref["band"]


@pytest.mark.parametrize("dim,tric,rc,lcell", REGIMES)
def test_velocity_histogram(cuda_ok, dim, tric, rc, lcell):
    import paper_2202_06427_gb300 as P
    x, h, rc = _set(dim, tric, rc, 500 + dim + 10 * tric + lcell)
    v = np.random.default_rng(6).normal(size=x.shape).astype(np.float32)
    nbins = 10
    binstep = rc / 10.0
    ref = oracle.velocity_hist(x, h, rc, v.astype(np.float64), binstep, nbins, band=BAND)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, lcell)
    counts, vsum = P.cl_map_velocity_hist(cl, torch.from_numpy(v).cuda(), binstep, nbins)
    c = counts.cpu().numpy()
    # a pair near a bin edge (or the cutoff) may land in its bin or a neighbour
    bc, bv = ref["band_counts"], ref["band_vsum"]
    near_c = bc + np.roll(bc, 1) + np.roll(bc, -1)
    near_v = bv + np.roll(bv, 1) + np.roll(bv, -1)
    assert np.all(c >= ref["counts"]) and np.all(c <= ref["counts"] + near_c), (c, ref["counts"])
    dv = vsum.cpu().numpy() - ref["vsum"]
    assert np.all(dv >= -1e-5 * ref["vsum"] - 1e-9) and np.all(dv <= 1e-5 * ref["vsum"] + near_v + 1e-9)


def test_pair_functions_reject_bad_arguments(cuda_ok):
    import paper_2202_06427_gb300 as P
    from paper_2202_06427_gb300 import CellMapError
    cl = P.cl_build(torch.zeros((4, 3), dtype=torch.float64, device="cuda") + 1.0, np.eye(3) * 10, 2.0, 2)
    with pytest.raises(CellMapError):
        P.cl_map_lj(cl, 1.0, 0.0)
    with pytest.raises(CellMapError):
        P.cl_map_velocity_hist(cl, torch.zeros((4, 3), device="cuda"), 0.5, 0)
    with pytest.raises(CellMapError):
        P.cl_map_velocity_hist(cl, torch.zeros((4, 3), device="cuda"), 0.5, 65)
