"""Randomised parity sweep: seeded random boxes (2D/3D, orthorhombic or
triclinic), cell sizes (lcell 1-4), cutoffs, ragged particle counts, positions
far outside the box, and in 3D dense clusters next to a sparse background, so
that every path of the sweeps is taken under many shapes (neighbourhood,
dense-cell and per-particle sweeps; staged and per-particle pair-list passes).
Every reduction and the pair list against the oracle, rules of parity_util.

Positions are jittered lattices (spacing 1 or 0.5 in the clusters) so that no
pair is much closer than the precision envelope of cell-centred FP32
coordinates allows (forces ~ 1/r^2)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import (BAND, TOL_GB, TOL_W, check_count, check_energy, check_forces, check_hist, check_matrix,
                         check_suminvr)

pytestmark = pytest.mark.gpu


def _config(seed):
    rng = np.random.default_rng(9000 + seed)
    dim = 3 if seed % 3 else 2
    tric = bool(seed % 2)
    lcell = 1 + seed % 4
    L = float(rng.integers(14, 21)) if dim == 3 else float(rng.integers(24, 41))
    h = np.eye(dim) * L
    if tric:
        for a in range(1, dim):
            for b in range(a):
                h[a, b] = rng.uniform(-0.3 * L, 0.3 * L)
    n_side = int(L)
    n_full = n_side ** dim
    n = int(n_full * rng.uniform(0.6, 1.0))
    x = synth.jittered_fractional(h, n_side, n, 0.35, 9100 + seed)
    if dim == 3 and (seed % 5 == 1 or seed % 7 == 3):
        # a dense sphere (spacing 0.5) replacing the background locally
        c = (rng.uniform(0.3, 0.7, size=3)) @ h
        r = rng.uniform(2.0, 3.2)
        g = np.stack(np.meshgrid(*[np.arange(-7, 8) * 0.5] * 3, indexing="ij"), -1).reshape(-1, 3)
        g = g[np.linalg.norm(g, axis=1) <= r]
        d = x - c
        d -= np.round(d @ np.linalg.inv(h)) @ h
        x = np.vstack([x[np.linalg.norm(d, axis=1) > r + 0.6], c + g + rng.uniform(-0.08, 0.08, size=g.shape)])
    x = x + rng.integers(-3, 4, size=x.shape).astype(np.float64) @ h
    x = np.ascontiguousarray(x[rng.permutation(x.shape[0])])
    w = oracle.geom_info(h, 1.0)["w"]
    if seed % 6 == 5:  # several images of one pair within the cutoff (no pair list)
        L = float(rng.integers(6, 10)) if dim == 3 else float(rng.integers(8, 14))
        h = h * (L / np.abs(np.diag(h)).max())
        x = synth.jittered_fractional(h, int(L), int(L) ** dim - int(L), 0.35, 9200 + seed)
        x = np.ascontiguousarray(x + rng.integers(-2, 3, size=x.shape).astype(np.float64) @ h)
        w = oracle.geom_info(h, 1.0)["w"]
        return dim, tric, lcell, x, h, float(rng.uniform(0.55, 0.9) * w.min())
    rc = float(rng.uniform(0.12, 0.45) * w.min())
    rc = min(rc, 4.5 if dim == 3 else 6.0)  # workload-like cutoffs (rc / spacing up to ~5)
    return dim, tric, lcell, x, h, rc


@pytest.mark.parametrize("seed", range(64))
def test_random_configuration(cuda_ok, seed):
    import paper_2202_06427_gb300 as P
    dim, tric, lcell, x, h, rc = _config(seed)
    nbins = 23
    ref = oracle.pair_map(x, h, rc, band=BAND, nbins=nbins)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, lcell)
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    check_suminvr(P.cl_map(cl, "sum_inv_r")["sum_inv_r"].item(), ref, rc)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])
    check_hist(P.cl_map(cl, "hist", nbins=nbins)["hist"].cpu().numpy(), ref)
    efv = P.cl_map(cl, "energy_forces_virial")
    check_energy(efv["energy"].item(), ref["energy"])
    check_forces(efv["forces"].cpu().numpy(), ref["forces"])
    check_matrix(efv["virial"].cpu().numpy(), ref["virial"], TOL_W)
    g = torch.tensor([1.25], dtype=torch.float64, device="cuda")
    gp, gb, vir = P.cl_backward(cl, g)
    check_forces(gp.cpu().numpy(), -1.25 * ref["forces"])
    check_matrix(gb.cpu().numpy(), 1.25 * ref["dedh"], TOL_GB)
    check_matrix(vir.cpu().numpy(), ref["virial"], TOL_W)
    e1, dedx, dedh, _ = P.cl_energy_grad(cl)
    check_energy(e1.item(), ref["energy"])
    check_forces(dedx.cpu().numpy(), -ref["forces"])
    check_matrix(dedh.cpu().numpy(), ref["dedh"], TOL_GB)
    if 2.0 * rc > oracle.geom_info(h, 1.0)["w"].min():
        with pytest.raises(P.CellMapError) as e:  # a pair may have several images: no list
            P.cl_map(cl, "pairlist")
        assert e.value.code == -3
        assert P.cl_status(cl) == 0
        return
    # the sorted i<j list: every certain oracle pair, nothing outside the band, distances within BAND rc
    pl = P.cl_map(cl, "pairlist")
    i, j, d = (pl[k].cpu().numpy() for k in ("i", "j", "d"))
    n = x.shape[0]
    key = i.astype(np.int64) * n + j
    assert np.all(i < j) and np.all(np.diff(key) > 0)
    lst = oracle.pairlist(x, h, rc, band=BAND, cap=1 << 24)
    rk = lst["i"] * n + lst["j"]
    certain = (lst["d"] < rc) & ~lst["band"]
    assert np.isin(rk[certain], key).all()
    pos = np.searchsorted(rk, key)
    assert np.array_equal(rk[np.minimum(pos, len(rk) - 1)], key)
    assert np.all(np.abs(d - lst["d"][pos]) <= BAND * rc)
    assert P.cl_status(cl) == 0
