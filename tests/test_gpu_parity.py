"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle
on the same seeded inputs. Rules and tolerances: parity_util."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import (BAND, TOL_GB, TOL_W, check_count, check_energy, check_forces, check_hist, check_matrix,
                         check_suminvr, oracle_pool)

pytestmark = pytest.mark.gpu


def _P():
    import paper_2202_06427_gb300 as P
    return P


def _box(dim, tric, L, rng):
    h = np.eye(dim) * L
    if tric:
        for a in range(1, dim):
            for b in range(a):
                h[a, b] = rng.uniform(-0.3 * L, 0.3 * L)
    return h


def _lattice_set(dim, tric, n_side, L, seed, wrap_far=True):
    """Jittered lattice in fractional coordinates of a random box, then each
    particle moved by a random lattice vector (positions far outside the box)."""
    rng = np.random.default_rng(seed)
    h = _box(dim, tric, L, rng)
    n = n_side ** dim - n_side  # ragged: not a full lattice
    x = synth.jittered_fractional(h, n_side, n, 0.4, seed + 1)
    if wrap_far:
        x = x + rng.integers(-3, 4, size=(n, dim)).astype(np.float64) @ h
    return np.ascontiguousarray(x), h


def _regime(dim, rc_frac):
    """Lattice spacing 1 and rc = 4 (2D) or 3 (3D), about 50 / 110 neighbours
    per particle as in the workloads (rc / spacing of 2 to 6); the box is
    sized so that rc is rc_frac of its side (0.6: several images per pair)."""
    rc = 4.0 if dim == 2 else 3.0
    L = rc / rc_frac
    n_side = int(round(L))
    return n_side, float(n_side), rc

SMALL = []
for dim in (2, 3):
    for tric in (False, True):
        for lcell in (1, 2, 3):
            for rc_frac in (0.08, 0.15, 0.6):
                SMALL.append((dim, tric, lcell, rc_frac))


@pytest.mark.parametrize("dim,tric,lcell,rc_frac", SMALL)
def test_small_all_reductions(cuda_ok, dim, tric, lcell, rc_frac):
    n_side, L, rc = _regime(dim, rc_frac)
    seed = 100 + dim * 1000 + tric * 100 + lcell * 10 + int(rc_frac * 100)
    x, h = _lattice_set(dim, tric, n_side, L, seed)
    w = oracle.geom_info(h, 1.0)["w"]
    assert rc < w.min()
    _check_all_reductions(x, h, rc, lcell)


def _dense_clusters(tric, seed):
    """Sparse jittered lattice (spacing 2) in a box of side 40 with two dense
    spheres (radius 3, lattice spacing 0.5, jitter 0.1: density 8, nearest
    pairs 0.3 apart) replacing it locally."""
    rng = np.random.default_rng(seed)
    L = 40.0
    h = np.eye(3) * L
    if tric:
        h[1, 0], h[2, 0], h[2, 1] = 6.0, -5.0, 4.0
    s = (np.stack(np.meshgrid(*[np.arange(20)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) / 20.0
    bg = (s + rng.uniform(-0.2, 0.2, size=s.shape) / 20.0) @ h
    centres = np.array([[12.0, 14.0, 13.0], [27.0, 25.0, 26.0]])
    g = np.stack(np.meshgrid(*[np.arange(-6, 7) * 0.5] * 3, indexing="ij"), -1).reshape(-1, 3)
    g = g[np.linalg.norm(g, axis=1) <= 3.0]
    parts = [bg[np.min(np.linalg.norm(bg[:, None, :] - centres[None], axis=2), axis=1) > 3.5]]
    for c in centres:
        parts.append(c + g + rng.uniform(-0.1, 0.1, size=g.shape))
    x = np.vstack(parts)
    return np.ascontiguousarray(x[rng.permutation(x.shape[0])]), h


@pytest.mark.parametrize("tric,lcell", [(False, 1), (True, 1), (False, 2), (True, 3)])
def test_dense_cells_all_reductions(cuda_ok, tric, lcell):
    """Cells with hundreds of particles and neighbourhoods far beyond the
    staging buffer (the dense-cell sweep, in groups of home particles), next to
    sparse cells (the per-particle companion) and ordinary ones."""
    P = _P()
    x, h = _dense_clusters(tric, 300 + lcell + 10 * tric)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, 4.0, lcell)
    if lcell == 1:
        assert P.cl_query(cl, "max_occupancy") > 256
    _check_all_reductions(x, h, 4.0, lcell)


def _check_all_reductions(x, h, rc, lcell):
    P = _P()
    nbins = 37
    ref = oracle.pair_map(x, h, rc, band=BAND, nbins=nbins)
    pos = torch.from_numpy(x).cuda()
    cl = P.cl_build(pos, h, rc, lcell)
    cnt = int(P.cl_map(cl, "count")["count"].item())
    check_count(cnt, ref)
    check_suminvr(P.cl_map(cl, "sum_inv_r")["sum_inv_r"].item(), ref, rc)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])
    hist = P.cl_map(cl, "hist", nbins=nbins)["hist"].cpu().numpy()
    check_hist(hist, ref)
    efv = P.cl_map(cl, "energy_forces_virial")
    check_energy(efv["energy"].item(), ref["energy"])
    check_forces(efv["forces"].cpu().numpy(), ref["forces"])
    check_matrix(efv["virial"].cpu().numpy(), ref["virial"], TOL_W)
    g = torch.tensor([0.75], dtype=torch.float64, device="cuda")
    gp, gb, vir = P.cl_backward(cl, g)
    check_forces(gp.cpu().numpy(), -0.75 * ref["forces"])
    check_matrix(gb.cpu().numpy(), 0.75 * ref["dedh"], TOL_GB)
    check_matrix(vir.cpu().numpy(), ref["virial"], TOL_W)
    # energy and gradient in one sweep, then the chain rule by cl_scale
    e1, dedx, dedh, vir1 = P.cl_energy_grad(cl, want_virial=True)
    check_energy(e1.item(), ref["energy"])
    check_forces(dedx.cpu().numpy(), -ref["forces"])
    check_matrix(dedh.cpu().numpy(), ref["dedh"], TOL_GB)
    check_matrix(vir1.cpu().numpy(), ref["virial"], TOL_W)
    check_forces(P.cl_scale(g, dedx).cpu().numpy(), -0.75 * ref["forces"])
    e2, gp2, _, _ = P.cl_energy_grad(cl, g, want_box=False)
    check_energy(e2.item(), ref["energy"])
    check_forces(gp2.cpu().numpy(), -0.75 * ref["forces"])
    assert P.cl_status(cl) == 0


@pytest.mark.parametrize("lcell", [1, 2, 3, 4])
def test_grid_independence(cuda_ok, lcell):
    """Results do not depend on the cell size (lcell, Sec. 2.8)."""
    P = _P()
    x, h = _lattice_set(3, True, 20, 28.0, 77)
    rc = 0.45 * oracle.geom_info(h, 1.0)["w"].min()
    ref = oracle.pair_map(x, h, rc, band=BAND, nbins=20)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, lcell)
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    check_hist(P.cl_map(cl, "hist", nbins=20)["hist"].cpu().numpy(), ref)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])


def test_workload_small_10k(cuda_ok):
    """3D, 10,000 particles, cubic box 46.416, rc 12: sum 1/r and the count."""
    P = _P()
    w = synth.w0_small()
    ref = oracle.pair_map(w["x"], w["h"], w["rc"], band=BAND, forces=False)
    cl = P.cl_build(torch.from_numpy(w["x"]).cuda(), w["h"], w["rc"], 2)
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    check_suminvr(P.cl_map(cl, "sum_inv_r")["sum_inv_r"].item(), ref, w["rc"])
    assert 3.5e6 < ref["count"] < 3.7e6


@pytest.mark.slow
def test_workload_lattice_1m(cuda_ok):
    """3D, 1,000,000 jittered lattice, box 215.44, rc 12: energy forward, forces,
    virial and box gradient from the backward kernel, in the launch
    configuration the benchmark times (lcell 2)."""
    P = _P()
    w = synth.w1_lattice()
    ref = oracle_pool(w["x"], w["h"], w["rc"], nbins=0, forces=True)
    pos = torch.from_numpy(w["x"]).cuda()
    cl = P.cl_build(pos, w["h"], w["rc"], 2)
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])
    g = torch.ones(1, dtype=torch.float64, device="cuda")
    gp, gb, vir = P.cl_backward(cl, g)
    check_forces(gp.cpu().numpy(), -ref["forces"])
    check_matrix(vir.cpu().numpy(), ref["virial"], TOL_W)
    check_matrix(gb.cpu().numpy(), ref["dedh"], TOL_GB)
    efv = P.cl_map(cl, "energy_forces_virial")
    check_forces(efv["forces"].cpu().numpy(), ref["forces"])
    check_energy(efv["energy"].item(), ref["energy"])
    del efv
    e1, dedx, dedh, vir1 = P.cl_energy_grad(cl, want_virial=True)
    check_energy(e1.item(), ref["energy"])
    check_forces(dedx.cpu().numpy(), -ref["forces"])
    check_matrix(dedh.cpu().numpy(), ref["dedh"], TOL_GB)
    check_matrix(vir1.cpu().numpy(), ref["virial"], TOL_W)


def test_empty_and_tiny(cuda_ok):
    P = _P()
    h = np.eye(3) * 10.0
    for n in (0, 1):
        pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda") + 1.0
        cl = P.cl_build(pos, h, 3.0, 2)
        assert int(P.cl_map(cl, "count")["count"].item()) == 0
        assert P.cl_map(cl, "energy")["energy"].item() == 0.0
        assert P.cl_map(cl, "sum_inv_r")["sum_inv_r"].item() == 0.0
        efv = P.cl_map(cl, "energy_forces_virial")
        assert efv["energy"].item() == 0.0
        assert int(P.cl_map(cl, "hist", nbins=4)["hist"].sum().item()) == 0
        gp, gb, vir = P.cl_backward(cl, torch.ones(1, dtype=torch.float64, device="cuda"))
        assert gp.shape == (n, 3) and float(gb.abs().max()) == 0.0
        e1, dedx, dedh, _ = P.cl_energy_grad(cl)
        assert e1.item() == 0.0 and dedx.shape == (n, 3) and float(dedh.abs().max()) == 0.0
        if n:
            assert float(dedx.abs().max()) == 0.0
    # two particles across the periodic boundary: distance 1.5 through the face
    x = np.array([[0.25, 5.0, 5.0], [8.75, 5.0, 5.0]])
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, 3.0, 2)
    assert int(P.cl_map(cl, "count")["count"].item()) == 1
    assert P.cl_map(cl, "sum_inv_r")["sum_inv_r"].item() == pytest.approx(1 / 1.5, rel=1e-6)


def test_all_in_one_cell_and_multi_image(cuda_ok):
    """Degenerate grids: one cell per axis (box < 2 rc, several images per
    pair) and every particle piled in one corner."""
    P = _P()
    rng = np.random.default_rng(5)
    h = np.array([[7.0, 0, 0], [1.0, 6.5, 0], [0.5, -1.0, 6.8]])
    rc = 0.9 * oracle.geom_info(h, 1.0)["w"].min()
    x = synth.jittered_fractional(h, 6, 200, 0.3, 9)
    ref = oracle.pair_map(x, h, rc, band=BAND, nbins=11)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, 1)
    assert P.cl_query(cl, "ncells") == 1
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])
    efv = P.cl_map(cl, "energy_forces_virial")
    check_forces(efv["forces"].cpu().numpy(), ref["forces"])
    # corner pile: particles within a 1.0 cube of a 30 box (min separation 0.1)
    g = np.stack(np.meshgrid(*[np.arange(8) * 0.12] * 3, indexing="ij"), -1).reshape(-1, 3) + 29.5
    h2 = np.eye(3) * 30.0
    ref2 = oracle.pair_map(g, h2, 2.0, band=BAND)
    cl2 = P.cl_build(torch.from_numpy(np.ascontiguousarray(g)).cuda(), h2, 2.0, 2)
    check_count(int(P.cl_map(cl2, "count")["count"].item()), ref2)
    check_energy(P.cl_map(cl2, "energy")["energy"].item(), ref2["energy"])
    assert P.cl_query(cl2, "max_occupancy") >= 1


def test_dense_single_cell_forces(cuda_ok):
    """A cell holding more particles than the staging window (2,197 on a 0.1
    lattice inside one cell of side 2, next to the periodic boundary) and a
    sparse background: the windowed half-shell sweep with home batches and
    several own-cell windows, forces and box gradient against the oracle.
    (The box gradient's X = sum x (x) F carries the FP32 force error times the
    raw position, so the pile sits near the origin.)"""
    P = _P()
    rng = np.random.default_rng(23)
    h = np.array([[30.0, 0, 0], [0.0, 30.0, 0], [0.0, 0, 30.0]])
    g = np.stack(np.meshgrid(*[np.arange(13) * 0.1] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.3
    bg = rng.uniform(0.0, 30.0, size=(6000, 3))
    bg = bg[np.min(np.abs(bg[:, None, :] - (g.mean(0))[None, None, :]).max(axis=2), axis=1) > 1.2]
    x = np.ascontiguousarray(np.vstack([g + rng.uniform(-0.01, 0.01, size=g.shape), bg])[rng.permutation(len(g) + len(bg))])
    rc = 2.0
    ref = oracle.pair_map(x, h, rc, band=BAND)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, 1)
    assert P.cl_query(cl, "max_occupancy") > 1536
    efv = P.cl_map(cl, "energy_forces_virial")
    assert P.cl_query(cl, "sweep_half") == 1
    check_energy(efv["energy"].item(), ref["energy"])
    check_forces(efv["forces"].cpu().numpy(), ref["forces"])
    check_matrix(efv["virial"].cpu().numpy(), ref["virial"], TOL_W)
    e1, dedx, dedh, vir1 = P.cl_energy_grad(cl, want_virial=True)
    check_energy(e1.item(), ref["energy"])
    check_forces(dedx.cpu().numpy(), -ref["forces"])
    check_matrix(dedh.cpu().numpy(), ref["dedh"], TOL_GB)
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)


def test_errors_are_reported(cuda_ok):
    P = _P()
    pos = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(P.CellMapError) as e:
        P.cl_build(pos, np.eye(3) * 10.0, 10.0, 1)
    assert e.value.code == -3
    with pytest.raises(P.CellMapError) as e:
        P.cl_build(pos, np.zeros((3, 3)), 1.0, 1)
    assert e.value.code == -2
    bad = torch.tensor([[1.0, 2.0, 3.0], [float("nan"), 0.0, 0.0], [4.0, 4.0, 4.0]], dtype=torch.float64,
                       device="cuda")
    cl = P.cl_build(bad, np.eye(3) * 10.0, 3.0, 2)
    assert P.cl_status(cl) == -4
    assert P.cl_status(cl) == 0  # latch cleared
    assert int(P.cl_map(cl, "count")["count"].item()) == 0


def test_update_matches_fresh_build(cuda_ok):
    P = _P()
    x, h = _lattice_set(3, True, 16, 24.0, 31)
    rc = 0.4 * oracle.geom_info(h, 1.0)["w"].min()
    x2 = x + np.random.default_rng(2).normal(0, 0.2, size=x.shape)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, 2)
    pos2 = torch.from_numpy(np.ascontiguousarray(x2)).cuda()
    P.cl_update(cl, pos2)
    ref = oracle.pair_map(x2, h, rc, band=BAND)
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])
    # new box with a different grid
    h3 = h * 1.3
    P.cl_update(cl, pos2, h=h3)
    ref3 = oracle.pair_map(x2, h3, rc, band=BAND)
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref3)


def pairlist_total(P, cl, capacity=16):
    """cl_map(CL_RED_PAIRLIST) through the C ABI with a buffer of `capacity`
    pairs: returns the total the call reports (CL_ERR_CAPACITY when it does
    not fit, CL_OK otherwise)."""
    import ctypes
    from paper_2202_06427_gb300 import _lib as L
    pi = torch.empty(capacity, dtype=torch.int32, device="cuda")
    pj = torch.empty(capacity, dtype=torch.int32, device="cuda")
    pd = torch.empty(capacity, dtype=torch.float32, device="cuda")
    npairs = ctypes.c_longlong(-1)
    res = L.cl_result()
    res.pair_i, res.pair_j, res.pair_d = pi.data_ptr(), pj.data_ptr(), pd.data_ptr()
    res.capacity = capacity
    res.npairs = ctypes.pointer(npairs)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = L.lib().cl_map(cl.handle, L.CL_RED_PAIRLIST, None, ctypes.byref(res), stream)
    assert code in (L.CL_OK, L.CL_ERR_CAPACITY), code
    assert (code == L.CL_ERR_CAPACITY) == (npairs.value > capacity)
    return int(npairs.value)


@pytest.mark.slow
def test_workload_clustered_16m(cuda_ok):
    """3D clustered, 16M particles in a cubic box of side 600 (2,000 Gaussian
    clusters + 20% background, minimum separation 0.5), rc 8: energy, forces
    and virial (forward, full shell) and the backward kernel. Energy and virial
    against the whole oracle (run in a process pool); forces on a sample of
    particles computed one by one by the oracle."""
    P = _P()
    w = synth.w4_clustered()
    x, h, rc = w["x"], w["h"], w["rc"]
    n = x.shape[0]
    ref = oracle_pool(x, h, rc, nbins=0, forces=False)
    sample = np.sort(np.random.default_rng(44).choice(n, size=3000, replace=False))
    f_ref, _ = oracle.particles(x, h, rc, sample)
    pos = torch.from_numpy(x).cuda()
    cl = P.cl_build(pos, h, rc, 1)
    assert P.cl_query(cl, "max_occupancy") > 10 * n / P.cl_query(cl, "ncells")  # strongly inhomogeneous
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    # more than 2^31 pairs: the pair list's offsets and total are 64-bit, so a
    # call with a small buffer reports CL_ERR_CAPACITY and the exact total
    total = pairlist_total(P, cl)
    assert total > 2 ** 31
    check_count(total, ref)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])
    efv = P.cl_map(cl, "energy_forces_virial")
    check_energy(efv["energy"].item(), ref["energy"])
    check_matrix(efv["virial"].cpu().numpy(), ref["virial"], TOL_W)
    check_forces(efv["forces"][torch.from_numpy(sample).cuda()].cpu().numpy(), f_ref)
    del efv
    gp, gb, vir = P.cl_backward(cl, torch.ones(1, dtype=torch.float64, device="cuda"))
    check_forces(gp[torch.from_numpy(sample).cuda()].cpu().numpy(), -f_ref)
    check_matrix(vir.cpu().numpy(), ref["virial"], TOL_W)
    check_matrix(gb.cpu().numpy(), ref["dedh"], TOL_GB)
    del gp
    cl2 = P.cl_build(pos, h, rc, 2)  # the launch configuration of the benchmark
    e1, dedx, dedh, vir1 = P.cl_energy_grad(cl2, want_virial=True)
    check_energy(e1.item(), ref["energy"])
    check_forces(dedx[torch.from_numpy(sample).cuda()].cpu().numpy(), -f_ref)
    check_matrix(vir1.cpu().numpy(), ref["virial"], TOL_W)
    check_matrix(dedh.cpu().numpy(), ref["dedh"], TOL_GB)


def _mixed_occupancy(seed):
    """Jittered lattice (spacing 1) in a box of side 40 with a spherical void
    (radius 7: empty cells and cells with a few particles at its rim) and two
    dense spheres (radius 3, spacing 0.5: hundreds of particles per cell of
    side 4). At cell side 4 (rc 4, lcell 1) the mean occupancy is about 60."""
    rng = np.random.default_rng(seed)
    L = 40.0
    h = np.eye(3) * L
    h[1, 0], h[2, 0], h[2, 1] = 3.0, -2.0, 2.5
    s = (np.stack(np.meshgrid(*[np.arange(40)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) / 40.0
    bg = (s + rng.uniform(-0.15, 0.15, size=s.shape) / 40.0) @ h
    void = np.array([20.0, 20.0, 20.0])
    centres = np.array([[8.0, 9.0, 8.5], [31.0, 30.0, 31.5]])
    g = np.stack(np.meshgrid(*[np.arange(-6, 7) * 0.5] * 3, indexing="ij"), -1).reshape(-1, 3)
    g = g[np.linalg.norm(g, axis=1) <= 3.0]
    keep = (np.linalg.norm(bg - void, axis=1) > 7.0) & \
           (np.min(np.linalg.norm(bg[:, None, :] - centres[None], axis=2), axis=1) > 3.5)
    parts = [bg[keep]] + [c + g + rng.uniform(-0.1, 0.1, size=g.shape) for c in centres]
    x = np.vstack(parts)
    return np.ascontiguousarray(x[rng.permutation(x.shape[0])]), h


@pytest.mark.parametrize("lcell", [1, 2])
def test_scalar_reductions_both_paths(cuda_ok, lcell):
    """Count, sum 1/r and the histogram on a set mixing ordinary, empty,
    sparse and very dense cells: at lcell 1 (about 60 particles per cell) the
    staged neighbourhood sweep with its per-particle companion for the cells
    it leaves, at lcell 2 (about 8) the per-particle sweep alone."""
    P = _P()
    x, h = _mixed_occupancy(517)
    rc, nbins = 4.0, 37
    ref = oracle.pair_map(x, h, rc, band=BAND, nbins=nbins, forces=False)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, lcell)
    occ = x.shape[0] / P.cl_query(cl, "ncells")
    assert (occ > 16) == (lcell == 1), occ
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    check_suminvr(P.cl_map(cl, "sum_inv_r")["sum_inv_r"].item(), ref, rc)
    check_hist(P.cl_map(cl, "hist", nbins=nbins)["hist"].cpu().numpy(), ref)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])


@pytest.mark.parametrize("lcell", [1, 2])
@pytest.mark.parametrize("nbins,rmax_frac", [(1, 1.0), (4096, 0.6), (257, 1.3)])
def test_hist_bins_and_rmax(cuda_ok, lcell, nbins, rmax_frac):
    """Histogram at the bin-count limits and with rmax below and above the
    cutoff (bins past the cutoff stay empty), on both sweep paths."""
    P = _P()
    x, h = _mixed_occupancy(518)
    rc = 4.0
    rmax = rmax_frac * rc
    ref = oracle.pair_map(x, h, rc, band=BAND, nbins=nbins, rmax=rmax, forces=False)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, lcell)
    hist = P.cl_map(cl, "hist", nbins=nbins, rmax=rmax)["hist"].cpu().numpy()
    check_hist(hist, ref)
    if rmax > rc:
        assert hist[int(np.ceil(nbins * rc / rmax)):].sum() == 0


def test_interleaved_calls_reuse_work_lists(cuda_ok):
    """The half-shell sweep keeps its per-cell work lists between calls on one
    list; calls that use the same buffers (the pair list, the histogram, the
    energy alone) and a rebuild must not leave stale lists behind."""
    P = _P()
    x, h = _mixed_occupancy(519)
    rc = 4.0
    ref = oracle.pair_map(x, h, rc, band=BAND, nbins=19)
    pos = torch.from_numpy(x).cuda()
    cl = P.cl_build(pos, h, rc, 1)

    def grad_ok():
        e, dedx, dedh, _ = P.cl_energy_grad(cl)
        check_energy(e.item(), ref["energy"])
        check_forces(dedx.cpu().numpy(), -ref["forces"])
        check_matrix(dedh.cpu().numpy(), ref["dedh"], TOL_GB)

    grad_ok()
    grad_ok()  # reused lists
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    grad_ok()
    lst = P.cl_map(cl, "pairlist")
    assert ref["count"] - ref["band_in"] <= lst["npairs"] <= ref["count"] + ref["band_out"]
    grad_ok()
    check_hist(P.cl_map(cl, "hist", nbins=19)["hist"].cpu().numpy(), ref)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])
    grad_ok()
    # a rebuild with the particles permuted: new cell contents, same physics
    perm = np.random.default_rng(3).permutation(x.shape[0])
    P.cl_update(cl, torch.from_numpy(np.ascontiguousarray(x[perm])).cuda())
    e, dedx, _, _ = P.cl_energy_grad(cl)
    check_energy(e.item(), ref["energy"])
    check_forces(dedx.cpu().numpy(), -ref["forces"][perm])
    check_suminvr(P.cl_map(cl, "sum_inv_r")["sum_inv_r"].item(), ref, rc)
