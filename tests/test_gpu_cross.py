"""Two sets (Code 8) and open boundaries (Sec. 4.1): cross counts, the cross
pair list, per-query k nearest, the global k nearest pairs and the open-box
cell list, against the oracle's cross pair-images (and brute force without
periodic images)."""
import numpy as np
import pytest
import torch

import oracle
from parity_util import BAND, check_count, check_energy, check_forces, check_hist

pytestmark = pytest.mark.gpu


def _sets(dim, tric, L, na, nb, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    h = np.eye(dim) * L
    if tric:
        for a in range(1, dim):
            for b in range(a):
                h[a, b] = rng.uniform(-0.25 * L, 0.25 * L)
    xa = rng.uniform(-spread, 1 + spread, size=(na, dim)) @ h
    yb = rng.uniform(-spread, 1 + spread, size=(nb, dim)) @ h
    return np.ascontiguousarray(xa), np.ascontiguousarray(yb), h


REGIMES = [(3, False, 20.0, 2.5, 2), (3, True, 20.0, 3.0, 1), (2, True, 40.0, 3.0, 2), (3, True, 6.0, 3.5, 2)]


@pytest.mark.parametrize("dim,tric,L,rc,lcell", REGIMES)
def test_cross_count_and_knn(cuda_ok, dim, tric, L, rc, lcell):
    import paper_2202_06427_gb300 as P
    xa, yb, h = _sets(dim, tric, L, 3000, 2000, 700 + dim + lcell)
    ref = oracle.cross_images(xa, yb, h, rc, band=BAND)
    inside = ref["r"] < rc
    edge = oracle.band_mask(ref, rc, BAND)
    cl = P.cl_build(torch.from_numpy(xa).cuda(), h, rc, lcell)
    yb_t = torch.from_numpy(yb).cuda()
    got = P.cl_cross_count(cl, yb_t)
    core = int(np.sum(inside & ~edge))
    assert core <= got <= core + int(np.sum(edge)), (got, core)
    k = 7
    a, d = P.cl_cross_knn(cl, yb_t, k)
    a, d = a.cpu().numpy(), d.cpu().numpy()
    for b in range(0, yb.shape[0], 97):
        sel = (ref["j"] == b) & inside
        want = np.sort(ref["r"][sel])[:k]
        m = min(k, len(want))
        assert np.all(a[b, m:] == -1) or np.any(edge[(ref["j"] == b)])
        assert np.allclose(d[b, :m], want[:m], rtol=2e-6, atol=2e-6 * rc)
        if m < k and not np.any(edge[(ref["j"] == b)]):
            assert np.all(np.isinf(d[b, m:]))
    top = P.cl_cross_topk(cl, yb_t, 5)
    want = oracle.knn_pairs(xa, yb, h, rc, 5, img=ref)
    assert top["n"] == len(want["r"])
    assert np.allclose(top["d"][:top["n"]].cpu().numpy(), want["r"], rtol=0, atol=4e-6 * rc)
    # the pairs themselves (distances here have no ties)
    assert np.array_equal(top["a"][:top["n"]].cpu().numpy(), want["i"])
    assert np.array_equal(top["b"][:top["n"]].cpu().numpy(), want["j"])


@pytest.mark.parametrize("dim,tric,L,rc,lcell", REGIMES[:3])
def test_cross_pairlist(cuda_ok, dim, tric, L, rc, lcell):
    import paper_2202_06427_gb300 as P
    xa, yb, h = _sets(dim, tric, L, 3000, 2500, 800 + dim + lcell)
    ref = oracle.cross_images(xa, yb, h, rc, band=BAND)
    edge = oracle.band_mask(ref, rc, BAND)
    core = (ref["r"] < rc) & ~edge
    cl = P.cl_build(torch.from_numpy(xa).cuda(), h, rc, lcell)
    out = P.cl_cross_pairlist(cl, torch.from_numpy(yb).cuda())
    a, b, d = out["a"].cpu().numpy(), out["b"].cpu().numpy(), out["d"].cpu().numpy()
    key = b.astype(np.int64) * xa.shape[0] + a
    assert np.all(np.diff(key) > 0), "not sorted by (b, a)"
    want = set((ref["j"][core].astype(np.int64) * xa.shape[0] + ref["i"][core]).tolist())
    maybe = set((ref["j"][edge].astype(np.int64) * xa.shape[0] + ref["i"][edge]).tolist())
    got = set(key.tolist())
    assert want <= got and got <= want | maybe
    rmap = dict(zip((ref["j"].astype(np.int64) * xa.shape[0] + ref["i"]).tolist(), ref["r"].tolist()))
    assert max(abs(d[q] - rmap[key[q]]) for q in range(len(key))) <= 1e-6 * rc * 4


def test_cross_pairlist_dense_queries(cuda_ok):
    """Queries inside a dense cluster of A: more than 1024 neighbours each,
    sorted by the long-segment pass."""
    import paper_2202_06427_gb300 as P
    rng = np.random.default_rng(811)
    h = np.eye(3) * 30.0
    u = rng.normal(size=(3000, 3))
    u *= (2.0 * rng.uniform(0, 1, size=(3000, 1)) ** (1 / 3)) / np.linalg.norm(u, axis=1, keepdims=True)
    xa = np.vstack([rng.uniform(0, 30, size=(2000, 3)), u + 15.0])
    yb = np.vstack([rng.uniform(0, 30, size=(300, 3)), rng.normal(size=(40, 3)) + 15.0])
    rc = 5.0
    ref = oracle.cross_images(xa, yb, h, rc, band=BAND)
    edge = oracle.band_mask(ref, rc, BAND)
    core = (ref["r"] < rc) & ~edge
    cl = P.cl_build(torch.from_numpy(xa).cuda(), h, rc, 2)
    out = P.cl_cross_pairlist(cl, torch.from_numpy(yb).cuda())
    a, b, d = out["a"].cpu().numpy(), out["b"].cpu().numpy(), out["d"].cpu().numpy()
    assert np.bincount(b).max() > 1024
    key = b.astype(np.int64) * xa.shape[0] + a
    assert np.all(np.diff(key) > 0), "not sorted by (b, a)"
    want = set((ref["j"][core].astype(np.int64) * xa.shape[0] + ref["i"][core]).tolist())
    maybe = set((ref["j"][edge].astype(np.int64) * xa.shape[0] + ref["i"][edge]).tolist())
    got = set(key.tolist())
    assert want <= got and got <= want | maybe


def test_open_boundaries_match_oracle(cuda_ok):
    """No periodic boundaries (Sec. 4.1): the bounding box makes every image but
    the direct one lie beyond the cutoff, so the cell list gives exactly the
    pairs of the open system (the oracle's open-system sums, pinned against a
    direct double loop)."""
    import paper_2202_06427_gb300 as P
    rng = np.random.default_rng(901)
    xa = rng.normal(size=(2500, 3)) * 4.0 + np.array([100.0, -50.0, 3.0])
    yb = rng.normal(size=(1500, 3)) * 4.0 + np.array([101.0, -49.0, 2.0])
    rc = 1.2
    pa = torch.from_numpy(xa).cuda()
    pb = torch.from_numpy(yb).cuda()
    cl = P.cl_build_open(pa, rc, 2, pos2=pb)
    # within set A
    ref = oracle.open_pair_map(xa, rc, band=BAND, nbins=30)
    check_count(int(P.cl_map(cl, "count")["count"].item()), ref)
    check_energy(P.cl_map(cl, "energy")["energy"].item(), ref["energy"])
    efv = P.cl_map(cl, "energy_forces_virial")
    check_forces(efv["forces"].cpu().numpy(), ref["forces"])
    check_hist(P.cl_map(cl, "hist", nbins=30)["hist"].cpu().numpy(), ref)
    pl = P.cl_map(cl, "pairlist")
    rl = oracle.open_pairlist(xa, rc, band=BAND)
    got = set((pl["i"].cpu().numpy().astype(np.int64) * 2500 + pl["j"].cpu().numpy()).tolist())
    key = rl["i"] * 2500 + rl["j"]
    certain = (rl["d"] < rc) & ~rl["band"]
    assert set(key[certain].tolist()) <= got <= set(key.tolist())
    # across the two sets
    img = oracle.open_cross_images(xa, yb, rc, band=BAND)
    edge = oracle.band_mask(img, rc, BAND)
    inside = img["r"] < rc
    n_cross = P.cl_cross_count(cl, pb)
    assert int(np.sum(inside & ~edge)) <= n_cross <= int(np.sum(inside | edge))
    out = P.cl_cross_pairlist(cl, pb)
    got = set((out["b"].cpu().numpy().astype(np.int64) * 2500 + out["a"].cpu().numpy()).tolist())
    key = img["j"].astype(np.int64) * 2500 + img["i"]
    assert set(key[inside & ~edge].tolist()) <= got <= set(key[inside | edge].tolist())


def test_cross_errors(cuda_ok):
    import paper_2202_06427_gb300 as P
    from paper_2202_06427_gb300 import CellMapError
    h = np.eye(3) * 10.0
    cl = P.cl_build(torch.rand(100, 3, dtype=torch.float64, device="cuda") * 10, h, 2.0, 2)
    yb = torch.rand(50, 3, dtype=torch.float64, device="cuda") * 10
    for k in (0, 33):
        with pytest.raises(CellMapError):
            P.cl_cross_knn(cl, yb, k)
    bad = yb.clone()
    bad[3, 1] = float("nan")
    with pytest.raises(CellMapError) as e:
        P.cl_cross_count(cl, bad)
    assert e.value.code == -4
    cl2 = P.cl_build(torch.rand(100, 3, dtype=torch.float64, device="cuda") * 10, h, 6.0, 2)
    with pytest.raises(CellMapError) as e:
        P.cl_cross_pairlist(cl2, yb)
    assert e.value.code == -3
    empty = P.cl_cross_topk(cl, torch.zeros((0, 3), dtype=torch.float64, device="cuda"), 5)
    assert empty["n"] == 0
