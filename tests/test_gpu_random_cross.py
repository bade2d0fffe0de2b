"""Randomised two-set sweep (Code 8): seeded random boxes (2D/3D, orthorhombic
or triclinic), lcell 1-4, cutoffs up to 0.45 of the smallest width, ragged set
sizes, query points far outside the box and, in 3D, queries inside a dense
sphere of the indexed set. Cross count, per-query k nearest, the k closest
cross pairs and the cross pair list against the oracle's cross pair-images."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import BAND

pytestmark = pytest.mark.gpu


def _config(seed):
    rng = np.random.default_rng(9500 + seed)
    dim = 3 if seed % 3 else 2
    tric = bool(seed % 2)
    lcell = 1 + seed % 4
    L = float(rng.integers(12, 19)) if dim == 3 else float(rng.integers(24, 41))
    h = np.eye(dim) * L
    if tric:
        for a in range(1, dim):
            for b in range(a):
                h[a, b] = rng.uniform(-0.3 * L, 0.3 * L)
    n_side = int(L)
    xa = synth.jittered_fractional(h, n_side, int(n_side ** dim * rng.uniform(0.5, 1.0)), 0.35, 9600 + seed)
    nb = int(rng.integers(50, 1500))
    yb = rng.uniform(0, 1, size=(nb, dim)) @ h
    if dim == 3 and seed % 4 == 2:  # a dense sphere of A with queries inside it
        c = rng.uniform(0.3, 0.7, size=3) @ h
        g = np.stack(np.meshgrid(*[np.arange(-6, 7) * 0.5] * 3, indexing="ij"), -1).reshape(-1, 3)
        g = g[np.linalg.norm(g, axis=1) <= 2.8]
        xa = np.vstack([xa, c + g + rng.uniform(-0.08, 0.08, size=g.shape)])
        yb = np.vstack([yb, c + rng.normal(size=(60, 3))])
    xa = xa + rng.integers(-3, 4, size=xa.shape).astype(np.float64) @ h
    yb = yb + rng.integers(-3, 4, size=yb.shape).astype(np.float64) @ h
    w = oracle.geom_info(h, 1.0)["w"]
    rc = float(min(rng.uniform(0.12, 0.45) * w.min(), 4.5 if dim == 3 else 6.0))
    return lcell, np.ascontiguousarray(xa), np.ascontiguousarray(yb), h, rc


@pytest.mark.parametrize("seed", range(24))
def test_random_two_sets(cuda_ok, seed):
    import paper_2202_06427_gb300 as P
    lcell, xa, yb, h, rc = _config(seed)
    ref = oracle.cross_images(xa, yb, h, rc, band=BAND)
    inside = ref["r"] < rc
    edge = oracle.band_mask(ref, rc, BAND)
    core = inside & ~edge
    cl = P.cl_build(torch.from_numpy(xa).cuda(), h, rc, lcell)
    yb_t = torch.from_numpy(yb).cuda()
    got = P.cl_cross_count(cl, yb_t)
    assert int(np.sum(core)) <= got <= int(np.sum(core)) + int(np.sum(edge)), got
    # per-query k nearest, on every query whose neighbours hold no band pair
    k = 1 + seed % 9
    a, d = P.cl_cross_knn(cl, yb_t, k)
    a, d = a.cpu().numpy(), d.cpu().numpy()
    for b in range(yb.shape[0]):
        mine = ref["j"] == b
        if np.any(edge[mine]):
            continue
        want = np.sort(ref["r"][mine & inside])[:k]
        m = len(want)
        assert np.allclose(d[b, :m], want, rtol=2e-6, atol=2e-6 * rc), b
        assert np.all(a[b, m:] == -1) and np.all(np.isinf(d[b, m:]))
    # the k closest cross pairs: distances (positions are a jittered lattice and uniform queries:
    # ties are not expected)
    kt = 1 + seed % 17
    top = P.cl_cross_topk(cl, yb_t, kt)
    want = oracle.knn_pairs(xa, yb, h, rc, kt, img=ref)
    assert top["n"] == len(want["r"])
    assert np.allclose(top["d"][:top["n"]].cpu().numpy(), want["r"], rtol=0, atol=4e-6 * rc)
    # the cross list sorted by (b, a)
    out = P.cl_cross_pairlist(cl, yb_t)
    ga, gb, gd = out["a"].cpu().numpy(), out["b"].cpu().numpy(), out["d"].cpu().numpy()
    key = gb.astype(np.int64) * xa.shape[0] + ga
    assert np.all(np.diff(key) > 0)
    want_keys = set((ref["j"][core].astype(np.int64) * xa.shape[0] + ref["i"][core]).tolist())
    maybe = set((ref["j"][edge].astype(np.int64) * xa.shape[0] + ref["i"][edge]).tolist())
    got_keys = set(key.tolist())
    assert want_keys <= got_keys and got_keys <= want_keys | maybe
    rmap = dict(zip((ref["j"].astype(np.int64) * xa.shape[0] + ref["i"]).tolist(), ref["r"].tolist()))
    assert max((abs(gd[q] - rmap[key[q]]) for q in range(len(key))), default=0.0) <= 4e-6 * rc
