"""GPU neighbour list (sorted i<j, FP32 distance) and histogram against the
oracle, including the 1M triclinic workload (rows (220,0,0), (30,215,0),
(20,25,210), rc 10, 200-bin histogram)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import BAND, check_count, check_hist, oracle_pool, pairlist_pool_check

pytestmark = pytest.mark.gpu


def _P():
    import paper_2202_06427_gb300 as P
    return P


def check_row(gpu_j, gpu_d, ref, rc):
    """One particle's row: every certain oracle neighbour present, nothing
    outside the oracle's band-widened row, distances within 1e-6 rc."""
    certain = ref["j"][(ref["d"] < rc) & ~ref["band"]]
    assert np.all(np.diff(gpu_j) > 0), "row not strictly increasing"
    assert np.isin(certain, gpu_j).all(), "missing neighbours"
    pos = np.searchsorted(ref["j"], gpu_j)
    assert np.all(pos < len(ref["j"])) and np.array_equal(ref["j"][np.minimum(pos, len(ref["j"]) - 1)], gpu_j), \
        "neighbours the oracle does not have"
    assert np.all(np.abs(gpu_d - ref["d"][pos]) <= BAND * rc)


def check_list_structure(pl, n, rc):
    i, j, d = (pl[k].cpu().numpy() for k in ("i", "j", "d"))
    assert np.all(i < j) and np.all(i >= 0) and np.all(j < n)
    key = i.astype(np.int64) * n + j
    assert np.all(np.diff(key) > 0), "not sorted by (i, j) or duplicated"
    assert np.all(d < rc * (1 + 1e-6)) and np.all(d >= 0)
    return i, j, d


@pytest.mark.parametrize("dim,tric,lcell", [(2, False, 2), (2, True, 3), (3, False, 1), (3, True, 2), (3, True, 4)])
def test_small_pairlist_equals_oracle(cuda_ok, dim, tric, lcell):
    P = _P()
    rng = np.random.default_rng(40 + dim * 7 + lcell + int(tric))
    L = 30.0 if dim == 3 else 50.0
    h = np.eye(dim) * L
    if tric:
        for a in range(1, dim):
            for b in range(a):
                h[a, b] = rng.uniform(-0.25 * L, 0.25 * L)
    n_side = int(L)
    x = synth.jittered_fractional(h, n_side, n_side ** dim - 3 * n_side, 0.4, 99)
    x = x + rng.integers(-2, 3, size=x.shape).astype(np.float64) @ h
    rc = 3.0 if dim == 3 else 4.0
    ref = oracle.pairlist(x, h, rc, band=BAND)
    cl = P.cl_build(torch.from_numpy(np.ascontiguousarray(x)).cuda(), h, rc, lcell)
    pl = P.cl_map(cl, "pairlist")
    i, j, d = check_list_structure(pl, x.shape[0], rc)
    certain = ~ref["band"] | (ref["d"] < rc - BAND * rc)
    gk = i.astype(np.int64) * x.shape[0] + j
    rk = ref["i"] * x.shape[0] + ref["j"]
    assert np.isin(rk[certain & (ref["d"] < rc)], gk).all()
    pos = np.searchsorted(rk, gk)
    assert np.array_equal(rk[np.minimum(pos, len(rk) - 1)], gk)
    assert np.all(np.abs(d - ref["d"][pos]) <= BAND * rc)
    assert pl["npairs"] == len(i)
    ref_map = oracle.pair_map(x, h, rc, band=BAND, forces=False)
    check_count(pl["npairs"], ref_map)  # a band pair may round differently than in the half-shell count


def _cluster_case(n_bg, n_cl, radius, seed, tric):
    rng = np.random.default_rng(seed)
    L = 30.0
    h = np.eye(3) * L
    if tric:
        h[1, 0], h[2, 0], h[2, 1] = 4.0, -3.0, 5.0
    bg = rng.uniform(0, 1, size=(n_bg, 3)) @ h
    u = rng.normal(size=(n_cl, 3))
    u *= (radius * rng.uniform(0, 1, size=(n_cl, 1)) ** (1 / 3)) / np.linalg.norm(u, axis=1, keepdims=True)
    x = np.vstack([bg, u + np.array([15.0, 14.0, 16.0])])
    return x[rng.permutation(x.shape[0])], h


def _check_against_oracle(P, x, h, rc, lcell):
    ref = oracle.pairlist(x, h, rc, band=BAND)
    cl = P.cl_build(torch.from_numpy(np.ascontiguousarray(x)).cuda(), h, rc, lcell)
    pl = P.cl_map(cl, "pairlist")
    i, j, d = check_list_structure(pl, x.shape[0], rc)
    certain = ~ref["band"] | (ref["d"] < rc - BAND * rc)
    gk = i.astype(np.int64) * x.shape[0] + j
    rk = ref["i"] * x.shape[0] + ref["j"]
    assert np.isin(rk[certain & (ref["d"] < rc)], gk).all()
    pos = np.searchsorted(rk, gk)
    assert np.array_equal(rk[np.minimum(pos, len(rk) - 1)], gk)
    assert np.all(np.abs(d - ref["d"][pos]) <= BAND * rc)
    return np.bincount(i, minlength=x.shape[0])


@pytest.mark.parametrize("tric,lcell", [(False, 1), (True, 2)])
def test_pairlist_dense_cluster(cuda_ok, tric, lcell):
    """A dense cluster in a sparse background: the cells around the cluster
    hold more neighbours than one cell's staging area (they take the
    per-particle path) and its particles have segments longer than one warp
    sorts in shared memory (they take the long-segment sort)."""
    P = _P()
    x, h = _cluster_case(4000, 2500, 2.5, 71 + lcell, tric)
    seg = _check_against_oracle(P, x, h, 6.0, lcell)
    assert seg.max() > 2000


def test_pairlist_long_segments_in_staged_cells(cuda_ok):
    """A cluster whose neighbourhood still fits the staging area: segments
    longer than 1024 written directly by the staged sweep."""
    P = _P()
    x, h = _cluster_case(800, 1500, 2.0, 77, False)
    seg = _check_against_oracle(P, x, h, 6.0, 1)
    assert seg.max() > 1024


def test_pairlist_capacity_protocol(cuda_ok):
    import ctypes
    from paper_2202_06427_gb300 import _lib
    P = _P()
    h = np.eye(3) * 20.0
    x = synth.jittered_fractional(h, 20, 8000, 0.4, 5)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, 3.0, 2)
    total = P.cl_map(cl, "pairlist")["npairs"]
    small = P.cl_map(cl, "pairlist", capacity=total)  # exactly enough
    assert small["npairs"] == total
    res = _lib.cl_result()
    npairs = ctypes.c_longlong(0)
    res.capacity = total - 1
    res.npairs = ctypes.pointer(npairs)
    buf = torch.empty(total, dtype=torch.int32, device="cuda")
    res.pair_i = res.pair_j = buf.data_ptr()
    res.pair_d = buf.data_ptr()
    code = _lib.lib().cl_map(cl.handle, 5, None, ctypes.byref(res), ctypes.c_void_p(0))
    assert code == -6 and npairs.value == total
    # a cutoff above half the box: pairs may have two images, the list is refused
    cl2 = P.cl_build(torch.from_numpy(x).cuda(), h, 11.0, 1)
    with pytest.raises(P.CellMapError) as e:
        P.cl_map(cl2, "pairlist")
    assert e.value.code == -3


@pytest.mark.slow
def test_workload_triclinic_1m(cuda_ok):
    P = _P()
    w = synth.w2_triclinic()
    x, h, rc, nbins = w["x"], w["h"], w["rc"], w["nbins"]
    n = x.shape[0]
    ref = oracle_pool(x, h, rc, nbins=nbins, forces=False)
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, 2)
    check_hist(P.cl_map(cl, "hist", nbins=nbins)["hist"].cpu().numpy(), ref)
    cnt = int(P.cl_map(cl, "count")["count"].item())
    check_count(cnt, ref)
    pl = P.cl_map(cl, "pairlist")
    check_count(pl["npairs"], ref)  # tested from the smaller index's end: band pairs may differ from cnt
    assert 2.0e8 < cnt < 2.2e8
    i, j, d = check_list_structure(pl, n, rc)
    # the whole list, row by row, against the oracle's rows (chunked in a pool)
    whole = pairlist_pool_check(x, h, rc, i, j, d)
    assert whole["rows"] == n and whole["pairs"] == len(i)
    assert whole["missing"] == 0 and whole["extra"] == 0, whole
    assert whole["max_d_err"] <= BAND * rc, whole
    rows = np.random.default_rng(3).choice(n, size=1500, replace=False)
    rows = np.sort(np.concatenate([rows, [0, n - 1]]))
    refs = oracle.neighbors(x, h, rc, rows, band=BAND)
    starts = np.searchsorted(i, rows, side="left")
    ends = np.searchsorted(i, rows, side="right")
    for a, s0, s1, r in zip(rows, starts, ends, refs):
        check_row(j[s0:s1], d[s0:s1], r, rc)
