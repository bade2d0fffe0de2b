"""Helpers shared by the GPU parity tests: tolerances, comparison rules and a
spawn-based pool that runs the (single-threaded) oracle on index ranges.

Tolerances. A pair whose FP64 distance lies within BAND * rc of the cutoff (or
of a bin edge) may be decided either way by a correct FP32 path; the oracle
counts such band pairs apart. The floating-point rules follow from FP32 pair
terms on cell-centred coordinates (relative error of order 1e-7 per term)
summed in FP64:
  counts       exact outside the band: oracle count - band_in <= gpu <= count + band_out
  histograms   exact outside the band: core[k] <= gpu[k] <= core[k] + maybe[k]
  sum 1/r      relative 1e-6, plus 1/rc for every band pair that may flip
  energy       relative 1e-6 (u and u' vanish at rc, band pairs add nothing)
  forces       max-norm 1e-5 relative to the largest oracle force component
  virial       1e-6 relative to its largest component
  box gradient 1e-5 relative to its largest component (X - W mixes FP32 forces
               with raw positions)
"""
import multiprocessing as mp

import numpy as np

BAND = 1e-6
TOL_E = 1e-6
TOL_F = 1e-5
TOL_W = 1e-6
TOL_GB = 1e-5


def check_count(gpu, ref):
    lo, hi = ref["count"] - ref["band_in"], ref["count"] + ref["band_out"]
    assert lo <= gpu <= hi, "count %d outside [%d, %d]" % (gpu, lo, hi)


def check_hist(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.int64)
    core, maybe = ref["hist_core"], ref["hist_maybe"]
    assert np.all(gpu >= core), "bins below the certain count: %s" % np.where(gpu < core)[0][:10]
    assert np.all(gpu <= core + maybe), "bins above the possible count: %s" % np.where(gpu > core + maybe)[0][:10]


def check_suminvr(gpu, ref, rc):
    slack = TOL_E * abs(ref["suminvr"]) + (ref["band_in"] + ref["band_out"]) / rc * (1 + 1e-5)
    assert abs(gpu - ref["suminvr"]) <= slack, (gpu, ref["suminvr"], slack)


def check_energy(gpu, ref_e):
    assert abs(gpu - ref_e) <= TOL_E * abs(ref_e) + 1e-12, (gpu, ref_e, abs(gpu - ref_e) / abs(ref_e))


def check_forces(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    scale = np.abs(ref).max()
    err = np.abs(gpu - ref).max()
    assert err <= TOL_F * scale, "force max-norm error %.3g > %.3g (scale %.3g)" % (err, TOL_F * scale, scale)
    return err / scale


def check_matrix(gpu, ref, tol):
    gpu = np.asarray(gpu, dtype=np.float64)
    scale = np.abs(ref).max()
    err = np.abs(gpu - ref).max()
    assert err <= tol * scale, "matrix error %.3g > %.3g\n%s\n%s" % (err, tol * scale, gpu, ref)
    return err / scale


def _part(args):
    import oracle
    path, h, rc, nbins, forces, lo, hi = args
    x = np.load(path, mmap_mode="r")
    return oracle.pair_map(x, h, rc, band=BAND, nbins=nbins, forces=forces, i_range=(lo, hi))


def oracle_pool(x, h, rc, nbins=0, forces=True, nproc=None):
    """oracle.pair_map over the whole set, split by the smaller index into
    chunks run in a spawn pool (the oracle itself stays single-threaded).
    The positions reach the workers through a memory-mapped file."""
    import tempfile
    n = x.shape[0]
    nproc = nproc or min(16, mp.cpu_count())
    # the smaller index carries more pairs at the start of the range: cut finer chunks
    cuts = np.unique(np.linspace(0, n, 4 * nproc + 1).astype(np.int64))
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as tmp:
        path = tmp + "/x.npy"
        np.save(path, np.ascontiguousarray(x, dtype=np.float64))
        jobs = [(path, h, rc, nbins, forces, int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:])]
        with ctx.Pool(nproc) as pool:
            parts = pool.map(_part, jobs)
    out = {k: sum(p[k] for p in parts) for k in ("count", "band_in", "band_out", "suminvr", "energy")}
    out["virial"] = sum(p["virial"] for p in parts)
    out["dedh"] = sum(p["dedh"] for p in parts)
    if forces:
        out["forces"] = sum(p["forces"] for p in parts)
    if nbins:
        out["hist_core"] = sum(p["hist_core"] for p in parts)
        out["hist_maybe"] = sum(p["hist_maybe"] for p in parts)
    return out


def _rows_part(args):
    """Compare the GPU list's rows [lo, hi) with the oracle's rows (spawned worker)."""
    import ctypes
    import oracle
    path, h, rc, lo, hi, gi, gj, gd = args
    x = np.load(path, mmap_mode="r")
    n = x.shape[0]
    idx = np.arange(lo, hi, dtype=np.int64)
    k = idx.shape[0]
    cap = max(1024, 4 * gj.shape[0] + 1024)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    xc = np.ascontiguousarray(x)
    hc = np.ascontiguousarray(h, dtype=np.float64)
    while True:
        offs = np.zeros(k + 1, dtype=np.int64)
        oj = np.zeros(cap, dtype=np.int64)
        od = np.zeros(cap)
        ob = np.zeros(cap, dtype=np.int8)
        ret = oracle._lib().or_neighbors(3 if hc.shape[0] == 3 else 2, n, p(xc), p(hc), rc, BAND, p(idx), k, cap,
                                         p(offs), p(oj), p(od), p(ob))
        if ret == -4:
            cap = int(offs[k]) + 1
            continue
        assert ret == 0, ret
        break
    m = int(offs[k])
    oi = np.repeat(idx, np.diff(offs))
    okey = oi * n + oj[:m]
    od, ob = od[:m], ob[:m].astype(bool)
    gkey = gi.astype(np.int64) * n + gj
    certain = (od < rc) & ~ob
    missing = int(np.sum(~np.isin(okey[certain], gkey)))
    pos = np.searchsorted(okey, gkey)
    known = (pos < m) & (okey[np.minimum(pos, m - 1)] == gkey)
    extra = int(np.sum(~known))
    derr = np.abs(gd[known].astype(np.float64) - od[pos[known]])
    return {"rows": k, "pairs": int(gkey.shape[0]), "oracle_certain": int(certain.sum()), "band": int(ob.sum()),
            "missing": missing, "extra": extra, "max_d_err": float(derr.max()) if derr.size else 0.0}


def pairlist_pool_check(x, h, rc, gi, gj, gd, nproc=None, chunks_per_proc=4):
    """Whole-list comparison of a sorted GPU pair list (gi, gj, gd host arrays,
    sorted by (i, j)) with the oracle's rows, chunked by index range in a
    spawn pool: per chunk the oracle lists the rows' neighbours j > i and the
    GPU slice of those rows is compared against them. Returns the summed
    counts of missing pairs (certain oracle pairs absent), extra pairs (absent
    from the oracle's band-widened rows) and the largest distance error."""
    import tempfile
    n = x.shape[0]
    nproc = nproc or min(16, mp.cpu_count())
    cuts = np.unique(np.linspace(0, n, chunks_per_proc * nproc + 1).astype(np.int64))
    bounds = np.searchsorted(gi, cuts)
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as tmp:
        path = tmp + "/x.npy"
        np.save(path, np.ascontiguousarray(x, dtype=np.float64))
        jobs = [(path, h, rc, int(a), int(b), gi[s0:s1], gj[s0:s1], gd[s0:s1])
                for a, b, s0, s1 in zip(cuts[:-1], cuts[1:], bounds[:-1], bounds[1:])]
        with ctx.Pool(nproc) as pool:
            parts = pool.map(_rows_part, jobs, chunksize=1)
    out = {k: sum(p[k] for p in parts) for k in ("rows", "pairs", "oracle_certain", "band", "missing", "extra")}
    out["max_d_err"] = max(p["max_d_err"] for p in parts)
    return out
