"""FP64 CPU oracle for the cell-list pair map (CellListMap.jl, arXiv 2202.06427).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` import this package. It shares no code with the
CUDA library and the library never calls it.

Every function takes positions ``x`` as an (n, dim) float64 array and the
lattice matrix ``h`` as a (dim, dim) array whose ROWS are the lattice vectors.
Indices are 0-based. ``band`` is the relative half-width of the band around
the cutoff and the histogram bin edges inside which a pair may be classified
either way by a correct FP32 implementation (Sec. 2.3 leaves "within the
cutoff" at the edge unspecified; the library reads it as strict r < rc).

Functions and the passages they follow:
  pair_map      -- Sec. 2.3 (Code 2), 2.6, 2.8: every pair-image within rc, with
                   count, sum 1/r (Code 5), shifted-force energy, forces (Code 7
                   pattern), virial, dE/dH, histogram (Code 10 pattern).
  pairlist      -- Sec. 4.1 neighbour list, i<j, sorted by (i, j).
  particles     -- force and half pair energy of chosen particles, one by one.
  brute_map / brute_pairlist -- O(n^2 * images) definitions used to pin the above.
  images        -- Sec. 2.3 (Code 2): every pair-image with its displacement vector,
                   the input of the mapped function; brute_images pins it.
  cross_images  -- Sec. 3.2 (Code 8): pair-images between two sets of particles;
                   brute_cross_images pins it.
  lj            -- Code 6 (Lennard-Jones energy) and Code 7 (its forces), with the
                   virial, summed over images().
  mass_potential -- Code 5, second example: sum of m_i m_j / r.
  velocity_hist -- Code 10: pair counts and summed |v_i - v_j| per distance bin.
  knn_pairs     -- Code 8: the k cross pair-images of smallest distance.
  open_box / open_pair_map / open_pairlist / open_cross_images
                -- Sec. 4.1 without periodic boundaries: the pair-images of a
                   box wider than the points' extent plus the cutoff on every
                   axis are exactly the direct pairs of the open system.
  geom_info     -- widths between lattice faces and the cell grid for lcell.
  closed_form   -- see oracle.closed_form (perfect-lattice sums).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

ERRORS = {0: "ok", -1: "invalid argument", -2: "singular box", -3: "pair with two images in cutoff",
          -4: "capacity", -5: "out of memory"}


class OracleError(RuntimeError):
    pass


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        ll, i32, dbl = ctypes.c_longlong, ctypes.c_int, ctypes.c_double
        lib.or_geom_info.argtypes = [i32, P, dbl, i32, P, P, P]
        lib.or_map.argtypes = [i32, ll, P, P, dbl, dbl, ll, ll, i32, dbl, P, P, P, P, P, P, P]
        lib.or_brute_map.argtypes = [i32, ll, P, P, dbl, dbl, i32, dbl, P, P, P, P, P, P, P]
        lib.or_pairlist.argtypes = [i32, ll, P, P, dbl, dbl, ll, P, P, P, P, P]
        lib.or_brute_pairlist.argtypes = [i32, ll, P, P, dbl, dbl, ll, P, P, P, P, P]
        lib.or_particles.argtypes = [i32, ll, P, P, dbl, P, ll, P, P]
        lib.or_neighbors.argtypes = [i32, ll, P, P, dbl, dbl, P, ll, ll, P, P, P, P]
        lib.or_images.argtypes = [i32, ll, P, P, dbl, dbl, ll, P, P, P, P, P]
        lib.or_brute_images.argtypes = [i32, ll, P, P, dbl, dbl, ll, P, P, P, P, P]
        lib.or_cross_images.argtypes = [i32, ll, P, ll, P, P, dbl, dbl, ll, P, P, P, P, P]
        lib.or_brute_cross_images.argtypes = [i32, ll, P, ll, P, P, dbl, dbl, ll, P, P, P, P, P]
        for f in (lib.or_geom_info, lib.or_map, lib.or_brute_map, lib.or_pairlist,
                  lib.or_brute_pairlist, lib.or_particles, lib.or_neighbors, lib.or_images,
                  lib.or_brute_images, lib.or_cross_images, lib.or_brute_cross_images):
            f.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise OracleError(ERRORS.get(rc, str(rc)))


def _prep(x, h):
    x = np.ascontiguousarray(x, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    dim = h.shape[0]
    if h.shape != (dim, dim) or dim not in (2, 3) or x.ndim != 2 or x.shape[1] != dim:
        raise OracleError("shapes: x (n, dim), h (dim, dim), dim in (2, 3)")
    return x, h, dim


def geom_info(h, rc, lcell=1):
    h = np.ascontiguousarray(h, dtype=np.float64)
    dim = h.shape[0]
    w = np.zeros(3)
    n = np.zeros(3, dtype=np.int32)
    m = np.zeros(3, dtype=np.int32)
    _check(_lib().or_geom_info(dim, _p(h), rc, lcell, _p(w), _p(n), _p(m)))
    return {"w": w[:dim].copy(), "n": n[:dim].copy(), "m": m[:dim].copy()}


def _result(dim, n, nbins, counts, sums, forces, virial, dedh, hc, hm):
    out = {"count": int(counts[0]), "band_in": int(counts[1]), "band_out": int(counts[2]),
           "suminvr": float(sums[0]), "energy": float(sums[1]),
           "virial": virial.reshape(dim, dim), "dedh": dedh.reshape(dim, dim)}
    if forces is not None:
        out["forces"] = forces.reshape(n, dim)
    if nbins > 0:
        out["hist_core"] = hc
        out["hist_maybe"] = hm
    return out


def pair_map(x, h, rc, band=1e-6, nbins=0, rmax=None, forces=True, i_range=None):
    """All reductions over the pair-images within rc (restricted to pairs whose
    smaller index lies in ``i_range`` when given)."""
    x, h, dim = _prep(x, h)
    n = x.shape[0]
    lo, hi = (0, n) if i_range is None else i_range
    counts = np.zeros(3, dtype=np.int64)
    sums = np.zeros(2)
    f = np.zeros((n, dim)) if forces else None
    vir = np.zeros(dim * dim)
    dedh = np.zeros(dim * dim)
    hc = np.zeros(max(nbins, 1), dtype=np.int64)
    hm = np.zeros(max(nbins, 1), dtype=np.int64)
    _check(_lib().or_map(dim, n, _p(x), _p(h), rc, band, lo, hi, nbins, rmax or rc,
                         _p(counts), _p(sums), _p(f), _p(vir), _p(dedh),
                         _p(hc) if nbins else None, _p(hm) if nbins else None))
    return _result(dim, n, nbins, counts, sums, f, vir, dedh, hc[:nbins], hm[:nbins])


def brute_map(x, h, rc, band=1e-6, nbins=0, rmax=None):
    x, h, dim = _prep(x, h)
    n = x.shape[0]
    counts = np.zeros(3, dtype=np.int64)
    sums = np.zeros(2)
    f = np.zeros((n, dim))
    vir = np.zeros(dim * dim)
    dedh = np.zeros(dim * dim)
    hc = np.zeros(max(nbins, 1), dtype=np.int64)
    hm = np.zeros(max(nbins, 1), dtype=np.int64)
    _check(_lib().or_brute_map(dim, n, _p(x), _p(h), rc, band, nbins, rmax or rc,
                               _p(counts), _p(sums), _p(f), _p(vir), _p(dedh),
                               _p(hc) if nbins else None, _p(hm) if nbins else None))
    return _result(dim, n, nbins, counts, sums, f, vir, dedh, hc[:nbins], hm[:nbins])


def _pairlist(fn, x, h, rc, band, cap):
    x, h, dim = _prep(x, h)
    n = x.shape[0]
    while True:
        pi = np.zeros(cap, dtype=np.int64)
        pj = np.zeros(cap, dtype=np.int64)
        pd = np.zeros(cap)
        pb = np.zeros(cap, dtype=np.int8)
        npairs = np.zeros(1, dtype=np.int64)
        rc_ = fn(dim, n, _p(x), _p(h), rc, band, cap, _p(pi), _p(pj), _p(pd), _p(pb), _p(npairs))
        if rc_ == -4:
            cap *= 4
            continue
        _check(rc_)
        k = int(npairs[0])
        return {"i": pi[:k], "j": pj[:k], "d": pd[:k], "band": pb[:k].astype(bool)}


def pairlist(x, h, rc, band=1e-6, cap=1 << 20):
    """Sorted i<j list of pairs with r < rc(1 + 4 band); ``band`` flags the
    pairs with |r - rc| <= band*rc."""
    return _pairlist(_lib().or_pairlist, x, h, rc, band, cap)


def brute_pairlist(x, h, rc, band=1e-6, cap=1 << 16):
    return _pairlist(_lib().or_brute_pairlist, x, h, rc, band, cap)


def particles(x, h, rc, idx):
    """Force (-dE/dx) and half pair energy of each particle in ``idx``."""
    x, h, dim = _prep(x, h)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    f = np.zeros((idx.shape[0], dim))
    e = np.zeros(idx.shape[0])
    _check(_lib().or_particles(dim, x.shape[0], _p(x), _p(h), rc, _p(idx), idx.shape[0], _p(f), _p(e)))
    return f, e


def neighbors(x, h, rc, idx, band=1e-6):
    """For each a in idx: its j > a with r < rc(1 + 4 band), sorted by j.
    Returns a list of dicts {"j", "d", "band"}."""
    x, h, dim = _prep(x, h)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    k = idx.shape[0]
    cap = max(1024, 512 * k)
    while True:
        offs = np.zeros(k + 1, dtype=np.int64)
        oj = np.zeros(cap, dtype=np.int64)
        od = np.zeros(cap)
        ob = np.zeros(cap, dtype=np.int8)
        rc_ = _lib().or_neighbors(dim, x.shape[0], _p(x), _p(h), rc, band, _p(idx), k, cap, _p(offs), _p(oj),
                                  _p(od), _p(ob))
        if rc_ == -4:
            cap = int(offs[k]) + 1
            continue
        _check(rc_)
        return [{"j": oj[offs[q]:offs[q + 1]], "d": od[offs[q]:offs[q + 1]],
                 "band": ob[offs[q]:offs[q + 1]].astype(bool)} for q in range(k)]


def energy(x, h, rc):
    """Shifted-force energy alone (no forces)."""
    return pair_map(x, h, rc, forces=False)["energy"]


def _images(call, dim, cap):
    while True:
        pi = np.zeros(cap, dtype=np.int64)
        pj = np.zeros(cap, dtype=np.int64)
        rv = np.zeros((cap, dim))
        r = np.zeros(cap)
        nimg = np.zeros(1, dtype=np.int64)
        rc_ = call(cap, pi, pj, rv, r, nimg)
        if rc_ == -4:
            cap = int(nimg[0]) + 1
            continue
        _check(rc_)
        k = int(nimg[0])
        return {"i": pi[:k], "j": pj[:k], "rv": rv[:k], "r": r[:k]}


def images(x, h, rc, band=1e-6, cap=1 << 20):
    """Every pair-image (i < j, image t) with r < rc(1 + 4 band): arrays i, j,
    rv = x_j - x_i + t.H (n_img, dim) and r. Pairs with r >= rc are only there
    so that a test can accept an FP32 inclusion; ``band_mask`` selects them."""
    x, h, dim = _prep(x, h)
    n = x.shape[0]
    return _images(lambda c, a, b, v, r, k: _lib().or_images(dim, n, _p(x), _p(h), rc, band, c, _p(a), _p(b), _p(v),
                                                             _p(r), _p(k)), dim, cap)


def brute_images(x, h, rc, band=1e-6, cap=1 << 16):
    x, h, dim = _prep(x, h)
    n = x.shape[0]
    return _images(lambda c, a, b, v, r, k: _lib().or_brute_images(dim, n, _p(x), _p(h), rc, band, c, _p(a), _p(b),
                                                                   _p(v), _p(r), _p(k)), dim, cap)


def cross_images(xa, yb, h, rc, band=1e-6, cap=1 << 20):
    """Pair-images between the sets xa and yb (Code 8): every (a, b, t) with
    |y_b - x_a + t.H| < rc(1 + 4 band); arrays i (= a), j (= b), rv, r."""
    xa, h, dim = _prep(xa, h)
    yb = np.ascontiguousarray(yb, dtype=np.float64).reshape(-1, dim)
    na, nb = xa.shape[0], yb.shape[0]
    return _images(lambda c, a, b, v, r, k: _lib().or_cross_images(dim, na, _p(xa), nb, _p(yb), _p(h), rc, band, c,
                                                                   _p(a), _p(b), _p(v), _p(r), _p(k)), dim, cap)


def brute_cross_images(xa, yb, h, rc, band=1e-6, cap=1 << 16):
    xa, h, dim = _prep(xa, h)
    yb = np.ascontiguousarray(yb, dtype=np.float64).reshape(-1, dim)
    na, nb = xa.shape[0], yb.shape[0]
    return _images(lambda c, a, b, v, r, k: _lib().or_brute_cross_images(dim, na, _p(xa), nb, _p(yb), _p(h), rc,
                                                                         band, c, _p(a), _p(b), _p(v), _p(r), _p(k)),
                   dim, cap)


def band_mask(img, rc, band=1e-6):
    """Images whose distance lies within band*rc of the cutoff."""
    return np.abs(img["r"] - rc) <= band * rc


def lj(x, h, rc, eps, sigma, band=1e-6, img=None):
    """Lennard-Jones energy of Code 6, u(r) = 4 eps ((sigma^2/r^2)^6 - (sigma^2/r^2)^3),
    over the pair-images with r < rc (not shifted), its forces F = -dE/dx (the
    gradient of that energy; Code 7 accumulates f[i] += g, f[j] -= g) and the
    virial W = -sum u'(r)/r rv (x) rv. Also the same sums over the band pairs
    alone, the amount by which an FP32 classification may differ."""
    if img is None:
        img = images(x, h, rc, band)
    n, dim = np.asarray(x).shape
    inside = img["r"] < rc
    edge = band_mask(img, rc, band)
    out = {}
    for key, sel in (("", inside & ~edge), ("band_", edge)):
        r, rv, i, j = img["r"][sel], img["rv"][sel], img["i"][sel], img["j"][sel]
        q = (sigma * sigma) / (r * r)
        q3 = q * q * q
        u = 4.0 * eps * (q3 * q3 - q3)
        dudr_over_r = -24.0 * eps * (2.0 * q3 * q3 - q3) / (r * r)   # u'(r)/r
        g = dudr_over_r[:, None] * rv                                # F_i += g, F_j -= g
        f = np.zeros((n, dim))
        np.add.at(f, i, g)
        np.add.at(f, j, -g)
        out[key + "energy"] = float(np.sum(u))
        out[key + "forces"] = f
        out[key + "virial"] = -(rv * dudr_over_r[:, None]).T @ rv
        out[key + "abs_energy"] = float(np.sum(np.abs(u)))
    return out


def mass_potential(x, h, rc, m, band=1e-6, img=None):
    """Code 5, second example: sum over pair-images within rc of m_i m_j / r;
    also the part of the band pairs."""
    if img is None:
        img = images(x, h, rc, band)
    m = np.asarray(m, dtype=np.float64)
    inside = img["r"] < rc
    edge = band_mask(img, rc, band)
    term = m[img["i"]] * m[img["j"]] / img["r"]
    return {"value": float(np.sum(term[inside & ~edge])), "band": float(np.sum(np.abs(term[edge])))}


def velocity_hist(x, h, rc, v, binstep, nbins, band=1e-6, img=None):
    """Code 10: for each pair-image within rc, bin k = ceil(r / binstep)
    (1-based, bins closed on the right); when k <= nbins the pair adds 1 to
    counts[k-1] and |v_i - v_j| to vsum[k-1]. Returns counts and vsum over the
    pairs away from the cutoff and the bin edges (by band*rc), and the same over
    the pairs near them (either classification is correct)."""
    if img is None:
        img = images(x, h, rc, band)
    v = np.asarray(v, dtype=np.float64)
    r = img["r"]
    k = np.ceil(r / binstep).astype(np.int64)
    near_edge = np.abs(r - np.round(r / binstep) * binstep) <= band * rc
    edge = band_mask(img, rc, band) | near_edge
    take = (r < rc) & (k >= 1) & (k <= nbins)
    dv = np.linalg.norm(v[img["i"]] - v[img["j"]], axis=1)
    out = {}
    for key, sel in (("", take & ~edge), ("band_", edge & (r < rc * (1 + 4 * band)))):
        out[key + "counts"] = np.bincount(k[sel] - 1, minlength=nbins)[:nbins] if np.any(sel) else np.zeros(nbins, np.int64)
        out[key + "vsum"] = (np.bincount(k[sel] - 1, weights=dv[sel], minlength=nbins)[:nbins]
                             if np.any(sel) else np.zeros(nbins))
    return out


def knn_pairs(xa, yb, h, rc, k, band=1e-6, img=None):
    """Code 8: the k cross pair-images (a in xa, b in yb) of smallest distance
    among those within rc, ordered by distance (fewer when fewer exist). Returns
    arrays i (= a), j (= b), r, and the distance of the k-th pair."""
    if img is None:
        img = cross_images(xa, yb, h, rc, band)
    sel = img["r"] < rc
    order = np.lexsort((img["j"][sel], img["i"][sel], img["r"][sel]))[:k]
    r = img["r"][sel][order]
    return {"i": img["i"][sel][order], "j": img["j"][sel][order], "r": r}


def open_box(*sets, rc):
    """Orthorhombic box for points without periodic boundaries (Sec. 4.1): on
    every axis the side exceeds the extent of all points plus rc + 1, so for
    any two points every lattice image but the direct one lies more than
    rc + 1 away, beyond rc(1 + 4 band)."""
    allx = np.vstack([np.asarray(x, dtype=np.float64) for x in sets if len(x)])
    dim = allx.shape[1]
    ext = allx.max(axis=0) - allx.min(axis=0) if allx.shape[0] else np.zeros(dim)
    return np.diag(ext + rc + 1.0)


def open_pair_map(x, rc, band=1e-6, nbins=0, rmax=None, forces=True):
    """pair_map over the direct pairs i < j with r < rc of an open system."""
    return pair_map(x, open_box(x, rc=rc), rc, band=band, nbins=nbins, rmax=rmax, forces=forces)


def open_pairlist(x, rc, band=1e-6):
    return pairlist(x, open_box(x, rc=rc), rc, band=band)


def open_cross_images(xa, yb, rc, band=1e-6):
    """cross_images between two open sets: every (a, b) with |y_b - x_a| < rc(1 + 4 band)."""
    return cross_images(xa, yb, open_box(xa, yb, rc=rc), rc, band=band)
