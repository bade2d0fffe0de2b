"""Closed-form pair sums for perfect Bravais lattices.

TEST INFRASTRUCTURE (part of the oracle package; pins the oracle, never used by
the product path).

For a perfect lattice with unit cell rows ``b`` (dim x dim) tiled periodically
(any commensurate box whose faces are more than rc apart), the pair-images of
every site are exactly the lattice vectors v = k.b, k integer, 0 < |v| < rc:
Sec. 2.6's ghost copies give each real particle "the correct number of
neighbours", here the full shells of the lattice. Over the N sites every
unordered pair-image is seen from both ends, so

    count  = N/2 * #{v}
    sum1/r = N/2 * sum_v 1/|v|
    E_sf   = N/2 * sum_v u(|v|),   u(r) = 1/r - 1/rc + (r - rc)/rc^2
    W      = N/2 * sum_v -u'(|v|)/|v| v (x) v
    F_i    = 0 for every site (inversion symmetry)
    hist_k = N/2 * #{v : floor(|v| nbins / rmax) = k}

The vectors are enumerated by brute force over an integer box; nothing here
uses a cell list.
"""
import itertools
import math

import numpy as np


def lattice_vectors(b, rc):
    """All lattice vectors v = k.b with 0 < |v| < rc, as an (m, dim) array."""
    b = np.asarray(b, dtype=np.float64)
    dim = b.shape[0]
    binv = np.linalg.inv(b)
    widths = 1.0 / np.sqrt((binv ** 2).sum(axis=0))
    kmax = [int(math.ceil(rc / w)) + 1 for w in widths]
    out = []
    for k in itertools.product(*[range(-m, m + 1) for m in kmax]):
        if not any(k):
            continue
        v = np.asarray(k, dtype=np.float64) @ b
        if math.sqrt(float(v @ v)) < rc:
            out.append(v)
    return np.asarray(out).reshape(-1, dim)


def lattice_sums(b, rc, nsites, nbins=0, rmax=None, band=1e-6):
    """Closed-form reductions for ``nsites`` sites of the lattice ``b``.

    Returns the same keys as ``oracle.pair_map`` (``forces`` excepted), plus
    ``min_edge_gap``: the smallest distance between a shell radius and the
    cutoff or a bin edge, relative to rc (so a test can tell that no shell sits
    inside the rounding band)."""
    v = lattice_vectors(b, rc)
    r = np.sqrt((v * v).sum(axis=1))
    half = nsites / 2.0
    up = -1.0 / r ** 2 + 1.0 / rc ** 2
    u = 1.0 / r - 1.0 / rc + (r - rc) / rc ** 2
    dim = v.shape[1]
    vir = np.zeros((dim, dim))
    for a in range(dim):
        for c in range(dim):
            vir[a, c] = half * float(np.sum(-up / r * v[:, a] * v[:, c]))
    out = {"count": int(round(half * len(v))), "suminvr": half * float(np.sum(1.0 / r)),
           "energy": half * float(np.sum(u)), "virial": vir, "nvec": len(v)}
    edges = [rc]
    if nbins:
        rmax = rmax or rc
        k = np.floor(r * nbins / rmax).astype(np.int64)
        hist = np.zeros(nbins, dtype=np.int64)
        ok = r < min(rc, rmax)
        np.add.at(hist, k[ok], 1)
        out["hist"] = (hist * nsites) // 2
        edges += [rmax * e / nbins for e in range(1, nbins + 1)]
    vw = lattice_vectors(b, rc * 1.01)  # shells just outside rc count for the gap too
    rw = np.sqrt((vw * vw).sum(axis=1))
    out["min_edge_gap"] = float(min(np.min(np.abs(rw - e)) for e in edges)) / rc
    return out
