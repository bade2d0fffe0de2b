"""Seeded synthetic particle sets for the cell-list pair map.

This module only draws inputs. It holds none of the arithmetic of the method
(no cell lists, no pair sums); both the CUDA path's tests and the FP64 oracle
read the same arrays from it. Every generator returns positions ``x`` as an
(n, dim) float64 array and the lattice matrix ``h`` (dim, dim) whose ROWS are
the lattice vectors, plus the cutoff of the workload.

The paper's own test systems (``xatomic``, ``xgalactic``, Sec. 3) are not
available; these stand-ins keep its density-to-cutoff ratios: about 724
neighbours per particle in the 3D molecular-like sets, as in water-density
atoms with rc = 1.2 nm (Sec. 4.1).

Workloads (seed = 2202064270 + workload number):
  w0_small          3D, 10,000 particles, cubic box 46.416, rc 12, sum 1/r + count
  w1_lattice_1m     3D, 100^3 jittered lattice, cubic box 215.44, rc 12
  w2_triclinic_1m   3D triclinic box rows (220,0,0),(30,215,0),(20,25,210), rc 10
  w3 serve stream   512 requests (see ``serve_stream``)
  w4_clustered_16m  3D, 16M, 2,000 Gaussian clusters + 20% background, rc 8
"""
import math

import numpy as np

SEED0 = 2202064270
DENSITY_3D = 0.1
SPACING_3D = (1.0 / DENSITY_3D) ** (1.0 / 3.0)  # 2.15443469...


def jittered_cubic(n_side, box_side, n_keep, jitter_abs, seed, dim=3):
    """Simple cubic (square) lattice of n_side^dim sites at spacing box_side/n_side;
    keep n_keep sites chosen by a seeded shuffle; add U(-jitter_abs, +jitter_abs)
    to every coordinate. Positions are NOT wrapped (wrapping is the method's job)."""
    rng = np.random.default_rng(seed)
    nsites = n_side ** dim
    if n_keep > nsites:
        raise ValueError("n_keep > sites")
    keep = np.sort(rng.permutation(nsites)[:n_keep]) if n_keep < nsites else np.arange(nsites)
    idx = np.stack(np.unravel_index(keep, (n_side,) * dim, order="F"), axis=1).astype(np.float64)
    a = box_side / n_side
    x = (idx + 0.5) * a + rng.uniform(-jitter_abs, jitter_abs, size=idx.shape)
    h = np.eye(dim) * box_side
    return np.ascontiguousarray(x), h


def jittered_fractional(h, n_side, n_keep, jitter_frac, seed):
    """Lattice in fractional coordinates: s = (site + 0.5 + U(+-jitter_frac)) / n_side
    per axis, for n_keep of the n_side^dim sites (seeded shuffle), x = s.H."""
    h = np.asarray(h, dtype=np.float64)
    dim = h.shape[0]
    rng = np.random.default_rng(seed)
    nsites = n_side ** dim
    keep = np.sort(rng.permutation(nsites)[:n_keep]) if n_keep < nsites else np.arange(nsites)
    idx = np.stack(np.unravel_index(keep, (n_side,) * dim, order="F"), axis=1).astype(np.float64)
    s = (idx + 0.5 + rng.uniform(-jitter_frac, jitter_frac, size=idx.shape)) / n_side
    return np.ascontiguousarray(s @ h)


def w0_small():
    """3D, N = 10,000 at density 0.1: box side (1e5)^(1/3) = 46.416; 10,000 is
    not a cube, so 10,000 of the 22^3 sites of a lattice at spacing L/22 are kept
    (seeded), each coordinate jittered by U(+-0.4 * 2.1544). rc = 12."""
    L = (10_000 / DENSITY_3D) ** (1.0 / 3.0)
    x, h = jittered_cubic(22, L, 10_000, 0.4 * SPACING_3D, SEED0 + 0)
    return {"name": "w0_small_10k", "x": x, "h": h, "rc": 12.0}


def w1_lattice(n_side=100, seed=SEED0 + 1):
    """3D jittered simple cubic lattice at density 0.1: n_side^3 sites at spacing
    2.15443 (box side 215.44 for n_side = 100), jitter U(+-0.4 a). rc = 12."""
    L = n_side * SPACING_3D
    x, h = jittered_cubic(n_side, L, n_side ** 3, 0.4 * SPACING_3D, seed)
    return {"name": "w1_lattice_%d" % n_side ** 3, "x": x, "h": h, "rc": 12.0}


W2_H = np.array([[220.0, 0.0, 0.0], [30.0, 215.0, 0.0], [20.0, 25.0, 210.0]])


def w2_triclinic(n_side=100, seed=SEED0 + 2, h=None):
    """3D triclinic box, rows (220,0,0), (30,215,0), (20,25,210) (volume 9.933e6,
    density 0.1007 at n_side = 100); particles on a 100^3 lattice in fractional
    coordinates jittered by U(+-0.4) of a lattice step. rc = 10; the workload asks
    for the sorted i<j list and a 200-bin histogram on [0, rc)."""
    h = W2_H if h is None else np.asarray(h, dtype=np.float64)
    x = jittered_fractional(h, n_side, n_side ** 3, 0.4, seed)
    return {"name": "w2_triclinic_%d" % n_side ** 3, "x": x, "h": h.copy(), "rc": 10.0, "nbins": 200}


def serve_stream(n_requests=512, seed=SEED0 + 3, mean_gap_s=2e-3, n_min=1_000, n_max=200_000):
    """Request stream: Poisson arrivals (exponential gaps, mean 2 ms); each request
    is 2D (square box, density 0.7, rc 2.5) or 3D (density 0.1, rc 12) with equal
    odds; N log-uniform in [n_min, n_max]; orthorhombic or triclinic (lower
    triangular rows, off-diagonals U(+-0.25 L), diagonal L, volume unchanged) with
    equal odds; task energy, forces or a 100-bin histogram on [0, rc) with equal
    odds. Positions are drawn lazily by ``request_positions``."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(mean_gap_s, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for k in range(n_requests):
        dim = 2 if rng.random() < 0.5 else 3
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        tric = rng.random() < 0.5
        task = ("energy", "forces", "hist")[int(rng.integers(0, 3))]
        dens, rc = (0.7, 2.5) if dim == 2 else (DENSITY_3D, 12.0)
        L = (n / dens) ** (1.0 / dim)
        h = np.eye(dim) * L
        if tric:
            for a in range(1, dim):
                for b in range(a):
                    h[a, b] = rng.uniform(-0.25 * L, 0.25 * L)
        reqs.append({"id": k, "arrival_s": float(t[k]), "dim": dim, "n": n, "h": h, "rc": rc,
                     "task": task, "nbins": 100, "seed": int(seed * 1000 + k)})
    return reqs


def request_positions(req):
    """Jittered lattice in fractional coordinates, n_side = ceil(N^(1/dim))."""
    dim, n = req["dim"], req["n"]
    n_side = int(math.ceil(n ** (1.0 / dim) - 1e-9))
    while n_side ** dim < n:
        n_side += 1
    return jittered_fractional(req["h"], n_side, n, 0.4, req["seed"])


def w4_clustered(n=16_000_000, L=600.0, n_clusters=2000, sigma=8.0, frac_clustered=0.8,
                 size_range=(2800.0, 20000.0), min_sep=0.5, seed=SEED0 + 4):
    """3D clustered set (see synth.clustered): Gaussian clusters with truncated
    power-law sizes p(s) ~ s^-2 on ``size_range`` rescaled to sum to 80% of n,
    20% uniform background, minimum separation by rejection. rc = 8."""
    from . import clustered
    x, stats = clustered.generate(n, L, n_clusters, sigma, frac_clustered, size_range, min_sep, seed)
    return {"name": "w4_clustered_%d" % n, "x": x, "h": np.eye(3) * L, "rc": 8.0, "stats": stats}
