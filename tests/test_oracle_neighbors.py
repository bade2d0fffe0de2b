"""Pin: the oracle's per-row neighbour lists (Sec. 4.1 list, chosen rows).

``oracle.neighbors`` is the checker for sampled rows of the large GPU pair
lists, so it is pinned against the two whole-list definitions: the cell-list
``oracle.pairlist`` and the brute-force ``oracle.brute_pairlist`` (all i < j
and all integer image vectors). For every row a, the entries j > a, their
distances and band flags must equal the pairs (a, j) of the whole list.

The boxes are small and triclinic, with the cutoff up to half the smallest
face distance, so that the grid has n_k < 2 m_k + 1 (one neighbour cell is met
under two lattice images, and only one of them can hold the pair), and some
pairs are planted within 4 band rc above the cutoff (kept in the lists, with
the band flag only within band rc): a row filter on rc instead of rc(1 + 4
band), or a lost image, fails here.
"""
import ctypes

import numpy as np
import pytest

import oracle

BAND = 1e-6


def _box(dim, rng, L=10.0):
    h = np.eye(dim) * L
    for a in range(1, dim):
        for b in range(a):
            h[a, b] = rng.uniform(-0.35 * L, 0.35 * L)
    return h


def _plant_edge_pairs(x, h, rc, rng, offs):
    """Append pairs at distances rc(1 + o), each next to a random particle's
    position shifted by a random lattice vector (so it arrives unwrapped)."""
    dim = h.shape[0]
    extra = []
    for o in offs:
        base = rng.uniform(0, 1, size=dim) @ h
        u = rng.normal(size=dim)
        u /= np.linalg.norm(u)
        t = rng.integers(-2, 3, size=dim) @ h
        extra.append(base)
        extra.append(base + rc * (1 + o) * u + t)
    return np.vstack([x, np.array(extra)])


def _rows_from_list(pl, n):
    rows = [[] for _ in range(n)]
    for i, j, d, b in zip(pl["i"], pl["j"], pl["d"], pl["band"]):
        rows[int(i)].append((int(j), float(d), bool(b)))
    return rows


CASES = [(3, 0.3), (3, 0.45), (3, 0.4999), (2, 0.35), (2, 0.4999)]


@pytest.mark.parametrize("dim,rc_frac", CASES)
def test_neighbor_rows_equal_whole_lists(dim, rc_frac):
    rng = np.random.default_rng(int(rc_frac * 1e4) + dim)
    h = _box(dim, rng)
    w = oracle.geom_info(h, 1.0)["w"]
    rc = rc_frac * w.min()
    g = oracle.geom_info(h, rc * (1 + 4 * BAND))
    n0 = 90 if dim == 3 else 110
    x = rng.uniform(-20.0, 30.0, size=(n0, dim))
    x = _plant_edge_pairs(x, h, rc, rng, [0.5e-6, 2e-6, 3.5e-6, -0.5e-6, -2e-6])
    n = x.shape[0]
    if rc_frac > 0.4:
        # the case this pins: a neighbour cell reached under several images
        assert np.any(g["n"] < 2 * g["m"] + 1), g
    brute = oracle.brute_pairlist(x, h, rc, band=BAND)
    cells = oracle.pairlist(x, h, rc, band=BAND)
    np.testing.assert_array_equal(cells["i"], brute["i"])
    np.testing.assert_array_equal(cells["j"], brute["j"])
    # the planted pairs above the cutoff are in the lists, flagged only within the band
    d_rel = brute["d"] / rc - 1
    assert np.any((d_rel > 1e-6) & (d_rel < 4e-6)), "no pair planted in (rc(1+band), rc(1+4 band))"
    assert np.all(brute["band"] == (np.abs(brute["d"] - rc) <= BAND * rc))
    want = _rows_from_list(brute, n)
    # every row, in a shuffled order with repeats
    idx = np.concatenate([rng.permutation(n), rng.integers(0, n, size=7)])
    rows = oracle.neighbors(x, h, rc, idx, band=BAND)
    for a, row in zip(idx, rows):
        exp = want[int(a)]
        np.testing.assert_array_equal(row["j"], [e[0] for e in exp], err_msg="row %d" % a)
        np.testing.assert_allclose(row["d"], [e[1] for e in exp], rtol=1e-13, err_msg="row %d" % a)
        np.testing.assert_array_equal(row["band"], [e[2] for e in exp], err_msg="row %d" % a)


def test_neighbor_rows_report_capacity():
    """Too small a buffer: OR_ERR_CAPACITY (-4) with the total in offs[k]."""
    rng = np.random.default_rng(3)
    h = _box(3, rng)
    rc = 0.45 * oracle.geom_info(h, 1.0)["w"].min()
    x = rng.uniform(0, 10, size=(120, 3))
    total = len(oracle.brute_pairlist(x, h, rc, band=BAND)["i"])
    idx = np.arange(120, dtype=np.int64)
    k, cap = idx.shape[0], 5
    offs = np.zeros(k + 1, dtype=np.int64)
    oj = np.zeros(cap, dtype=np.int64)
    od = np.zeros(cap)
    ob = np.zeros(cap, dtype=np.int8)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    ret = oracle._lib().or_neighbors(3, 120, p(x), p(h), rc, BAND, p(idx), k, cap, p(offs), p(oj), p(od), p(ob))
    assert ret == -4
    assert offs[k] == total and total > cap


def test_pair_just_beyond_cutoff_across_two_cells():
    """A grid built for rc instead of rc(1 + 4 band) would miss this pair.

    Cubic box of side L with rc = L/3 (1 - 1e-6): cells built for rc would be
    L/3 wide with reach one cell, yet a pair at r = rc(1 + 3e-6) > L/3 along x,
    starting at the end of cell 0, ends in cell 2. It lies within
    rc(1 + 4 band), so the lists keep it (unflagged: r - rc > band rc)."""
    L = 30.0
    h = np.eye(3) * L
    rc = L / 3 * (1 - 1e-6)
    r = rc * (1 + 3e-6)
    xi = np.array([L / 3 - 1e-7 * L, 4.0, 7.0])
    x = np.array([xi, xi + [r, 0.0, 0.0], [15.0, 20.0, 25.0]])
    for fn in (oracle.brute_pairlist, oracle.pairlist):
        pl = fn(x, h, rc, band=BAND)
        np.testing.assert_array_equal(pl["i"], [0])
        np.testing.assert_array_equal(pl["j"], [1])
        assert not pl["band"][0]
    row = oracle.neighbors(x, h, rc, np.array([0, 1, 2]), band=BAND)
    np.testing.assert_array_equal(row[0]["j"], [1])
    assert row[0]["d"][0] == pytest.approx(r, rel=1e-12)
    assert len(row[1]["j"]) == 0 and len(row[2]["j"]) == 0
