"""Pin: invariances that any correct pair map obeys.

Translating every particle, moving single particles by lattice vectors
(positions need not be wrapped, Sec. 2.6 ghosts make the map agnostic to the
periodic boundary), and relabelling the particles leave every reduction
unchanged (forces permute with the labels). Results do not depend on how the
work is split (Sec. 2.8 parallel batches are summed): restricting the smaller
index to disjoint ranges and adding the parts gives the whole.
"""
import numpy as np
import pytest

import oracle


def _sys(dim, seed, n=250):
    rng = np.random.default_rng(seed)
    if dim == 3:
        h = np.array([[13.0, 0.0, 0.0], [3.0, 12.0, 0.0], [-2.0, 2.5, 12.5]])
    else:
        h = np.array([[13.0, 0.0], [4.0, 12.0]])
    x = rng.uniform(0, 13, size=(n, dim))
    rc = 0.45 * oracle.geom_info(h, 1.0)["w"].min()
    return x, h, rc, rng


@pytest.mark.parametrize("dim", [2, 3])
def test_translation_and_lattice_shifts(dim):
    x, h, rc, rng = _sys(dim, 5 + dim)
    base = oracle.pair_map(x, h, rc, nbins=25)
    x2 = x + rng.uniform(-40, 40, size=(1, dim))
    k = rng.integers(-3, 4, size=(x.shape[0], dim)).astype(np.float64)
    x3 = x + k @ h
    for xx in (x2, x3):
        r = oracle.pair_map(xx, h, rc, nbins=25)
        assert r["count"] == base["count"]
        # pairs near a bin edge may move between bins; compare the certain part
        assert np.all(np.abs(r["hist_core"] - base["hist_core"]) <= base["hist_maybe"] + r["hist_maybe"])
        assert r["energy"] == pytest.approx(base["energy"], rel=1e-11)
        assert r["suminvr"] == pytest.approx(base["suminvr"], rel=1e-11)
        np.testing.assert_allclose(r["forces"], base["forces"], rtol=0, atol=1e-9 * np.abs(base["forces"]).max())
        np.testing.assert_allclose(r["virial"], base["virial"], rtol=0, atol=1e-9 * np.abs(base["virial"]).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_permutation(dim):
    x, h, rc, rng = _sys(dim, 21 + dim)
    base = oracle.pair_map(x, h, rc)
    perm = rng.permutation(x.shape[0])
    r = oracle.pair_map(x[perm], h, rc)
    assert r["count"] == base["count"]
    assert r["energy"] == pytest.approx(base["energy"], rel=1e-12)
    np.testing.assert_allclose(r["forces"], base["forces"][perm], atol=1e-10)
    pa, pb = oracle.pairlist(x, h, rc), oracle.pairlist(x[perm], h, rc)
    inv = np.argsort(perm)
    mapped = sorted((min(inv[i], inv[j]), max(inv[i], inv[j])) for i, j in zip(pa["i"], pa["j"]))
    assert mapped == sorted(zip(pb["i"].tolist(), pb["j"].tolist()))


def test_split_by_index_range_sums_to_whole():
    x, h, rc, _ = _sys(3, 40, n=300)
    whole = oracle.pair_map(x, h, rc, nbins=10)
    parts = [oracle.pair_map(x, h, rc, nbins=10, i_range=(a, b)) for a, b in ((0, 77), (77, 200), (200, 300))]
    assert sum(p["count"] for p in parts) == whole["count"]
    np.testing.assert_array_equal(sum(p["hist_core"] for p in parts), whole["hist_core"])
    assert sum(p["energy"] for p in parts) == pytest.approx(whole["energy"], rel=1e-12)
    np.testing.assert_allclose(sum(p["forces"] for p in parts), whole["forces"], atol=1e-10)


def test_widths_match_linear_algebra():
    """Face distances w_k = V / |cross product of the other two rows|."""
    h = np.array([[220.0, 0, 0], [30.0, 215.0, 0], [20.0, 25.0, 210.0]])
    w = oracle.geom_info(h, 10.0)["w"]
    V = abs(np.linalg.det(h))
    expect = [V / np.linalg.norm(np.cross(h[1], h[2])), V / np.linalg.norm(np.cross(h[2], h[0])),
              V / np.linalg.norm(np.cross(h[0], h[1]))]
    np.testing.assert_allclose(w, expect, rtol=1e-13)
