"""Pin: the cell-list oracle equals the O(n^2 * images) brute-force definition.

Tiny random inputs in 2D and 3D, orthorhombic and triclinic boxes, with the
cutoff near half the smallest face distance and near the face distance itself
(several images of one pair inside the cutoff), unwrapped positions far
outside the box. Integer outputs must be identical; floating point agrees to
summation-order rounding.
"""
import numpy as np
import pytest

import oracle

CASES = []
for dim in (2, 3):
    for tric in (False, True):
        for rc_frac in (0.3, 0.49, 0.95):
            CASES.append((dim, tric, rc_frac))


def _box(dim, tric, rng, L=10.0):
    h = np.eye(dim) * L
    if tric:
        for a in range(1, dim):
            for b in range(a):
                h[a, b] = rng.uniform(-0.3 * L, 0.3 * L)
    return h


@pytest.mark.parametrize("dim,tric,rc_frac", CASES)
def test_oracle_equals_brute_force(dim, tric, rc_frac):
    rng = np.random.default_rng(1000 + dim * 10 + int(tric) * 5 + int(rc_frac * 100))
    h = _box(dim, tric, rng)
    w = oracle.geom_info(h, 1.0)["w"]
    rc = rc_frac * w.min()
    n = 120 if dim == 3 else 160
    x = rng.uniform(-25.0, 35.0, size=(n, dim))  # far outside the box: wrapping is exercised
    a = oracle.pair_map(x, h, rc, nbins=17)
    b = oracle.brute_map(x, h, rc, nbins=17)
    assert a["count"] == b["count"] and a["count"] > 0
    assert a["band_in"] == b["band_in"] and a["band_out"] == b["band_out"]
    np.testing.assert_array_equal(a["hist_core"], b["hist_core"])
    np.testing.assert_array_equal(a["hist_maybe"], b["hist_maybe"])
    for k in ("suminvr", "energy"):
        assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-12)
    fs = np.abs(b["forces"]).max()
    np.testing.assert_allclose(a["forces"], b["forces"], rtol=0, atol=1e-11 * fs)
    vs = np.abs(b["virial"]).max()
    np.testing.assert_allclose(a["virial"], b["virial"], rtol=0, atol=1e-11 * vs)
    np.testing.assert_allclose(a["dedh"], b["dedh"], rtol=0, atol=1e-11 * max(np.abs(b["dedh"]).max(), 1.0))
    if rc_frac <= 0.49:
        pa = oracle.pairlist(x, h, rc)
        pb = oracle.brute_pairlist(x, h, rc)
        np.testing.assert_array_equal(pa["i"], pb["i"])
        np.testing.assert_array_equal(pa["j"], pb["j"])
        np.testing.assert_allclose(pa["d"], pb["d"], rtol=1e-13)
        assert np.all(pa["i"] < pa["j"])
        assert int((pa["d"] < rc).sum()) == a["count"]


def test_multi_image_pairs_are_distinct():
    """rc > w/2: a pair seen under two lattice vectors counts twice (both
    pair-images lie inside the cutoff); the pair list refuses such input."""
    h = np.eye(3) * 10.0
    x = np.array([[1.0, 5.0, 5.0], [6.0, 5.0, 5.0]])  # 5 apart, images at 5 and 5
    r = oracle.pair_map(x, h, 5.5)
    assert r["count"] == 2
    assert r["suminvr"] == pytest.approx(2 / 5.0)
    with pytest.raises(oracle.OracleError):
        oracle.pairlist(x, h, 5.5)


def test_cutoff_not_below_face_distance_is_rejected():
    h = np.eye(2) * 4.0
    x = np.zeros((2, 2))
    with pytest.raises(oracle.OracleError):
        oracle.pair_map(x, h, 4.0)


def test_particles_matches_pair_map():
    rng = np.random.default_rng(7)
    h = np.array([[12.0, 0, 0], [2.0, 11.0, 0], [-1.5, 3.0, 10.0]])
    x = rng.uniform(0, 12, size=(200, 3))
    rc = 4.0
    full = oracle.pair_map(x, h, rc)
    idx = np.array([0, 17, 99, 199])
    f, e = oracle.particles(x, h, rc, idx)
    np.testing.assert_allclose(f, full["forces"][idx], rtol=1e-11, atol=1e-12)
    _, e_all = oracle.particles(x, h, rc, np.arange(200))
    assert e_all.sum() == pytest.approx(full["energy"], rel=1e-12)
