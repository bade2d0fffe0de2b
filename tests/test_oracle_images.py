"""Pins of the oracle's pair-image enumeration (the input of the mapped
function, Code 2), its cross-set form (Code 8) and the pair functions built on
it (Code 5, 6, 7, 8, 10): brute force on tiny inputs, the already pinned
reductions of pair_map, set identities, closed forms and finite differences."""
import numpy as np
import pytest

import oracle


def _box(dim, tric, L, rng):
    h = np.eye(dim) * L
    if tric:
        for a in range(1, dim):
            for b in range(a):
                h[a, b] = rng.uniform(-0.3 * L, 0.3 * L)
    return h


def _key(img, digits=9):
    """Multiset of (i, j, rounded displacement) of an image set."""
    return sorted(zip(img["i"].tolist(), img["j"].tolist(), *[np.round(c, digits).tolist() for c in img["rv"].T]))


@pytest.mark.parametrize("dim,tric,rc_frac", [(3, False, 0.3), (3, True, 0.45), (2, True, 0.8), (3, True, 0.9)])
def test_images_match_brute_force(dim, tric, rc_frac):
    rng = np.random.default_rng(11 + dim + 10 * tric)
    L = 6.0
    h = _box(dim, tric, L, rng)
    w = oracle.geom_info(h, 1.0)["w"]
    rc = rc_frac * w.min()  # rc_frac > 0.5: pairs with two images inside the cutoff
    x = rng.uniform(-2 * L, 2 * L, size=(60, dim))
    a, b = oracle.images(x, h, rc), oracle.brute_images(x, h, rc)
    assert len(a["r"]) == len(b["r"]) > 0
    assert _key(a) == _key(b)


@pytest.mark.parametrize("dim,tric", [(3, True), (2, False)])
def test_images_reproduce_the_pinned_reductions(dim, tric):
    """Count, sum 1/r, shifted-force energy, forces and virial recomputed from
    the images equal pair_map's (pinned by brute force, closed forms and finite
    differences elsewhere): the displacement vectors carry the right sign and
    image."""
    rng = np.random.default_rng(21 + dim)
    h = _box(dim, tric, 9.0, rng)
    rc = 0.4 * oracle.geom_info(h, 1.0)["w"].min()
    x = rng.uniform(0, 9.0, size=(300, dim)) @ (h / 9.0)
    ref = oracle.pair_map(x, h, rc)
    img = oracle.images(x, h, rc)
    sel = img["r"] < rc
    r, rv, i, j = img["r"][sel], img["rv"][sel], img["i"][sel], img["j"][sel]
    assert len(r) == ref["count"]
    assert np.isclose(np.sum(1.0 / r), ref["suminvr"], rtol=1e-12)
    u = 1.0 / r - 1.0 / rc + (r - rc) / rc ** 2
    assert np.isclose(np.sum(u), ref["energy"], rtol=1e-12)
    dudr = -1.0 / r ** 2 + 1.0 / rc ** 2
    g = (dudr / r)[:, None] * rv
    f = np.zeros_like(x)
    np.add.at(f, i, g)
    np.add.at(f, j, -g)
    assert np.allclose(f, ref["forces"], rtol=1e-10, atol=1e-12 * np.abs(f).max())
    vir = -(rv * (dudr / r)[:, None]).T @ rv
    assert np.allclose(vir, ref["virial"], rtol=1e-10, atol=1e-12 * np.abs(vir).max())


@pytest.mark.parametrize("dim,tric", [(3, True), (2, True), (3, False)])
def test_cross_images_match_brute_force(dim, tric):
    rng = np.random.default_rng(31 + dim)
    h = _box(dim, tric, 7.0, rng)
    rc = 0.7 * oracle.geom_info(h, 1.0)["w"].min()
    xa = rng.uniform(-7, 14, size=(40, dim))
    yb = rng.uniform(-7, 14, size=(55, dim))
    a, b = oracle.cross_images(xa, yb, h, rc), oracle.brute_cross_images(xa, yb, h, rc)
    assert len(a["r"]) == len(b["r"]) > 0
    assert _key(a) == _key(b)


def test_cross_images_complete_the_union():
    """Pair-images of A u B = those within A + those within B + the cross ones
    (with indices of B shifted by |A|); the cross enumeration is independent of
    the within-set one."""
    rng = np.random.default_rng(41)
    h = _box(3, True, 10.0, rng)
    rc = 0.45 * oracle.geom_info(h, 1.0)["w"].min()
    xa = rng.uniform(0, 10, size=(150, 3))
    yb = rng.uniform(0, 10, size=(170, 3))
    na = xa.shape[0]
    u = oracle.images(np.vstack([xa, yb]), h, rc)
    ia, ib, c = oracle.images(xa, h, rc), oracle.images(yb, h, rc), oracle.cross_images(xa, yb, h, rc)
    parts = list(zip(ia["i"], ia["j"], np.round(ia["r"], 9))) + \
        list(zip(ib["i"] + na, ib["j"] + na, np.round(ib["r"], 9))) + \
        list(zip(c["i"], c["j"] + na, np.round(c["r"], 9)))
    whole = list(zip(u["i"], u["j"], np.round(u["r"], 9)))
    assert sorted(parts) == sorted(whole)


def test_lj_two_particles_closed_form():
    """Two particles at distance d along x in a large box: E = 4 eps (s^12/d^12
    - s^6/d^6), F_0 = u'(d) x_hat = -F_1 (pointing away from the other particle
    when the pair repels), W_xx = -u'(d) d."""
    eps, sigma, d = 0.3, 1.1, 1.05
    h = np.eye(3) * 20.0
    x = np.array([[5.0, 5.0, 5.0], [5.0 + d, 5.0, 5.0]])
    out = oracle.lj(x, h, 3.0, eps, sigma)
    s6 = (sigma / d) ** 6
    assert np.isclose(out["energy"], 4 * eps * (s6 * s6 - s6), rtol=1e-14)
    dudd = 4 * eps * (-12 * s6 * s6 + 6 * s6) / d
    assert np.allclose(out["forces"][0], [dudd, 0, 0], rtol=1e-13)
    assert np.allclose(out["forces"][1], [-dudd, 0, 0], rtol=1e-13)
    assert out["forces"][0][0] < 0  # d < 2^(1/6) sigma: repulsive, pushes particle 0 to -x
    assert np.isclose(out["virial"][0, 0], -dudd * d, rtol=1e-13)


def test_lj_forces_are_minus_the_energy_gradient():
    rng = np.random.default_rng(51)
    h = _box(3, True, 8.0, rng)
    rc = 2.5
    x = rng.uniform(0, 8, size=(60, 3))
    eps, sigma = 0.2, 0.8
    f = oracle.lj(x, h, rc, eps, sigma)["forces"]
    step = 1e-6
    for p in (0, 7, 33):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[p, a] += step
            xm[p, a] -= step
            fd = -(oracle.lj(xp, h, rc, eps, sigma)["energy"] - oracle.lj(xm, h, rc, eps, sigma)["energy"]) / (2 * step)
            # the energy jumps when a pair crosses rc; with these positions none is within 2 steps of it
            assert np.isclose(fd, f[p, a], rtol=1e-5, atol=1e-7 * np.abs(f).max())


def test_mass_potential_with_unit_masses_is_sum_inv_r():
    rng = np.random.default_rng(61)
    h = _box(3, True, 9.0, rng)
    rc = 3.0
    x = rng.uniform(0, 9, size=(200, 3))
    ref = oracle.pair_map(x, h, rc)
    assert np.isclose(oracle.mass_potential(x, h, rc, np.ones(200))["value"], ref["suminvr"], rtol=1e-12)
    m = rng.uniform(0.5, 2.0, size=200)
    # scaling every mass by c scales the sum by c^2
    assert np.isclose(oracle.mass_potential(x, h, rc, 3 * m)["value"],
                      9 * oracle.mass_potential(x, h, rc, m)["value"], rtol=1e-12)


def test_velocity_hist_counts_and_alternating_velocities():
    """Counts: the distance histogram of the pairs (bins of width binstep on
    [0, nbins binstep), right-closed); with velocities +u on one set and -u on
    another, |v_i - v_j| is 2|u| for cross pairs and 0 otherwise, so the
    velocity sums are 2|u| times the cross pairs' counts (cross_images)."""
    rng = np.random.default_rng(71)
    h = np.eye(3) * 12.0
    rc, binstep, nbins = 3.0, 0.5, 5   # bins up to 2.5: pairs in (2.5, 3) are not binned
    xa = rng.uniform(0, 12, size=(150, 3))
    yb = rng.uniform(0, 12, size=(160, 3))
    x = np.vstack([xa, yb])
    u = np.array([0.3, -0.4, 1.2])
    v = np.vstack([np.tile(u, (150, 1)), np.tile(-u, (160, 1))])
    out = oracle.velocity_hist(x, h, rc, v, binstep, nbins)
    assert np.sum(out["band_counts"]) == 0  # random positions: no pair near an edge
    img = oracle.images(x, h, rc)
    r = img["r"][img["r"] < rc]
    want = np.histogram(r, bins=np.arange(nbins + 1) * binstep)[0]
    assert np.array_equal(out["counts"], want)
    c = oracle.cross_images(xa, yb, h, rc)
    rcx = c["r"][c["r"] < rc]
    cross = np.histogram(rcx, bins=np.arange(nbins + 1) * binstep)[0]
    assert np.allclose(out["vsum"], 2 * np.linalg.norm(u) * cross, rtol=1e-12)


def test_knn_pairs():
    rng = np.random.default_rng(81)
    h = _box(3, True, 6.0, rng)
    rc = 1.5
    xa = rng.uniform(0, 6, size=(30, 3))
    yb = rng.uniform(0, 6, size=(40, 3))
    allp = oracle.brute_cross_images(xa, yb, h, rc)
    d = np.sort(allp["r"][allp["r"] < rc])
    for k in (1, 5, len(d) + 3):
        out = oracle.knn_pairs(xa, yb, h, rc, k)
        assert np.allclose(out["r"], d[:k])
        assert np.all(np.diff(out["r"]) >= 0)
