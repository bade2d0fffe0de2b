"""Pin: the oracle's band accounting on hand-built pairs.

Sec. 2.3 and 2.8 say "within the cutoff" without fixing the edge; the library
reads it as strict r < rc and decides each pair once in FP32. A pair whose FP64
distance lies within delta = band * rc of the cutoff, or of a histogram bin edge
(bins [k d, (k+1) d), d = rmax / nbins, the left-closed reading of Code 10's
bins), may be decided either way by a correct FP32 path. The oracle therefore
reports, beside the exact results:

  band_in    pairs with rc - delta <= r < rc   (counted, might be missed)
  band_out   pairs with rc <= r < rc + delta   (not counted, might be taken)
  hist_core  per bin, pairs whose bin is the same for every distance in
             [r - delta, r + delta]
  hist_maybe per bin, pairs that may land in it (all bins met by that
             interval that lie below min(rc, rmax)); such a pair is not in core

Each case below places pairs at chosen distances and writes the expected
numbers from those rules by hand, not from the oracle's code. The distances
sit at 0.5 delta and 2 delta from the edges, so FP64 rounding of the
positions (about 1e-14 relative) cannot move a pair across a rule.
"""
import numpy as np
import pytest

import oracle

BAND = 1e-6


def _build(dim, rc, dists, tric=False, seed=0):
    """Positions for pairs at the given distances. The box is a cube (or a
    sheared cube) of side 4 rc * k with one pair per cell of side 4 rc, so
    pairs never reach each other: the nearest foreign particle is at least
    4 rc - 2 * 1.001 rc away, under any image."""
    rng = np.random.default_rng(seed)
    per_axis = int(np.ceil(len(dists) ** (1.0 / dim)))
    side = 4.0 * rc * per_axis
    h = np.eye(dim) * side
    if tric:
        h[1, 0] = 0.23 * side
        if dim == 3:
            h[2, 0] = -0.17 * side
            h[2, 1] = 0.11 * side
    x = []
    for q, r in enumerate(dists):
        idx = np.unravel_index(q, (per_axis,) * dim)
        # cell centre in fractional coordinates, then Cartesian through H
        s = (np.array(idx, dtype=np.float64) + 0.5) / per_axis
        c = s @ h
        u = rng.normal(size=dim)
        u /= np.linalg.norm(u)
        x.append(c - 0.5 * r * u)
        x.append(c + 0.5 * r * u)
    return np.array(x), h


def _check_isolated(x, h, rc):
    """Every pair-image within 1.1 rc is one of the planted pairs (2q, 2q+1)."""
    img = oracle.brute_images(x, h, 1.1 * rc)
    assert np.all(img["i"] % 2 == 0) and np.all(img["j"] == img["i"] + 1)


CUT = [
    # (relative offset from rc, count, band_in, band_out)
    (-2e-6, 1, 0, 0),     # inside, beyond the band
    (-0.5e-6, 1, 1, 0),   # inside, in the band
    (+0.5e-6, 0, 0, 1),   # outside, in the band
    (+2e-6, 0, 0, 0),     # outside, beyond the band (still enumerated: r < rc(1 + 4 band))
    (-0.3, 1, 0, 0),      # well inside
]


@pytest.mark.parametrize("dim,tric", [(2, False), (2, True), (3, False), (3, True)])
@pytest.mark.parametrize("walk", ["cells", "brute"])
def test_cutoff_band_each_pair_alone(dim, tric, walk):
    rc = 3.0
    for off, cnt, bin_, bout in CUT:
        x, h = _build(dim, rc, [rc * (1 + off)], tric=tric, seed=int(1e7 * abs(off)) + dim)
        fn = oracle.pair_map if walk == "cells" else oracle.brute_map
        r = fn(x, h, rc, band=BAND)
        assert (r["count"], r["band_in"], r["band_out"]) == (cnt, bin_, bout), (off, r["count"], r["band_in"],
                                                                                  r["band_out"])


@pytest.mark.parametrize("dim,tric", [(2, True), (3, False), (3, True)])
def test_cutoff_band_many_pairs(dim, tric):
    rc = 2.5
    dists, cnt, bin_, bout = [], 0, 0, 0
    for off, c, bi, bo in CUT:
        for _ in range(3):
            dists.append(rc * (1 + off))
            cnt, bin_, bout = cnt + c, bin_ + bi, bout + bo
    x, h = _build(dim, rc, dists, tric=tric, seed=5)
    _check_isolated(x, h, rc)
    r = oracle.pair_map(x, h, rc, band=BAND)
    assert (r["count"], r["band_in"], r["band_out"]) == (cnt, bin_, bout)
    b = oracle.brute_map(x, h, rc, band=BAND)
    assert (b["count"], b["band_in"], b["band_out"]) == (cnt, bin_, bout)


def _hist_cases(rc, nbins, rmax):
    """(distance, expected core bin or None, expected maybe bins) from the
    rules in the module docstring, with d = rmax / nbins and top = min(rc, rmax)."""
    d = rmax / nbins
    dl = BAND * rc
    last = nbins - 1 if rmax <= rc else int(np.ceil(rc / d)) - 1
    cases = [
        (3.5 * d, 3, []),                         # middle of bin 3
        (5 * d + 0.5 * dl, None, [4, 5]),         # just above the edge between bins 4 and 5
        (5 * d - 0.5 * dl, None, [4, 5]),         # just below it
        (7 * d + 2 * dl, 7, []),                  # clear of the edge: core
        (7 * d - 2 * dl, 6, []),
        (0.25 * d, 0, []),                        # first bin
    ]
    top = min(rc, rmax)
    cases += [
        (top - 0.5 * dl, None, [last]),           # may fall off the top: maybe in the last bin
        (top - 2 * dl, last, []),
    ]
    if rmax >= rc:
        cases += [(top + 0.5 * dl, None, [last]), (top + 2 * dl, None, [])]
    else:
        # rmax < rc: a pair above rmax but below rc is counted, never binned
        cases += [(top + 0.5 * dl, None, [last]), (top + 2 * dl, None, []), (0.5 * (rmax + rc), None, [])]
    return cases


@pytest.mark.parametrize("dim,tric,rmax_frac,nbins", [
    (3, False, 1.0, 10), (3, True, 1.0, 23), (2, True, 1.0, 8), (3, True, 0.5, 10), (2, False, 0.75, 12),
    (3, True, 1.37, 10),   # rmax > rc: the top is rc, inside bin 7; bins 8 and 9 stay empty
])
def test_histogram_band(dim, tric, rmax_frac, nbins):
    rc = 4.0
    rmax = rmax_frac * rc
    cases = _hist_cases(rc, nbins, rmax)
    dists = [c[0] for c in cases]
    x, h = _build(dim, rc, dists, tric=tric, seed=nbins)
    _check_isolated(x, h, rc)
    core = np.zeros(nbins, dtype=np.int64)
    maybe = np.zeros(nbins, dtype=np.int64)
    for _, kc, km in cases:
        if kc is not None:
            core[kc] += 1
        for k in km:
            maybe[k] += 1
    for fn in (oracle.pair_map, oracle.brute_map):
        r = fn(x, h, rc, band=BAND, nbins=nbins, rmax=rmax)
        np.testing.assert_array_equal(r["hist_core"], core)
        np.testing.assert_array_equal(r["hist_maybe"], maybe)
    # every case one by one as well, so a wrong bin cannot hide behind a sum
    for dist, kc, km in cases:
        xs, hs = _build(dim, rc, [dist], tric=tric, seed=3)
        r = oracle.pair_map(xs, hs, rc, band=BAND, nbins=nbins, rmax=rmax)
        ec = np.zeros(nbins, dtype=np.int64)
        em = np.zeros(nbins, dtype=np.int64)
        if kc is not None:
            ec[kc] = 1
        em[km] = 1
        np.testing.assert_array_equal(r["hist_core"], ec, err_msg="r/d = %.9f" % (dist / (rmax / nbins)))
        np.testing.assert_array_equal(r["hist_maybe"], em, err_msg="r/d = %.9f" % (dist / (rmax / nbins)))


def test_pairlist_band_flags():
    """The pair list keeps pairs up to rc(1 + 4 band) and flags |r - rc| <= band rc."""
    rc = 3.0
    offs = [-2e-6, -0.5e-6, 0.5e-6, 2e-6, -0.3, 5e-6]
    x, h = _build(3, rc, [rc * (1 + o) for o in offs], tric=True, seed=11)
    _check_isolated(x, h, rc)
    for fn in (oracle.pairlist, oracle.brute_pairlist):
        pl = fn(x, h, rc, band=BAND)
        kept = [2 * q for q, o in enumerate(offs) if o < 4e-6]
        np.testing.assert_array_equal(pl["i"], kept)
        np.testing.assert_array_equal(pl["j"], np.array(kept) + 1)
        flags = [abs(o) <= 1e-6 for o in offs if o < 4e-6]
        np.testing.assert_array_equal(pl["band"], flags)
        np.testing.assert_allclose(pl["d"], [rc * (1 + o) for o in offs if o < 4e-6], rtol=1e-12)


def test_histogram_band_spans_several_bins():
    """Bins narrower than the band: a pair may land in every bin its interval
    [r - delta, r + delta] meets, up to the last bin below the top."""
    rc, nbins = 2.0, 2_000_000           # d = rc / nbins = 0.5 delta
    d = rc / nbins
    dl = BAND * rc
    x, h = _build(3, rc, [rc - 0.25 * dl, 1000.5 * d], seed=2)
    r = oracle.pair_map(x, h, rc, band=BAND, nbins=nbins)
    assert r["hist_core"].sum() == 0
    # first pair: [rc - 1.25 delta, rc + 0.75 delta] meets bins nbins-3 .. nbins-1 (top cuts it)
    # second pair: [1000.5 d - 2 d, 1000.5 d + 2 d] meets bins 998 .. 1002
    want = np.zeros(nbins, dtype=np.int64)
    want[nbins - 3:] = 1
    want[998:1003] = 1
    np.testing.assert_array_equal(np.nonzero(r["hist_maybe"])[0], np.nonzero(want)[0])
    np.testing.assert_array_equal(r["hist_maybe"], want)
