"""Pin: the oracle's open-system (non-periodic) sums of Sec. 4.1 against a
direct double loop over the points, with no box and no images at all."""
import numpy as np
import pytest

import oracle


def _direct(x, rc):
    n = x.shape[0]
    count, e, f = 0, 0.0, np.zeros_like(x)
    pairs = []
    for i in range(n):
        for j in range(i + 1, n):
            rv = x[j] - x[i]
            r = float(np.sqrt(rv @ rv))
            if r < rc:
                count += 1
                e += 1 / r - 1 / rc + (r - rc) / rc ** 2
                g = (-1 / r ** 2 + 1 / rc ** 2) * rv / r
                f[i] += g
                f[j] -= g
                pairs.append((i, j, r))
    return count, e, f, pairs


@pytest.mark.parametrize("dim", [2, 3])
def test_open_pair_map_equals_direct_loop(dim):
    rng = np.random.default_rng(17 + dim)
    # two blobs far apart plus a far outlier: the extent is large, pairs are local
    x = np.vstack([rng.normal(size=(120, dim)) * 1.5 + 40.0, rng.normal(size=(100, dim)) * 1.5 - 35.0,
                   np.full((1, dim), 400.0)])
    rc = 1.3
    count, e, f, pairs = _direct(x, rc)
    r = oracle.open_pair_map(x, rc)
    assert r["count"] == count and count > 100
    assert r["energy"] == pytest.approx(e, rel=1e-12)
    np.testing.assert_allclose(r["forces"], f, rtol=0, atol=1e-11 * np.abs(f).max())
    pl = oracle.open_pairlist(x, rc)
    np.testing.assert_array_equal(np.stack([pl["i"], pl["j"]], 1), np.array([(i, j) for i, j, _ in pairs]))
    # positions are wrapped into a box of side ~800: absolute rounding of order 1e-13
    np.testing.assert_allclose(pl["d"], [d for _, _, d in pairs], rtol=0, atol=1e-11)


def test_open_cross_images_equal_direct_loop():
    rng = np.random.default_rng(5)
    xa = rng.normal(size=(150, 3)) * 2.0
    yb = rng.normal(size=(90, 3)) * 2.0 + 1.0
    rc = 1.1
    img = oracle.open_cross_images(xa, yb, rc)
    got = sorted(zip(img["i"].tolist(), img["j"].tolist()))
    want = sorted((a, b) for a in range(150) for b in range(90) if np.linalg.norm(yb[b] - xa[a]) < rc * (1 + 4e-6))
    assert got == want and len(want) > 50
    for a, b, rv in zip(img["i"], img["j"], img["rv"]):
        np.testing.assert_allclose(rv, yb[b] - xa[a], atol=1e-12)
