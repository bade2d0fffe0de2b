"""Pin: the oracle's forces, virial and box gradient are derivatives of its
energy (central finite differences, h = 1e-6).

The shifted-force energy u(r) = 1/r - 1/rc + (r - rc)/rc^2 is C1 at the
cutoff (u(rc) = u'(rc) = 0), so finite differences are valid even when a pair
crosses rc. Code 9 (Sec. 3.3) differentiates a pair sum by automatic
differentiation; the derivatives pinned here are the adjoints the library's
backward kernel returns:
  forces F = -dE/dx,
  dE/dH at fixed Cartesian positions,
  dE/dH at fixed fractional coordinates = -H^-T W (W the virial).
"""
import numpy as np
import pytest

import oracle


def _sys(dim, seed):
    rng = np.random.default_rng(seed)
    if dim == 3:
        h = np.array([[9.0, 0.0, 0.0], [1.5, 8.5, 0.0], [-1.0, 2.0, 9.5]])
        n = 90
    else:
        h = np.array([[9.0, 0.0], [2.0, 8.0]])
        n = 70
    x = rng.uniform(-3, 12, size=(n, dim))
    rc = 0.9 * oracle.geom_info(h, 1.0)["w"].min()  # several images per pair
    return x, h, rc


@pytest.mark.parametrize("dim", [2, 3])
def test_forces_are_minus_energy_gradient(dim):
    x, h, rc = _sys(dim, 3 + dim)
    r = oracle.pair_map(x, h, rc)
    eps = 1e-6
    for i in (0, 5, x.shape[0] - 1):
        for a in range(dim):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += eps
            xm[i, a] -= eps
            fd = -(oracle.energy(xp, h, rc) - oracle.energy(xm, h, rc)) / (2 * eps)
            assert r["forces"][i, a] == pytest.approx(fd, rel=1e-5, abs=1e-6)


@pytest.mark.parametrize("dim", [2, 3])
def test_box_gradient_at_fixed_positions(dim):
    x, h, rc = _sys(dim, 13 + dim)
    r = oracle.pair_map(x, h, rc)
    eps = 1e-6
    for a in range(dim):
        for b in range(dim):
            hp, hm = h.copy(), h.copy()
            hp[a, b] += eps
            hm[a, b] -= eps
            fd = (oracle.energy(x, hp, rc) - oracle.energy(x, hm, rc)) / (2 * eps)
            assert r["dedh"][a, b] == pytest.approx(fd, rel=1e-5, abs=1e-6)


@pytest.mark.parametrize("dim", [2, 3])
def test_virial_is_strain_derivative(dim):
    """Scaling positions with the box (fractional coordinates fixed) changes E
    by -H^-T W per unit change of H."""
    x, h, rc = _sys(dim, 23 + dim)
    r = oracle.pair_map(x, h, rc)
    s = x @ np.linalg.inv(h)
    eps = 1e-6
    want = -np.linalg.inv(h).T @ r["virial"]
    for a in range(dim):
        for b in range(dim):
            hp, hm = h.copy(), h.copy()
            hp[a, b] += eps
            hm[a, b] -= eps
            fd = (oracle.energy(s @ hp, hp, rc) - oracle.energy(s @ hm, hm, rc)) / (2 * eps)
            assert want[a, b] == pytest.approx(fd, rel=1e-5, abs=1e-6)
