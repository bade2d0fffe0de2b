"""Pin: the oracle on perfect lattices equals closed-form lattice sums.

Every site of a perfect periodic lattice sees the same full shells of lattice
vectors (Sec. 2.6: ghost copies give each real particle its full set of
neighbours), so count, sum 1/r, energy, virial and histogram are N/2 times a
sum over integer vectors, and every force vanishes. The closed form
enumerates integer vectors and never builds a cell list.

The 1M-particle workload geometry (spacing 2.15443, rc = 12) gives 738
neighbours per site, hence 369,000,000 pairs for the unjittered 100^3 lattice.
"""
import numpy as np
import pytest

import oracle
from oracle import closed_form as cf

A3 = 10.0 ** (1.0 / 3.0)  # spacing at density 0.1


def _lattice_positions(b, reps):
    dim = b.shape[0]
    grid = np.stack(np.meshgrid(*[np.arange(r) for r in reps], indexing="ij"), axis=-1).reshape(-1, dim)
    return grid.astype(np.float64) @ b, np.diag(reps).astype(np.float64) @ b


def test_workload_lattice_neighbour_count():
    v = cf.lattice_vectors(np.eye(3) * A3, 12.0)
    assert len(v) == 738
    assert cf.lattice_sums(np.eye(3) * A3, 12.0, 100 ** 3)["count"] == 369_000_000


@pytest.mark.parametrize("name,b,reps,rc,nbins", [
    ("sc3d", np.eye(3) * A3, (13, 13, 13), 12.0, 200),
    ("sc3d_small_box", np.eye(3) * A3, (7, 7, 7), 12.0, 50),          # box 15.1 < 2 rc: multi-image
    ("square2d", np.eye(2) * 1.2, (40, 40), 2.5, 97),
    ("hex2d", np.array([[1.1, 0.0], [0.55, 1.1 * np.sqrt(3) / 2]]), (30, 30), 2.5, 64),
    ("fcc_primitive", np.array([[0.0, 1.6, 1.6], [1.6, 0.0, 1.6], [1.6, 1.6, 0.0]]), (12, 12, 12), 5.0, 41),
    ("triclinic3d", np.array([[2.0, 0.0, 0.0], [0.7, 2.1, 0.0], [-0.4, 0.5, 1.9]]), (10, 11, 12), 5.9, 31),
])
def test_oracle_equals_lattice_closed_form(name, b, reps, rc, nbins):
    x, h = _lattice_positions(b, reps)
    w = oracle.geom_info(h, rc)["w"]
    assert rc < w.min()
    n = x.shape[0]
    cfs = cf.lattice_sums(b, rc, n, nbins=nbins)
    assert cfs["min_edge_gap"] > 1e-5, "a shell sits on the cutoff or a bin edge"
    r = oracle.pair_map(x, h, rc, nbins=nbins)
    assert r["count"] == cfs["count"]
    assert r["band_in"] == 0 and r["band_out"] == 0
    np.testing.assert_array_equal(r["hist_core"], cfs["hist"])
    assert r["hist_maybe"].sum() == 0
    assert r["suminvr"] == pytest.approx(cfs["suminvr"], rel=1e-11)
    assert r["energy"] == pytest.approx(cfs["energy"], rel=1e-10)
    vs = np.abs(cfs["virial"]).max()
    np.testing.assert_allclose(r["virial"], cfs["virial"], rtol=0, atol=1e-10 * vs)
    assert np.abs(r["forces"]).max() < 1e-9 * max(1.0, np.abs(cfs["virial"]).max() / n)


def test_equivalent_lattice_basis_gives_same_sums():
    """A unimodular change of basis H -> U.H describes the same periodic
    system, so every reduction is unchanged."""
    rng = np.random.default_rng(11)
    h = np.diag([14.0, 15.0, 16.0])
    x = rng.uniform(0, 16, size=(300, 3))
    U = np.array([[1, 0, 0], [1, 1, 0], [0, -1, 1]], dtype=np.float64)
    assert round(np.linalg.det(U)) == 1
    h2 = U @ h
    rc = 0.45 * min(oracle.geom_info(h2, 1.0)["w"].min(), 14.0)
    a = oracle.pair_map(x, h, rc, nbins=20)
    b = oracle.pair_map(x, h2, rc, nbins=20)
    assert a["count"] == b["count"]
    np.testing.assert_array_equal(a["hist_core"], b["hist_core"])
    assert a["energy"] == pytest.approx(b["energy"], rel=1e-12)
    np.testing.assert_allclose(a["forces"], b["forces"], atol=1e-10)
    np.testing.assert_allclose(a["virial"], b["virial"], atol=1e-9)
