"""Golden fixtures: values printed by the paper (cited in each file) and the
closed-form lattice numbers written by tests/golden/make_golden.py."""
import os

import numpy as np

import oracle

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_fixture(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [float(v) for v in vals]
    return out


def test_paper_code3_orthorhombic_grid():
    """Sec. 2.5, Code 3: Box([10,20,15], 1.2) -> computing cells [10,18,14] of
    side 1.25, total 2520, i.e. [8,16,12] periodic cells plus one ghost layer
    per side. The oracle's grid rule n_k = floor(w_k lcell / rc) reproduces it."""
    g = read_fixture("paper_code3_box.txt")
    h = np.diag(g["sides"])
    info = oracle.geom_info(h, g["cutoff"][0], int(g["lcell"][0]))
    n = info["n"]
    np.testing.assert_array_equal(n + 2, np.array(g["computing_cells"], dtype=int))
    np.testing.assert_allclose(np.array(g["sides"]) / n, g["cell_size"], rtol=1e-12)
    assert int(np.prod(n + 2)) == int(g["total_cells"][0])


def test_lattice_fixture_matches_closed_form_and_oracle_on_a_subbox():
    """The stored 1M-lattice numbers (738 neighbours per site) equal the oracle
    per site on a smaller box of the same lattice: per-site sums are
    independent of the number of sites once the box is wider than 2 rc."""
    g = read_fixture("lattice_w1.txt")
    assert int(g["neighbours_per_site"][0]) == 738
    assert int(g["count"][0]) == 369_000_000
    a = 10.0 ** (1.0 / 3.0)
    reps = 12
    grid = np.stack(np.meshgrid(*[np.arange(reps)] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    x = grid.astype(np.float64) * a
    h = np.eye(3) * reps * a
    r = oracle.pair_map(x, h, 12.0, nbins=200, forces=False)
    scale = 100 ** 3 / reps ** 3
    assert r["count"] * scale == g["count"][0]
    assert abs(r["suminvr"] * scale / g["suminvr"][0] - 1) < 1e-12
    assert abs(r["energy"] * scale / g["energy"][0] - 1) < 1e-11
    np.testing.assert_array_equal(np.round(r["hist_core"] * scale).astype(np.int64),
                                  np.array(g["hist200"], dtype=np.int64))
