"""cl_energy_noalloc, the entry point for callers that may not allocate device
memory (applications whose framework or pool allocator owns all device memory
and forbids raw cudaMalloc/cudaFree, latency-critical loops that cannot pay
for an allocation): its energy must equal the regular path, cl_build +
cl_map(CL_RED_SF_ENERGY), and the FP64 oracle within the energy tolerance of
the parity tests, on consecutive calls that reuse its fixed device workspace,
up to the largest input it accepts (65,536 particles on a grid of 65,536
cells).

Collected last on purpose (file name), so a failure here leaves every other
test already run."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import BAND, TOL_E, check_energy

pytestmark = pytest.mark.gpu


def _noalloc(x, h, rc, lcell, out):
    from paper_2202_06427_gb300 import _lib, api
    box = api.make_box(h, rc, lcell)
    return _lib.lib().cl_energy_noalloc(ctypes.c_void_p(x.data_ptr()), x.shape[0], ctypes.byref(box),
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _regular(x, h, rc, lcell):
    import paper_2202_06427_gb300 as P
    return P.cl_map(P.cl_build(x, h, rc, lcell), "energy")["energy"].item()


def _systems():
    h3 = np.array([[20.0, 0.0, 0.0], [3.0, 20.0, 0.0], [-2.0, 4.0, 20.0]])
    x3 = synth.jittered_fractional(h3, 20, 7980, 0.4, 71)
    h2 = np.array([[60.0, 0.0], [-9.0, 60.0]])
    x2 = synth.jittered_fractional(h2, 60, 3500, 0.4, 72)
    return [(x3, h3, 3.0, 2), (x2, h2, 4.0, 3)]


def test_noalloc_energy_matches_regular_path_on_consecutive_calls(cuda_ok):
    cases = _systems()
    order = [0, 1, 0]  # a second system in between: leftovers of one call must not leak into the next
    for k in order:
        x_np, h, rc, lcell = cases[k]
        x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(x, h, rc, lcell, out) == 0
        got = out.item()
        want = _regular(x, h, rc, lcell)
        assert abs(got - want) <= TOL_E * abs(want), (k, got, want)
        check_energy(got, oracle.pair_map(x_np, h, rc, band=BAND, forces=False)["energy"])


def test_noalloc_energy_at_its_largest_input(cuda_ok):
    """n = CL_NOALLOC_MAX_N particles on a 64 x 32 x 32 grid (= CL_NOALLOC_MAX_CELLS
    cells: box 48.01 x 24.01 x 24.01, rc 3, four cells per cutoff length), two
    calls in a row, against the oracle and the regular path."""
    h = np.diag([48.01, 24.01, 24.01])
    x_np = synth.jittered_fractional(h, 41, 65_536, 0.4, 73)
    rc, lcell = 3.0, 4
    import paper_2202_06427_gb300 as P
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    assert P.cl_query(P.cl_build(x, h, rc, lcell), "ncells") == 65_536
    ref = oracle.pair_map(x_np, h, rc, band=BAND, forces=False)["energy"]
    want = _regular(x, h, rc, lcell)
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(x, h, rc, lcell, out) == 0
        check_energy(out.item(), ref)
        assert abs(out.item() - want) <= TOL_E * abs(want)


def test_noalloc_rejects_inputs_beyond_its_workspace(cuda_ok):
    x = torch.zeros((65537, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(x, np.eye(3) * 100.0, 3.0, 1, out) == -9
    # a grid with more than 65,536 cells is refused the same way
    x_small = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    assert _noalloc(x_small, np.eye(3) * 300.0, 3.0, 2, out) == -9
