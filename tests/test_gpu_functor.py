"""The compile-time functor hook (include/cellmap_functor.cuh): user functors
compiled in their own translation unit, mapped over a built cell list, against
the oracle's pair list (Code 2 mapped function; Code 6 Lennard-Jones energy)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import BAND

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    from paper_2202_06427_gb300 import _lib, build
    build.build()
    out = str(tmp_path_factory.mktemp("fx") / "libfx.so")
    pkg = os.path.join(ROOT, "paper_2202_06427_gb300")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "functor_example.cu"), "-o", out, "-L", pkg, "-lcellmap",
                    "-Xlinker", "-rpath," + pkg], check=True)
    _lib.lib()  # libcellmap.so first, so the functor library binds to the same copy
    lib = ctypes.CDLL(out)
    lib.fx_neighbour_counts.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.fx_lj_energy.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                 ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("dim,lcell", [(3, 2), (3, 1), (2, 2)])
def test_functors_match_oracle(cuda_ok, fx, dim, lcell):
    import paper_2202_06427_gb300 as P
    h = np.array([[24.0, 0, 0], [3.0, 23.0, 0], [-2.0, 4.0, 25.0]]) if dim == 3 else np.array([[60.0, 0], [7.0, 58.0]])
    n_side = 22 if dim == 3 else 56
    x = synth.jittered_fractional(h, n_side, n_side ** dim - 5, 0.4, 17 + dim + lcell)
    rc = 3.0 if dim == 3 else 4.0
    cl = P.cl_build(torch.from_numpy(x).cuda(), h, rc, lcell)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    counts = torch.zeros(x.shape[0], dtype=torch.int32, device="cuda")
    assert fx.fx_neighbour_counts(cl.handle, ctypes.c_void_p(counts.data_ptr()), stream) == 0
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    eps, sigma = 0.0442, 1.1
    assert fx.fx_lj_energy(cl.handle, eps, sigma, ctypes.c_void_p(e.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    ref = oracle.pairlist(x, h, rc, band=BAND)
    inside = (ref["d"] < rc) & ~ref["band"]
    maybe = ref["band"]
    want = np.bincount(ref["i"][inside], minlength=x.shape[0]) + np.bincount(ref["j"][inside], minlength=x.shape[0])
    slack = np.bincount(ref["i"][maybe], minlength=x.shape[0]) + np.bincount(ref["j"][maybe], minlength=x.shape[0])
    got = counts.cpu().numpy()
    assert np.all(got >= want) and np.all(got <= want + slack)
    d = ref["d"][ref["d"] < rc]
    q3 = (sigma * sigma / d ** 2) ** 3
    lj = float(np.sum(4 * eps * (q3 * q3 - q3)))
    assert abs(e.item() - lj) <= 1e-5 * np.sum(np.abs(4 * eps * (q3 * q3 - q3)))
