"""CPU-only checks of the C ABI: the library builds and loads, it exports every
function include/*.h declares, and the host-side box preparation (no GPU)
follows the paper's grid rule and the oracle's geometry."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_06427_gb300 import build
    build.build()
    from paper_2202_06427_gb300 import _lib
    return _lib.lib()


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|long long|double)\s*\*?\s*(cl_\w+)\s*\(", text,
                             flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name


def test_pairlist_capacity_guard(lib):
    """The guard applied to the 64-bit pair total before a pair list is
    written: totals past 2^31 (the 16M clustered set has 5.2e9 pairs) are
    compared in 64 bits, never wrapped."""
    from paper_2202_06427_gb300 import _lib as L
    L.lib()
    fits = lib.cl_pairlist_fits
    assert fits(0, 0) == L.CL_OK
    assert fits(16, 16) == L.CL_OK
    assert fits(17, 16) == L.CL_ERR_CAPACITY
    assert fits(5_209_002_118, 16) == L.CL_ERR_CAPACITY
    assert fits(5_209_002_118, 5_209_002_118) == L.CL_OK
    assert fits((1 << 31) + 5, (1 << 31) + 4) == L.CL_ERR_CAPACITY
    assert fits((1 << 32) + 1, 2) == L.CL_ERR_CAPACITY  # wraps to 1 in 32 bits
    assert fits(-1, 10) == -1  # CL_ERR_INVALID_ARG


def test_error_strings(lib):
    from paper_2202_06427_gb300 import cl_error_string
    assert cl_error_string(0) == "ok"
    assert "cutoff" in cl_error_string(-3)
    assert cl_error_string(12345) == "unknown error"


def test_paper_code3_grid(lib):
    """Sec. 2.5, Code 3: sides [10,20,15], rc 1.2 -> [8,16,12] periodic cells of
    side 1.25 (printed with one ghost layer per side as [10,18,14])."""
    from paper_2202_06427_gb300 import cl_box_info
    info = cl_box_info(np.diag([10.0, 20.0, 15.0]), 1.2, 1)
    assert info["grid"] == [8, 16, 12]
    assert [g + 2 for g in info["grid"]] == [10, 18, 14]
    assert info["stencil_full"] == 27 and info["stencil_half"] == 14


@pytest.mark.parametrize("lcell", [1, 2, 3, 4])
@pytest.mark.parametrize("h,rc", [
    (np.eye(3) * 215.443469, 12.0),
    (np.array([[220.0, 0, 0], [30.0, 215.0, 0], [20.0, 25.0, 210.0]]), 10.0),
    (np.array([[37.8, 0.0], [-8.0, 37.8]]), 2.5),
    (np.array([[21.5, 0, 0], [5.0, 21.5, 0], [-4.0, 3.0, 21.5]]), 12.0),
])
def test_grid_matches_oracle_rule(lib, h, rc, lcell):
    from paper_2202_06427_gb300 import cl_box_info
    info = cl_box_info(h, rc, lcell)
    ref = oracle.geom_info(h, rc, lcell)
    assert info["grid"] == [int(v) for v in np.minimum(ref["n"], 1023)]
    np.testing.assert_allclose(info["widths"], ref["w"], rtol=1e-12)
    dim = h.shape[0]
    full = np.prod(2 * ref["m"] + 1)
    assert info["stencil_full"] <= full
    assert info["stencil_half"] == (info["stencil_full"] + 1) // 2


def test_stencil_prunes_far_corners(lib):
    """lcell 3 in a cubic box: the 3x3x3 corner offsets lie at least rc apart
    (minimum cell-to-cell distance sqrt(3) * 2 * side > rc) and are dropped."""
    from paper_2202_06427_gb300 import cl_box_info
    info = cl_box_info(np.eye(3) * 215.443469, 12.0, 3)
    assert info["grid"] == [53, 53, 53]
    assert info["stencil_full"] < 343
    side = 215.443469 / 53
    kept = 0
    for o in np.ndindex(7, 7, 7):
        d = np.maximum(np.abs(np.array(o) - 3) - 1, 0) * side
        kept += float(d @ d) < 144.0 * (1 + 1e-9)
    assert info["stencil_full"] == kept


@pytest.mark.parametrize("h,rc,lcell,code", [
    (np.eye(3) * 10.0, 10.0, 1, -3),
    (np.zeros((3, 3)), 1.0, 1, -2),
    (np.eye(3) * 10.0, -1.0, 1, -1),
    (np.eye(3) * 10.0, 1.0, 0, -1),
    (np.array([[1.0, 0.0], [1.0, 0.0]]), 0.1, 1, -2),
])
def test_box_errors(lib, h, rc, lcell, code):
    from paper_2202_06427_gb300 import CellMapError, cl_box_info
    with pytest.raises(CellMapError) as e:
        cl_box_info(h, rc, lcell)
    assert e.value.code == code


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2202_06427_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.lib()
