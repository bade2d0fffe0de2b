"""ctypes declarations of the C ABI in include/cellmap.h.

Loading fails loudly when libcellmap.so is missing: there is no fallback
implementation anywhere in the package.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcellmap.so")

CL_OK = 0
CL_ERR_CAPACITY = -6
ERRORS = {
    -1: "CL_ERR_INVALID_ARG", -2: "CL_ERR_INVALID_BOX", -3: "CL_ERR_CUTOFF_TOO_LARGE", -4: "CL_ERR_NONFINITE",
    -5: "CL_ERR_OOM", -6: "CL_ERR_CAPACITY", -7: "CL_ERR_TIMEOUT", -8: "CL_ERR_CUDA", -9: "CL_ERR_UNSUPPORTED",
}

CL_RED_COUNT, CL_RED_SUM_INV_R, CL_RED_SF_ENERGY, CL_RED_SF_ENERGY_FORCES_VIRIAL, CL_RED_HIST, CL_RED_PAIRLIST = range(6)

INFO = {"n": 0, "dim": 1, "grid_x": 2, "grid_y": 3, "grid_z": 4, "ncells": 5, "nonempty": 6, "max_occupancy": 7,
        "bytes": 8, "stencil_half": 9, "stencil_full": 10, "candidates": 11, "work_tiles": 12,
        "sweep_candidates": 13, "sweep_half": 14}


class cl_box(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("h", ctypes.c_double * 9), ("cutoff", ctypes.c_double),
                ("lcell", ctypes.c_int)]


class cl_params(ctypes.Structure):
    _fields_ = [("nbins", ctypes.c_int), ("rmax", ctypes.c_double)]


class cl_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_void_p), ("sum_inv_r", ctypes.c_void_p), ("energy", ctypes.c_void_p),
                ("forces", ctypes.c_void_p), ("virial", ctypes.c_void_p), ("hist", ctypes.c_void_p),
                ("pair_i", ctypes.c_void_p), ("pair_j", ctypes.c_void_p), ("pair_d", ctypes.c_void_p),
                ("capacity", ctypes.c_longlong), ("npairs", ctypes.POINTER(ctypes.c_longlong))]


class CellMapError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__("%s%s (%d)" % (where + ": " if where else "", ERRORS.get(code, "?"), code))


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libcellmap.so is not built (run __graft_entry__.build() or "
                              "python paper_2202_06427_gb300/build.py); there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        P, ll, i32 = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int
        L.cl_build.argtypes = [P, ll, ctypes.POINTER(cl_box), P, ctypes.POINTER(P)]
        L.cl_update.argtypes = [P, P, ctypes.POINTER(cl_box), P]
        L.cl_map.argtypes = [P, i32, ctypes.POINTER(cl_params), ctypes.POINTER(cl_result), P]
        L.cl_backward.argtypes = [P, P, P, P, P, P]
        L.cl_energy_grad.argtypes = [P, P, P, P, P, P, P]
        L.cl_scale.argtypes = [P, P, P, ll, P]
        L.cl_pairlist_fits.argtypes = [ll, ll]
        L.cl_map_mass.argtypes = [P, P, P, P]
        L.cl_map_lj.argtypes = [P, ctypes.c_double, ctypes.c_double, P, P, P]
        L.cl_map_velocity_hist.argtypes = [P, P, ctypes.c_double, i32, P, P, P]
        L.cl_box_nonperiodic.argtypes = [P, ll, P, ll, i32, ctypes.c_double, i32, P, ctypes.POINTER(cl_box)]
        L.cl_cross_count.argtypes = [P, P, ll, P, P]
        L.cl_cross_pairlist.argtypes = [P, P, ll, ll, P, P, P, ctypes.POINTER(ll), P]
        L.cl_cross_knn.argtypes = [P, P, ll, i32, P, P, P]
        L.cl_cross_topk.argtypes = [P, P, ll, i32, P, P, P, ctypes.POINTER(ll), P]
        L.cl_query.argtypes = [P, i32, ctypes.POINTER(ll), P]
        L.cl_box_info.argtypes = [ctypes.POINTER(cl_box), P, P, P]
        L.cl_status.argtypes = [P, P]
        L.cl_free.argtypes = [P]
        L.cl_free.restype = None
        L.cl_energy_noalloc.argtypes = [P, ll, ctypes.POINTER(cl_box), P, P]
        L.cl_energy_noalloc.restype = ctypes.c_int
        L.cl_error_string.argtypes = [i32]
        L.cl_error_string.restype = ctypes.c_char_p
        for f in ("cl_build", "cl_update", "cl_map", "cl_backward", "cl_energy_grad", "cl_scale", "cl_query",
                  "cl_box_info", "cl_status", "cl_map_mass", "cl_map_lj", "cl_map_velocity_hist",
                  "cl_box_nonperiodic", "cl_cross_count", "cl_cross_pairlist", "cl_cross_knn", "cl_cross_topk"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def check(code, where=""):
    if code != CL_OK:
        raise CellMapError(code, where)
