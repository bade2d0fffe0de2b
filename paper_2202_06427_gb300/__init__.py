"""GB300 cell-list pair map (CellListMap.jl, arXiv 2202.06427): binning and
neighbour-cell sweep in hand-written CUDA for sm_103a behind a C ABI
(include/cellmap.h), with this thin Python binding over it."""
from .api import (CellList, CellMapError, box_nonperiodic, cl_backward, cl_box_info, cl_build, cl_build_open,
                  cl_cross_count, cl_cross_knn, cl_cross_pairlist, cl_cross_topk,
                  cl_energy_grad, cl_error_string,
                  cl_free, cl_map, cl_map_lj, cl_map_mass, cl_map_velocity_hist, cl_query, cl_scale, cl_status,
                  cl_update, make_box)
from .autograd import ShiftedForceEnergy, energy

__all__ = ["CellList", "CellMapError", "box_nonperiodic", "cl_build_open", "cl_cross_count", "cl_cross_knn",
           "cl_cross_pairlist", "cl_cross_topk", "cl_backward", "cl_box_info", "cl_build", "cl_energy_grad", "cl_error_string",
           "cl_free", "cl_map", "cl_map_lj", "cl_map_mass", "cl_map_velocity_hist", "cl_query", "cl_scale",
           "cl_status", "cl_update", "make_box", "ShiftedForceEnergy", "energy"]
