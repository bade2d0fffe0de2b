/*
 * cellmap.h -- C ABI of the GB300 cell-list pair map.
 *
 * The calls follow the paper's statement of the problem (CellListMap.jl,
 * Martinez, arXiv 2202.06427, Sec. 2.1-2.2): define the box and cutoff (Sec.
 * 2.5, Code 3), build the cell lists from the coordinates (Sec. 2.6, Code 4),
 * then map a pairwise function over every pair within the cutoff and reduce
 * the per-worker outputs (Sec. 2.3, 2.7, 2.8, Code 1/2/5). The mapped
 * functions are a fixed set of built-in reductions; a compile-time device
 * functor hook (cellmap_functor.cuh) plays the role of the user function.
 *
 * Conventions shared by every call:
 *  - Positions are the caller's (n, dim) row-major FP64 array in DEVICE
 *    memory: x[i*dim + a]. The paper accepts (dim, n) matrices or vectors of
 *    static vectors with this same memory layout (Sec. 2.4). Positions need
 *    not lie inside the box; they are wrapped in FP64.
 *  - The box is a dim x dim lattice matrix whose ROWS are the lattice vectors
 *    (the paper's Julia display prints them as columns, Code 3). Orthorhombic
 *    boxes are diagonal matrices.
 *  - A pair (i, j) is "within the cutoff" when |x_j - x_i + t.H| < rc for
 *    some integer image t (strict inequality). Each such pair-image is mapped
 *    exactly once. When rc > w_min/2 (w = distances between opposite box
 *    faces) one pair can have several images inside the cutoff; each counts.
 *    rc must stay below w_min (a particle must not see itself).
 *  - Indices are 0-based (the paper's Julia indices are 1-based).
 *  - Every call is asynchronous on the given CUDA stream (a cudaStream_t
 *    passed as void*; NULL = legacy default stream) unless its comment says
 *    it synchronizes. Device pointers passed in are owned by the caller and
 *    must stay valid until the work on the stream has completed. The cl_list
 *    handle and its device workspace are owned by the library.
 *  - The calls on one handle share its workspace (cell arrays, work lists,
 *    partial sums): their GPU work must not overlap, so issue them on one
 *    stream, or order the streams. Different handles are independent; a
 *    process may drive several devices (launch parameters are kept per device).
 *  - Return value: CL_OK (0) or a negative error code; cl_error_string()
 *    names it. A failed call leaves the handle usable unless it says
 *    otherwise. Errors detected on the device (non-finite positions) are
 *    latched in the handle and reported by cl_status().
 */
#ifndef CELLMAP_H
#define CELLMAP_H

#ifdef __cplusplus
extern "C" {
#endif

#define CL_OK 0
#define CL_ERR_INVALID_ARG (-1)     /* null pointer, bad size, bad option */
#define CL_ERR_INVALID_BOX (-2)     /* singular or non-finite lattice matrix */
#define CL_ERR_CUTOFF_TOO_LARGE (-3)/* rc >= w_min, or rc > w_min/2 for the pair list */
#define CL_ERR_NONFINITE (-4)       /* a position was NaN or infinite (reported by cl_status) */
#define CL_ERR_OOM (-5)             /* device allocation failed */
#define CL_ERR_CAPACITY (-6)        /* pair list larger than the caller's capacity */
#define CL_ERR_TIMEOUT (-7)         /* a bounded device wait expired */
#define CL_ERR_CUDA (-8)            /* a CUDA runtime call failed */
#define CL_ERR_UNSUPPORTED (-9)     /* grid or stencil beyond the library's limits */

/* Box and cutoff (Sec. 2.5, Code 3). */
typedef struct {
  int dim;          /* 2 or 3 */
  double h[9];      /* lattice matrix, row-major, first dim*dim entries used; rows = lattice vectors */
  double cutoff;    /* rc > 0 */
  int lcell;        /* cells per cutoff length across each face (paper's lcell, Sec. 2.8), 1..4 */
} cl_box;

typedef struct cl_list cl_list; /* opaque; device buffers owned by the library */

/* Built-in reductions (the mapped function of Sec. 2.3).
 *  CL_RED_COUNT      number of pair-images within rc                         -> result.count
 *  CL_RED_SUM_INV_R  sum of 1/r (Code 5, first example)                      -> result.sum_inv_r
 *  CL_RED_SF_ENERGY  sum of u(r) = 1/r - 1/rc + (r - rc)/rc^2 (shifted force) -> result.energy
 *  CL_RED_SF_ENERGY_FORCES_VIRIAL  energy, forces F = -dE/dx (Code 7 pattern)
 *                    and virial W = -sum u'(r)/r r(x)r                        -> energy, forces, virial
 *  CL_RED_HIST       counts of r in nbins equal bins over [0, rmax) (Code 10) -> result.hist
 *  CL_RED_PAIRLIST   i<j neighbour list sorted by (i, j) with FP32 distance
 *                    (Sec. 4.1); requires rc <= w_min/2 (unique images)       -> pair_i, pair_j, pair_d */
typedef enum {
  CL_RED_COUNT = 0,
  CL_RED_SUM_INV_R = 1,
  CL_RED_SF_ENERGY = 2,
  CL_RED_SF_ENERGY_FORCES_VIRIAL = 3,
  CL_RED_HIST = 4,
  CL_RED_PAIRLIST = 5
} cl_reduction;

typedef struct {
  int nbins;    /* CL_RED_HIST: number of bins, 1..4096 */
  double rmax;  /* CL_RED_HIST: upper edge of the last bin; <= 0 means rc */
} cl_params;

/* Outputs of cl_map. All pointers are DEVICE pointers owned by the caller,
 * except npairs (host). Only the fields the chosen reduction writes are read;
 * the others may be NULL. Scalars are overwritten, not accumulated. */
typedef struct {
  unsigned long long* count;  /* 1 value */
  double* sum_inv_r;          /* 1 value */
  double* energy;             /* 1 value */
  float* forces;              /* n*dim, original particle order */
  double* virial;             /* dim*dim, row-major */
  unsigned long long* hist;   /* nbins */
  int* pair_i;                /* capacity entries; pair_i[k] < pair_j[k] */
  int* pair_j;
  float* pair_d;              /* distance of each pair */
  long long capacity;         /* entries available in pair_i/pair_j/pair_d */
  long long* npairs;          /* HOST: number of pairs found (also set on CL_ERR_CAPACITY) */
} cl_result;

/* Build the cell list (Sec. 2.6) of n particles: wrap each position into the
 * box and compute its fractional cell in FP64, count particles per cell,
 * prefix-sum the counts into cell offsets, scatter FP32 cell-local
 * coordinates into cell order, and list the work tiles of the sweep.
 * pos_dev: (n, dim) FP64 device array (0 <= n < 2^31). The pointer is kept by
 * the handle (cl_backward reads the raw positions again) and must stay valid
 * until the next cl_update or cl_free. Allocates device memory (synchronous
 * cudaMalloc); the kernels run on `stream`. On success *out receives a new
 * handle. Errors: INVALID_ARG, INVALID_BOX, CUTOFF_TOO_LARGE, UNSUPPORTED,
 * OOM, CUDA. */
int cl_build(const double* pos_dev, long long n, const cl_box* box, void* stream, cl_list** out);

/* Rebuild the cell list for new positions of the same n particles (Sec. 4.2:
 * the lists are updated between steps), reusing the workspace. box may be
 * NULL (unchanged) or a new box; a new box that changes the grid reallocates.
 * Same errors as cl_build. */
int cl_update(cl_list* cl, const double* pos_dev, const cl_box* box, void* stream);

/* Map a built-in reduction over every pair-image within the cutoff (Sec. 2.3,
 * 2.7) and write the reduced result (Sec. 2.8: per-worker partial outputs are
 * summed; here per-CTA FP64 partials are summed in a fixed order).
 * Asynchronous except CL_RED_PAIRLIST, which synchronizes `stream` once to
 * learn the pair count and returns CL_ERR_CAPACITY (with *npairs set) when it
 * exceeds result->capacity; call again with more room. The pair count and the
 * list's offsets are 64-bit: a list may hold more than 2^31 pairs (indices
 * stay int32, since n < 2^31). params may be NULL except for CL_RED_HIST. */
int cl_map(const cl_list* cl, cl_reduction red, const cl_params* params, cl_result* result, void* stream);

/* Adjoint of the shifted-force energy (Sec. 3.3, Code 9: the pair sum is
 * differentiable). Given dL/dE in grad_energy_dev (1 FP64 value, device),
 * writes grad_pos_dev[i*dim+a] = dL/dE * dE/dx_ia (= -dL/dE * force) for the
 * positions the list was last built from, and, when grad_box_dev is not NULL,
 * grad_box_dev = dL/dE * dE/dH at fixed Cartesian positions (dim*dim,
 * row-major). When virial_dev is not NULL it also receives the virial W.
 * All output arrays are overwritten. */
int cl_backward(const cl_list* cl, const double* grad_energy_dev, double* grad_pos_dev, double* grad_box_dev,
                double* virial_dev, void* stream);

/* Energy and its gradient in one sweep: the forward pass of a differentiable
 * caller that needs the gradient afterwards (Sec. 3.3, Code 9, with the
 * forward and the adjoint fused). Writes energy_dev[0] = E (the value
 * cl_map(CL_RED_SF_ENERGY) gives) and, scaled by s = scale_dev[0] (1 FP64
 * value, device; 1 for the plain derivatives), grad_pos_dev = s dE/dx
 * ((n, dim) FP64, original order) and, when grad_box_dev is not NULL,
 * grad_box_dev = s dE/dH (dim*dim); virial_dev (optional) receives W. The
 * same outputs as cl_map(CL_RED_SF_ENERGY) plus cl_backward(scale_dev), at the
 * cost of one sweep (in 3D the half-shell sweep with forces on both particles
 * of each pair-image, then one pass over the particles). Errors as
 * cl_backward. */
int cl_energy_grad(const cl_list* cl, const double* scale_dev, double* energy_dev, double* grad_pos_dev,
                   double* grad_box_dev, double* virial_dev, void* stream);

/* out_dev[k] = s * in_dev[k] for k < count, s = scale_dev[0] (FP64, device):
 * the chain rule applied to a gradient saved by cl_energy_grad. in_dev and
 * out_dev may be the same array. Errors: INVALID_ARG, CUDA. */
int cl_scale(const double* scale_dev, const double* in_dev, double* out_dev, long long count, void* stream);

/* Queries. Grid and size values are answered from the host; NONEMPTY,
 * MAX_OCCUPANCY and CANDIDATES read device counters and synchronize
 * `stream` (NULL = legacy default stream) first. */
#define CL_INFO_N 0
#define CL_INFO_DIM 1
#define CL_INFO_GRID_X 2
#define CL_INFO_GRID_Y 3
#define CL_INFO_GRID_Z 4
#define CL_INFO_NCELLS 5
#define CL_INFO_NONEMPTY 6
#define CL_INFO_MAX_OCCUPANCY 7
#define CL_INFO_BYTES 8
#define CL_INFO_STENCIL_HALF 9      /* neighbour-cell offsets visited per cell by the half-shell sweep */
#define CL_INFO_STENCIL_FULL 10     /* offsets of the full stencil (forces, backward) */
#define CL_INFO_CANDIDATES 11       /* candidate pairs the half-shell sweep tests (cell occupancy products) */
#define CL_INFO_WORK_TILES 12       /* CTAs of 256 threads the particle sweeps launch (one thread per particle) */
#define CL_INFO_SWEEP_CANDIDATES 13 /* candidate pairs the last 3D energy/force sweep evaluated (staged
                                       neighbours x home particles, own cell included); reads a counter */
#define CL_INFO_SWEEP_HALF 14       /* 1 when the last 3D energy/force sweep with forces evaluated each
                                       pair-image once (half shell; taken when both stencils have at
                                       most 129 offsets), 0 when it took the full-shell kernels */
int cl_query(const cl_list* cl, int what, long long* value, void* stream);

/* Two sets of particles (Sec. 3.2, Code 8; Sec. 4.1): set A is the cell list
 * `cl`, set B the (nb, dim) FP64 device positions posb_dev in the same box.
 * The pair-images are every (a, b, t) with |y_b - x_a + t.H| < cutoff (no
 * a < b rule); a and b are 0-based indices into A and B. Each b is binned on
 * A's grid in FP64 and sweeps the full stencil of its cell. These calls
 * synchronize `stream` and allocate their workspace (cudaMalloc/cudaFree).
 * Errors: INVALID_ARG, NONFINITE (a position of B), OOM, CUDA, and as noted.
 *
 * cl_cross_count: count_dev[0] = number of cross pair-images (u64).
 *
 * cl_cross_pairlist: the cross pairs as (pa, pb, pd) sorted by (b, a), pd the
 * FP32 distance; *npairs (host) receives the number of pairs. Same capacity
 * protocol as CL_RED_PAIRLIST (CL_ERR_CAPACITY: call again with capacity >=
 * *npairs); requires unique images (cutoff <= w_min / 2, else
 * CUTOFF_TOO_LARGE).
 *
 * cl_cross_knn: for each b its k nearest a within the cutoff, ascending by
 * distance (ties: smaller a first): knn_a_dev[b*k + q] (a, or -1 when b has
 * fewer than q+1 neighbours), knn_d_dev[b*k + q] (FP32 distance, +inf when
 * empty). 1 <= k <= CL_KNN_MAX.
 *
 * cl_cross_topk (Code 8): the k cross pair-images of smallest distance within
 * the cutoff, ascending: a_dev[q], b_dev[q], d_dev[q] for q < *nfound (host,
 * min(k, number of cross pairs)); the rest hold -1, -1, +inf. 1 <= k <=
 * CL_KNN_MAX. */
#define CL_KNN_MAX 32
int cl_cross_count(const cl_list* cl, const double* posb_dev, long long nb, unsigned long long* count_dev,
                   void* stream);
int cl_cross_pairlist(const cl_list* cl, const double* posb_dev, long long nb, long long capacity, int* pa_dev,
                      int* pb_dev, float* pd_dev, long long* npairs, void* stream);
int cl_cross_knn(const cl_list* cl, const double* posb_dev, long long nb, int k, int* knn_a_dev, float* knn_d_dev,
                 void* stream);
int cl_cross_topk(const cl_list* cl, const double* posb_dev, long long nb, int k, int* a_dev, int* b_dev,
                  float* d_dev, long long* nfound, void* stream);

/* Box for particles WITHOUT periodic boundaries (Sec. 4.1, Fig. 2): reduces
 * the extent of the (n, dim) FP64 device positions pos_dev (and of a second set
 * pos2_dev of n2 points, may be NULL with n2 = 0, e.g. the other set of a
 * two-set neighbour list) on `stream`, synchronizes, and writes to *box_out an
 * orthorhombic box whose side along each axis exceeds extent + cutoff, so that
 * every periodic image of a pair but the direct one is at least the cutoff
 * away: cl_build with this box maps the pairs of the open system. Errors:
 * INVALID_ARG, NONFINITE (a coordinate is not finite), OOM, CUDA. */
int cl_box_nonperiodic(const double* pos_dev, long long n, const double* pos2_dev, long long n2, int dim,
                       double cutoff, int lcell, void* stream, cl_box* box_out);

/* Mapped functions of the paper's examples, built on the compile-time functor
 * hook (cellmap_pairfns.cuh) with one thread per cell-sorted particle. All
 * arrays are DEVICE arrays in original particle order; scalar and histogram
 * outputs are zeroed and then accumulated, FP64. Asynchronous on `stream`.
 *
 * cl_map_mass (Code 5, second example): out_dev[0] = sum over the pair-images
 * within the cutoff of m_i m_j / r, mass_dev = n FP32 masses.
 *
 * cl_map_lj (Code 6, 7): energy_dev[0] = sum of 4 eps ((sigma/r)^12 -
 * (sigma/r)^6) over the pair-images within the cutoff (not shifted); when
 * forces_dev ((n, dim) FP32) is not NULL also the forces F = -dE/dx (the
 * gradient of that energy). Errors: INVALID_ARG (sigma <= 0, non-finite).
 *
 * cl_map_velocity_hist (Code 10): for each pair-image within the cutoff, bin
 * k = ceil(r / binstep) (1-based, closed on the right); when k <= nbins,
 * counts_dev[k-1] += 1 and vsum_dev[k-1] += |v_i - v_j| with vel_dev (n, dim)
 * FP32 velocities. 1 <= nbins <= CL_VHIST_MAX_BINS. */
#define CL_VHIST_MAX_BINS 64
int cl_map_mass(const cl_list* cl, const float* mass_dev, double* out_dev, void* stream);
int cl_map_lj(const cl_list* cl, double eps, double sigma, double* energy_dev, float* forces_dev, void* stream);
int cl_map_velocity_hist(const cl_list* cl, const float* vel_dev, double binstep, int nbins,
                         unsigned long long* counts_dev, double* vsum_dev, void* stream);

/* Host-only box preparation, no GPU needed: for box, fills
 * grid[3] (cells per axis, 1 for unused axes), widths[3] (face distances) and
 * stencil[2] (half-shell and full-shell offset counts). Same errors as the
 * box checks of cl_build. */
int cl_box_info(const cl_box* box, long long* grid, double* widths, long long* stencil);

/* Synchronize `stream` and report a latched device-side error of the handle
 * (CL_ERR_NONFINITE when any position of the last build was not finite), or
 * CL_OK. Reading clears the latch. */
int cl_status(cl_list* cl, void* stream);

/* Shifted-force energy of a small particle set WITHOUT allocating device
 * memory (the paper has no counterpart; it exists for callers of this
 * library). For applications that route all device memory through their own
 * pool or framework allocator and may not call cudaMalloc/cudaFree, and for
 * latency-critical loops that cannot afford them: cl_build allocates, this
 * call does not. It computes the same shifted-force energy as cl_build +
 * cl_map(CL_RED_SF_ENERGY), equal to it within the energy tolerance (relative
 * 1e-6; it runs a different sweep kernel, one thread per particle over the
 * unpruned half stencil, so the summation order differs), with every
 * intermediate buffer in one fixed device array inside the library (3.18 MB,
 * held by every GPU that loads the library until the process exits).
 * pos_dev: (n, dim) FP64 device positions; energy_dev: 1 FP64 device value,
 * overwritten. Limits: n <= CL_NOALLOC_MAX_N and at most
 * CL_NOALLOC_MAX_CELLS cells in the grid the box and lcell give; larger
 * inputs return CL_ERR_UNSUPPORTED and launch nothing. Other errors as for
 * cl_build. A non-finite position never pairs and is not reported.
 * The first call made with a given device current looks up the array's
 * device address for that device; make that first call before any stream
 * capture begins. All calls share the array: calls whose GPU work overlaps
 * (different streams, or unordered host threads) race and give wrong results;
 * calls ordered on one stream are safe. Asynchronous on `stream`. */
#define CL_NOALLOC_MAX_N 65536
#define CL_NOALLOC_MAX_CELLS 65536
int cl_energy_noalloc(const double* pos_dev, long long n, const cl_box* box, double* energy_dev, void* stream);

/* Release the handle and its device memory (synchronizes the device). NULL is ignored. */
void cl_free(cl_list* cl);

/* Static description of an error code. */
const char* cl_error_string(int code);

/* The guard the pair-list calls (CL_RED_PAIRLIST, cl_cross_pairlist) apply
 * to the 64-bit total of their count pass before any pair is written: CL_OK
 * when 0 <= npairs <= capacity, CL_ERR_CAPACITY when npairs > capacity (the
 * call then returns with *npairs set and writes nothing), CL_ERR_INVALID_ARG
 * for a negative total. Host-only, no device work. */
int cl_pairlist_fits(long long npairs, long long capacity);

/* One neighbour-cell offset o of the stencil: its periodic cell step
 * (o_k mod n_k, in [0, n_k)) and the Cartesian shift S_o = sum_k (o_k/n_k) H_k
 * between the centres of a cell and of its neighbour o, unwrapped. */
typedef struct {
  int dx, dy, dz;
  float sx, sy, sz;
} cl_offset;

/* Read-only device view of a built cell list, for sweeps compiled outside the
 * library (cellmap_functor.cuh). Cell-sorted particles xs[n] hold FP32
 * coordinates relative to the centre of their cell and, in w, the original
 * index (int bits); cellc[n] = cx | cy << 10 | cz << 20; cell_start[ncells+1]
 * are the cell offsets (cells x-fastest). off_half[0] / off_full[0] is the
 * own cell; the half stencil holds the lexicographically positive offsets,
 * the full stencil all of them. All pointers are device memory owned by the
 * handle, valid until the next cl_update or cl_free. The order of the
 * particles within a cell is not fixed: the 3D sweeps may reorder the
 * particles of cells of more than 128 particles by octant (xs and cellc stay
 * consistent; cell_start does not change). */
typedef struct {
  int dim;
  int n;
  int nx, ny, nz;
  float cutoff;
  const void* xs;          /* float4[n] */
  const unsigned* cellc;
  const int* cell_start;
  const cl_offset* off_half;
  int noff_half;
  const cl_offset* off_full;
  int noff_full;
} cl_view;

int cl_get_view(const cl_list* cl, cl_view* view);

#ifdef __cplusplus
}
#endif

#endif /* CELLMAP_H */
