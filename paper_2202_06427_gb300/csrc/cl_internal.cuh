// cl_internal.cuh -- types shared by the translation units of libcellmap.
//
// Data layout in device memory (one cl_list):
//   xs[n]        float4  cell-sorted particles: (x, y, z) FP32 relative to the
//                        CENTRE of the particle's own cell, w = original index
//                        (int bits). 2D sets z = 0.
//   cellc[n]     uint32  packed cell coordinates of each sorted particle:
//                        cx | cy << 10 | cz << 20 (at most 1023 cells per axis)
//   cell_start[ncells+1] prefix sum of the per-cell counts: particles of cell
//                        c occupy xs[cell_start[c] .. cell_start[c+1]). Cells
//                        are linearised x-fastest, c = cx + nx (cy + ny cz),
//                        so a row of cells along x is one contiguous range.
// The displacement from particle i (cell ci) to particle j in the neighbour
// cell reached by the integer offset o (wrapped periodically) is
//   r = (xs_j + S_o) - xs_i,   S_o = sum_k (o_k / n_k) H_k,
// because the centre of cell ci + o, unwrapped, is the centre of the wrapped
// cell plus the lattice translation. S_o depends on o only, so one FP32 shift
// per stencil entry serves every cell (Sec. 2.6 replicates ghost particles to
// the same end; this build stores no ghosts).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "cellmap.h"

namespace clk {

// Launch parameters worked out once per device (occupancy, opt-in shared
// memory, which cudaFuncSetAttribute sets for the current device only): one
// slot per device, 0 until known. Devices past the table are not cached.
constexpr int kCacheDevices = 64;
struct DevCache {
  std::atomic<int> v[kCacheDevices];
  int get(int dev) const { return dev >= 0 && dev < kCacheDevices ? v[dev].load(std::memory_order_relaxed) : 0; }
  void put(int dev, int x) {
    if (dev >= 0 && dev < kCacheDevices) v[dev].store(x, std::memory_order_relaxed);
  }
};

constexpr int kMaxOff = 768;      // stencil entries (9^3 = 729 plus margin)
constexpr int kMaxAxis = 1023;    // cells per axis (10-bit packing)
constexpr int kMaxBins = 4096;    // histogram bins (shared-memory histogram)
// Cells of kOctMin to kOctCap particles are ordered by the octant of their
// particles' local coordinates (sign of x, y, z) by the 3D half-shell sweep
// when it builds its work lists, so that it can split their particles into
// compact groups.
constexpr int kOctMin = 129;
constexpr int kOctCap = 2048;

// One neighbour-cell offset of the stencil.
struct Off {
  int dx, dy, dz;     // o_k mod n_k, in [0, n_k)
  float sx, sy, sz;   // Cartesian shift S_o (FP32 of an FP64 value)
};

// Box geometry after preparation (host and device copies).
struct Geo {
  int dim;
  int n[3];           // cells per axis (1 for unused axes)
  long long ncells;
  double h[9];        // lattice rows, 3x3 (2D padded with identity z)
  double hinv[9];     // H^-1, 3x3
  double m[9];        // M = H^-1 diag(n): t = x M is the position in cell units
  double w[3];        // distances between opposite faces
  float g[9];         // cell edge vectors G_k = H_k / n_k (rows), FP32
  int ortho;          // 1 when H is diagonal
  double rc;
  int lcell;
};

// Device-side error latch bits.
constexpr int kErrNonFinite = 1;

// Stand-in coordinates for a particle whose input position is not finite (and
// for the element past the last one in the shifted-pair arrays): far outside
// any box, unique per index and at least 1e12 apart from each other, finite,
// so that every distance test against them fails without producing NaN.
__device__ __forceinline__ float4 sentinel_pos(int i) {
  const float big = 1e15f, step = 1.0f / 1024.0f;
  return make_float4(big * (1.0f + (float)(i & 1023) * step), big * (1.0f + (float)((i >> 10) & 1023) * step),
                     big * (1.0f + (float)((i >> 20) & 1023) * step), 0.0f);
}

// Launch arguments of the sweep kernels (passed as one __grid_constant__ parameter).
struct SweepArgs {
  const float4* xs;
  const unsigned* cellc;
  const int* cell_start;
  int n;
  int nx, ny, nz;
  float rc2, irc, irc2;
  // Half-widths of one cell's Cartesian bounding box, padded by 1e-3 rc (3D
  // packed per-particle sweep: a neighbour cell whose box lies at least rc
  // from the particle is skipped); 0 turns the test off.
  float ex, ey, ez;
  int noff;             // entries in off[]; off[0] is the own cell
  Off off[kMaxOff];
};

// Host helpers implemented in cl_geom.cu.
int prepare_geometry(const cl_box* box, Geo* geo);
// Builds the half-shell (half = 1) or full stencil; returns the entry count or a
// negative error. opk (optional) receives each entry's unwrapped offset packed
// as bytes: (ox & 255) | (oy & 255) << 8 | (oz & 255) << 16.
int build_stencil(const Geo& geo, int half, Off* out, int cap, int* opk = nullptr);
// Half-widths of one cell's Cartesian bounding box (sum over the cell edge
// vectors of |G_k,a| / 2 per axis a), each padded by 1e-3 rc.
void cell_halfwidths(const Geo& geo, float* e);

}  // namespace clk

namespace clk {

// Buffers of one binning pipeline (cl_build.cu).
struct BuildBufs {
  const double* pos;
  int n;
  int* slot;    // per original particle: position inside its cell
  float4* xl;   // per original particle: centred local coordinate, w = packed cell (cx | cy << 10 | cz << 20)
  int* counts;
  int* cell_start;
  int* tile_sum;
  int* meta;  // [0] error latch, [1] non-empty cells, [2] max occupancy
  float4* xs;
  unsigned* cellc;
};
int scan_tiles_for(long long ncells);
int launch_build(const Geo& g, const BuildBufs& b, cudaStream_t s);
// Orders the particles of the listed cells (ncells_listed of them, read on the
// device) with kOctMin..kOctCap particles by octant; slots follow.
int launch_octsort(const int* cells, const int* ncells_listed, const int* cell_start, float4* xs, int* slot,
                   cudaStream_t s);
int launch_scan64(const int* counts, long long n, long long* tile_sum, long long* start, int* meta, cudaStream_t s);

// Sweeps and reductions (cl_sweep.cu).
int sweep_partials_needed(int n);
int launch_count(const SweepArgs& A, int dim, unsigned long long* out, cudaStream_t s);
int launch_scalar(const SweepArgs& A, int dim, int kind, double* partials, double* sums, double* out,
                  cudaStream_t s);
int launch_hist(const SweepArgs& A, int dim, int nbins, float rmax, unsigned long long* hist, cudaStream_t s);
// The same three sweeps (3D) over the particles of the cells with flag != 0
// only (the cells a neighbourhood sweep left), adding to out / hist without
// zeroing them; the sum 1/r kind writes blocks_for(n) partials and no final
// reduction.
int launch_count_flagged(const SweepArgs& A, const unsigned char* flag, unsigned long long* out, cudaStream_t s);
int launch_suminvr_flagged(const SweepArgs& A, const unsigned char* flag, double* partials, cudaStream_t s);
int launch_hist_flagged(const SweepArgs& A, const unsigned char* flag, int nbins, float rmax,
                        unsigned long long* hist, cudaStream_t s);
int flagged_blocks(int n);
int launch_force(const SweepArgs& A, int dim, int mode, const double* hinv, float* forces, double* grad,
                 const double* gE, const double* pos, double* partials, double* sums, double* energy,
                 double* virial, double* gradbox, cudaStream_t s);
int launch_candidates(const SweepArgs& A, long long ncells, unsigned long long* out, cudaStream_t s);
// Sums per-CTA partials[nblocks][nv] and writes the caller's outputs. final_mode:
// 0 sum 1/r, 1 energy, 2 forward forces (energy + virial), 3 backward, 4 energy
// and backward (partials S6, X9, E).
int launch_scale(const double* g, const double* in, double* out, long long count, cudaStream_t s);
int finish_reduction(int final_mode, int dim, const double* hinv, int nblocks, int nv, const double* partials,
                     double* sums, double* scalar, double* virial, double* gradbox, const double* gE,
                     cudaStream_t s);

// Neighbourhood sweep of the 3D shifted-force energy (cl_hood.cu).
struct HoodArgs {
  int opk[2][kMaxOff];  // unwrapped stencil offsets (see build_stencil): [0] full, [1] half stencil
  // rows of the half stencil (entries 1..: runs of consecutive ox with one
  // (oy, oz)) as (ox0, ox1, oy, oz); nrows_half of them, 0 when more than 128
  signed char rows_half[128][4];
  int nrows_half;
  double g[9];        // cell edge vectors G_k = H_k / n_k (rows), FP64
  float gf[9];        // the same, FP32
  float rc;
  float hd;           // largest distance of a cell point from the cell centre
  float eps;          // rounding margin of the staging radius
  int ncells;
  int* work;          // [0] work counter, [2..3] candidates, [5] the dense cells' work counter (zeroed
                      // by the launcher); [6] list length, [7] dense cells (written by k_hood_list)
  int* list;          // cells the neighbourhood sweep takes (ncells capacity)
  unsigned long long* cand;  // candidate pairs evaluated (work[2..3] of the same buffer), zeroed by the launcher
  unsigned char* flag;       // per cell: 1 per-particle companion sweep, 2 dense-cell sweep
  int* dense;                // cells of the dense-cell sweep (ncells capacity)
  int* ndense;               // their number (work[7])
  float hrow[9];             // lattice rows H (FP32): lattice image T maps to the shift T.H
  float4* hforce;            // half-shell path: per sorted particle, accumulated force (n entries)
  const float4* xl;          // per original particle: local coordinate, w = packed cell (binning output)
  const int* slot;           // per original particle: position inside its cell
  int half;                  // 1 when the half-shell path is tried for this launch
  // scalar reductions of the staged half-shell sweep (launch_hood_scalar)
  unsigned long long* count;  // pair count, added to
  unsigned long long* hist;   // nbins counts of r in [0, rmax), added to
  int nbins;
  float rmax, hscale;         // hscale = nbins / rmax
  float hxlim;                // min(nbins, rc hscale): bin coordinate limit of counted pairs
  int hcopies, hstride;       // shared-memory copies of the histogram (a power of two) and their stride
};
int fill_hood_args(const Geo& geo, const int* opk_full, int noff_full, const int* opk_half, int noff_half,
                   HoodArgs* H);
size_t hood_smem_bytes();
// mode 0: energy, forces, virial; 1: backward; 2: energy (half shell, A = half
// stencil); 3: energy and the backward outputs.
// partials_cap: doubles available in partials (sweep_partials_needed).
// lists_half (host, may be null): 1 when the list buffers (list, dense, flag,
// work[6..7]) hold the half-shell work lists of the current cell list; they
// are then reused, and the flag is set after a half-shell launch and cleared
// by any other.
// Ahalf (modes 0, 1, 3; may be null): the half stencil, for the half-shell
// path, taken when both stencils fit the kernels' table (H.hforce must then
// hold n entries); the full-shell kernels take the launch otherwise.
bool half_path_applies(const SweepArgs& A, const SweepArgs* Ahalf, const HoodArgs& H, int mode);
int launch_hood(const SweepArgs& A, const SweepArgs* Ahalf, const HoodArgs& H, int* work, int mode, const double* hinv, float* forces,
                double* grad, const double* gE, const double* pos, double* partials, long long partials_cap,
                double* sums, double* energy, double* virial, double* gradbox, cudaStream_t s,
                int* lists_half = nullptr);

// Count (kind 0), sum 1/r (1), distance histogram (2) or shifted-force
// energy (3) over the half stencil (A = half stencil, 3D): the staged sweeps
// (home-major for the fast-path cells, the windowed half-shell sweep for the
// others), or, when the stencil does not fit the kernels' table, the staged
// sweep for the cells that fit it and the per-particle sweep for the rest
// (the energy then returns CL_ERR_UNSUPPORTED: launch_hood's mode 2 takes it).
// The outputs (count: 1 value, scalar_out: 1 value, hist: nbins values) are
// overwritten.
bool hood_half_fits(const SweepArgs& A);
int launch_hood_scalar(const SweepArgs& A, const HoodArgs& H, int* work, int kind, unsigned long long* count,
                       double* partials, long long partials_cap, double* sums, double* scalar_out, int nbins,
                       float rmax, unsigned long long* hist, cudaStream_t s, int* lists_half = nullptr);

// Two sets (cl_cross.cu): what 0 counts per query (count may be null) and their
// total, 1 fills the pairs of each query's segment (start), 2 the per-query k
// nearest. err: device error latch.
int launch_cross(int what, const SweepArgs& A, const Geo& g, const double* posb, long long nb, int k, int* count,
                 unsigned long long* total, const long long* start, int* pa, int* pb, float* pd, int* knn_a, float* knn_d,
                 int* err, cudaStream_t s);
int launch_topk_merge(const int* la, const float* ld, long long nb, int k, int* oa, int* ob, float* od, int* found,
                      cudaStream_t s);

// Neighbour list (cl_pairs.cu). count[n] (int: one particle's pairs), start[n+1]
// (64-bit scan of count: the list may pass 2^31 pairs), tiles, meta:
// workspace; outputs pair_i/j/d of capacity entries.
constexpr int kMaxSegment = 1024;  // segments up to this length are sorted by one warp in shared memory
// Count pass of the pair list: per-cell staged sweep, then the per-particle
// sweep for the cells it flags (flag: ncells bytes; fcells: ncells ints, the
// flagged cells, *nfcells of them; all written here).
// cap: staged entries per cell (32..3072), the same for the count and fill passes.
int launch_pairs_count(const SweepArgs& A, int dim, float ball2, int cap, unsigned char* flag, int* fcells,
                       int* nfcells, int* count, cudaStream_t s);
// Sorts each segment [start[a], start[a] + count[a]) of pj (carrying pd) by pj;
// longs (n ints) and nlong (1 int) are workspace.
int launch_pairs_sort(int n, const int* count, const long long* start, int* pj, float* pd, int* longs, int* nlong,
                      cudaStream_t s);
// Fill pass: the same two sweeps, each segment sorted by j and written.
// longs (n ints) and nlong (1 int): workspace for segments longer than kMaxSegment.
int launch_pairs_fill(const SweepArgs& A, int dim, float ball2, int cap, const unsigned char* flag, const int* fcells,
                      const int* nfcells, const int* count, const long long* start, int* pi, int* pj, float* pd, int* longs,
                      int* nlong, cudaStream_t s);

}  // namespace clk
