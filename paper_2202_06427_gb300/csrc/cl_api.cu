// cl_api.cu -- the extern "C" boundary (cellmap.h): handle lifecycle,
// argument checks, and dispatch of the binning, sweep and reduction kernels.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "cl_internal.cuh"

struct cl_list {
  clk::Geo geo;
  int n;
  const double* pos;
  long long ncells_alloc;
  // device workspace
  int* slot;
  float4* xl;
  float4* xs;
  unsigned* cellc;
  int* counts;
  int* cell_start;
  unsigned char* hflag;  // per cell: 1 when a staged sweep (neighbourhood or pair list) leaves it to a per-particle sweep
  int* hlist;            // cells the neighbourhood sweep takes
  int* hdense;           // cells the dense-cell sweep takes
  int* tile_sum;
  int* meta;
  double* partials;
  double* sums;
  int* work;  // work counters of the persistent neighbourhood sweeps
  float4* hforce;  // per sorted particle: forces accumulated by the half-shell sweep (kept zero between launches)
  int last_half;   // the last 3D energy/force sweep took the half-shell path
  int lists_half;  // hlist / hdense / work[6..7] hold the half-shell work lists of the current cell list
  unsigned long long* u64;
  // neighbour-list workspace, allocated on the first CL_RED_PAIRLIST call
  int* pl_count;
  long long* pl_start;  // 64-bit: a list may pass 2^31 pairs
  long long* pl_tiles;
  int* pl_meta;
  int* pl_long;  // particles whose segments are sorted by the long-segment pass
  // device copies of the stencils (for sweeps compiled outside the library)
  clk::Off* d_off_half;
  clk::Off* d_off_full;
  // stencils (host copies of the sweep arguments)
  clk::SweepArgs* half;
  clk::SweepArgs* full;
  clk::HoodArgs* hood;  // 3D neighbourhood sweep arguments
  size_t bytes;
};

namespace {

template <class T>
int dev_alloc(T** p, size_t count, size_t* bytes) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return CL_ERR_OOM;
  }
  *bytes += sizeof(T) * count;
  return CL_OK;
}

void free_cells(cl_list* c) {
  cudaFree(c->counts);
  cudaFree(c->cell_start);
  cudaFree(c->tile_sum);
  cudaFree(c->hflag);
  cudaFree(c->hlist);
  c->hlist = nullptr;
  cudaFree(c->hdense);
  c->hdense = nullptr;
  c->counts = nullptr;
  c->cell_start = nullptr;
  c->tile_sum = nullptr;
  c->hflag = nullptr;
}

void free_all(cl_list* c) {
  free_cells(c);
  cudaFree(c->slot);
  cudaFree(c->xl);
  cudaFree(c->xs);
  cudaFree(c->cellc);
  cudaFree(c->meta);
  cudaFree(c->partials);
  cudaFree(c->sums);
  cudaFree(c->work);
  cudaFree(c->hforce);
  cudaFree(c->u64);
  cudaFree(c->d_off_half);
  cudaFree(c->d_off_full);
  cudaFree(c->pl_count);
  cudaFree(c->pl_start);
  cudaFree(c->pl_tiles);
  cudaFree(c->pl_meta);
  cudaFree(c->pl_long);
  delete c->half;
  delete c->full;
  delete c->hood;
}

int alloc_cells(cl_list* c, long long ncells) {
  size_t b = 0;
  int e;
  if ((e = dev_alloc(&c->counts, (size_t)ncells, &b))) return e;
  if ((e = dev_alloc(&c->cell_start, (size_t)ncells + 1, &b))) return e;
  if ((e = dev_alloc(&c->tile_sum, (size_t)clk::scan_tiles_for(ncells), &b))) return e;
  if ((e = dev_alloc(&c->hflag, (size_t)ncells, &b))) return e;
  if ((e = dev_alloc(&c->hlist, (size_t)ncells, &b))) return e;
  if ((e = dev_alloc(&c->hdense, (size_t)ncells, &b))) return e;
  c->ncells_alloc = ncells;
  c->bytes += b;
  return CL_OK;
}

// Partials (doubles) available to the neighbourhood sweep and its per-particle companion.
long long hood_cap(const cl_list* c) { return clk::sweep_partials_needed(c->n); }

// Count, sum 1/r and the histogram take the staged neighbourhood sweep when
// the cells hold enough particles on average to pay for staging the half
// neighbourhood once per cell (measured: 23 per cell on the 1M lattice runs
// the count in 0.57 ms staged against 0.75 ms per particle), else one thread
// per particle over the stencil.
constexpr double kStagedMinOccupancy = 16.0;
bool scalar_staged(const cl_list* c) {
  return c->geo.dim == 3 && c->n > 0 && (double)c->n >= kStagedMinOccupancy * (double)c->geo.ncells;
}

void fill_sweep_args(cl_list* c, clk::SweepArgs* A) {
  A->xs = c->xs;
  A->cellc = c->cellc;
  A->cell_start = c->cell_start;
  A->n = c->n;
  A->nx = c->geo.n[0];
  A->ny = c->geo.n[1];
  A->nz = c->geo.n[2];
  A->rc2 = (float)(c->geo.rc * c->geo.rc);
  A->irc = (float)(1.0 / c->geo.rc);
  A->irc2 = (float)(1.0 / (c->geo.rc * c->geo.rc));
  float e[3];
  clk::cell_halfwidths(c->geo, e);
  A->ex = e[0];
  A->ey = e[1];
  A->ez = e[2];
}

int set_geometry(cl_list* c, const cl_box* box) {
  clk::Geo g;
  int e = clk::prepare_geometry(box, &g);
  if (e) return e;
  clk::Off* th = new (std::nothrow) clk::Off[2 * clk::kMaxOff];
  int* opk = new (std::nothrow) int[2 * clk::kMaxOff];
  clk::HoodArgs* hood = new (std::nothrow) clk::HoodArgs;
  if (!th || !opk || !hood) {
    delete[] th;
    delete[] opk;
    delete hood;
    return CL_ERR_OOM;
  }
  clk::Off* tf = th + clk::kMaxOff;
  int nh = clk::build_stencil(g, 1, th, clk::kMaxOff, opk + clk::kMaxOff);
  int nf = nh < 0 ? nh : clk::build_stencil(g, 0, tf, clk::kMaxOff, opk);
  if (nh < 0 || nf < 0) {
    delete[] th;
    delete[] opk;
    delete hood;
    return nh < 0 ? nh : nf;
  }
  std::memset(hood, 0, sizeof(*hood));
  if (g.dim == 3) clk::fill_hood_args(g, opk, nf, opk + clk::kMaxOff, nh, hood);
  delete[] opk;
  if (g.ncells != c->ncells_alloc) {
    free_cells(c);
    if ((e = alloc_cells(c, g.ncells))) {
      delete[] th;
      delete hood;
      return e;
    }
  }
  std::memcpy(c->half->off, th, sizeof(clk::Off) * nh);
  std::memcpy(c->full->off, tf, sizeof(clk::Off) * nf);
  if (cudaMemcpy(c->d_off_half, th, sizeof(clk::Off) * nh, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_off_full, tf, sizeof(clk::Off) * nf, cudaMemcpyHostToDevice) != cudaSuccess) {
    delete[] th;
    delete hood;
    return CL_ERR_CUDA;
  }
  *c->hood = *hood;
  c->hood->flag = c->hflag;
  c->hood->list = c->hlist;
  c->hood->dense = c->hdense;
  c->hood->hforce = c->hforce;
  c->hood->xl = c->xl;
  c->hood->slot = c->slot;
  delete hood;
  c->half->noff = nh;
  c->full->noff = nf;
  delete[] th;
  c->geo = g;
  fill_sweep_args(c, c->half);
  fill_sweep_args(c, c->full);
  return CL_OK;
}

int run_build(cl_list* c, cudaStream_t s) {
  clk::BuildBufs b;
  b.pos = c->pos;
  b.n = c->n;
  b.slot = c->slot;
  c->lists_half = 0;  // new cell contents: the sweeps' work lists are rebuilt
  b.xl = c->xl;
  b.counts = c->counts;
  b.cell_start = c->cell_start;
  b.tile_sum = c->tile_sum;
  b.meta = c->meta;
  b.xs = c->xs;
  b.cellc = c->cellc;
  return clk::launch_build(c->geo, b, s);
}

// Squared radius about a cell's centre that holds every particle within rc of
// a point of the cell: (rc + half the longest cell diagonal + a margin)^2.
float pairs_ball2(const clk::Geo& g) {
  double hd = 0.0;
  for (int corner = 0; corner < (1 << g.dim); ++corner) {
    double v[3] = {0, 0, 0};
    for (int k = 0; k < g.dim; ++k) {
      const double sg = ((corner >> k) & 1) ? 0.5 : -0.5;
      for (int a = 0; a < g.dim; ++a) v[a] += sg * g.h[k * 3 + a] / g.n[k];
    }
    hd = std::max(hd, std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
  }
  const double r = g.rc + hd * (1.0 + 1e-6) + 1e-4 * (g.rc + hd);
  return (float)(r * r);
}

// Staged entries per cell for the pair list: the particles of the staging ball
// at the box's mean density, with 30 % to spare, in steps of 128 (1,024 to
// 3,072). Denser cells overflow and take the per-particle path.
int pairs_stage_cap(const clk::Geo& g, long long n, float ball2) {
  double vol = 1.0;
  if (g.dim == 3)
    vol = std::fabs(g.h[0] * (g.h[4] * g.h[8] - g.h[5] * g.h[7]) - g.h[1] * (g.h[3] * g.h[8] - g.h[5] * g.h[6]) +
                    g.h[2] * (g.h[3] * g.h[7] - g.h[4] * g.h[6]));
  else
    vol = std::fabs(g.h[0] * g.h[4] - g.h[1] * g.h[3]);
  const double r = std::sqrt((double)ball2);
  const double ball = g.dim == 3 ? 4.18879020478639 * r * r * r : 3.14159265358979 * r * r;
  const double est = (vol > 0 ? (double)n / vol : 0.0) * ball * 1.3 + 64.0;
  int cap = (int)std::ceil(est / 128.0) * 128;
  return std::min(3072, std::max(1024, cap));
}

// Neighbour list: count pass, scan, one synchronisation to learn the total,
// fill pass (each segment sorted as it is written).
int map_pairlist(cl_list* c, cl_result* r, cudaStream_t s) {
  if (!r->npairs || r->capacity < 0) return CL_ERR_INVALID_ARG;
  for (int k = 0; k < c->geo.dim; ++k)
    if (!(2.0 * c->geo.rc <= c->geo.w[k])) return CL_ERR_CUTOFF_TOO_LARGE;  // unique images only
  int e;
  if (!c->pl_count) {
    size_t b = 0;
    const size_t n = (size_t)c->n;
    if ((e = dev_alloc(&c->pl_count, n, &b)) || (e = dev_alloc(&c->pl_start, n + 1, &b)) ||
        (e = dev_alloc(&c->pl_tiles, (size_t)clk::scan_tiles_for(c->n), &b)) || (e = dev_alloc(&c->pl_meta, 8, &b)) ||
        (e = dev_alloc(&c->pl_long, n, &b))) {
      cudaFree(c->pl_count);
      cudaFree(c->pl_start);
      cudaFree(c->pl_tiles);
      cudaFree(c->pl_meta);
      cudaFree(c->pl_long);
      c->pl_count = c->pl_meta = c->pl_long = nullptr;
      c->pl_start = c->pl_tiles = nullptr;
      return e;
    }
    c->bytes += b;
  }
  const int dim = c->geo.dim;
  const float ball2 = pairs_ball2(c->geo);
  // hflag / hlist: per-cell flags and the flagged cells (shared with the
  // neighbourhood sweep, which rewrites them on every launch); pl_meta[4]: their number
  const int cap = pairs_stage_cap(c->geo, c->n, ball2);
  c->lists_half = 0;  // the pair list's passes use the list buffers
  if ((e = clk::launch_pairs_count(*c->full, dim, ball2, cap, c->hflag, c->hlist, c->pl_meta + 4, c->pl_count, s)))
    return e;
  if ((e = clk::launch_scan64(c->pl_count, c->n, c->pl_tiles, c->pl_start, c->pl_meta, s))) return e;
  long long total = 0;
  int meta[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(&total, c->pl_start + c->n, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(meta, c->pl_meta, sizeof(meta), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CL_ERR_CUDA;
  *r->npairs = total;
  if ((e = cl_pairlist_fits(total, r->capacity))) return e;
  if (total == 0) return CL_OK;
  if (!r->pair_i || !r->pair_j || !r->pair_d) return CL_ERR_INVALID_ARG;
  return clk::launch_pairs_fill(*c->full, dim, ball2, cap, c->hflag, c->hlist, c->pl_meta + 4, c->pl_count, c->pl_start,
                               r->pair_i, r->pair_j, r->pair_d, c->pl_long, c->pl_meta + 3, s);
}

}  // namespace

extern "C" {

int cl_pairlist_fits(long long npairs, long long capacity) {
  if (npairs < 0) return CL_ERR_INVALID_ARG;  // a total read back from the 64-bit scan is never negative
  return npairs > capacity ? CL_ERR_CAPACITY : CL_OK;
}

const char* cl_error_string(int code) {
  switch (code) {
    case CL_OK: return "ok";
    case CL_ERR_INVALID_ARG: return "invalid argument";
    case CL_ERR_INVALID_BOX: return "singular or non-finite box matrix";
    case CL_ERR_CUTOFF_TOO_LARGE: return "cutoff too large for the box";
    case CL_ERR_NONFINITE: return "non-finite position";
    case CL_ERR_OOM: return "device out of memory";
    case CL_ERR_CAPACITY: return "pair list capacity exceeded";
    case CL_ERR_TIMEOUT: return "device wait timed out";
    case CL_ERR_CUDA: return "CUDA runtime error";
    case CL_ERR_UNSUPPORTED: return "grid or stencil beyond library limits";
    default: return "unknown error";
  }
}

int cl_box_info(const cl_box* box, long long* grid, double* widths, long long* stencil) {
  if (!box) return CL_ERR_INVALID_ARG;
  clk::Geo g;
  int e = clk::prepare_geometry(box, &g);
  if (e) return e;
  clk::Off* tmp = new (std::nothrow) clk::Off[clk::kMaxOff];
  if (!tmp) return CL_ERR_OOM;
  int nh = clk::build_stencil(g, 1, tmp, clk::kMaxOff);
  int nf = clk::build_stencil(g, 0, tmp, clk::kMaxOff);
  delete[] tmp;
  if (nh < 0) return nh;
  if (nf < 0) return nf;
  for (int k = 0; k < 3; ++k) {
    if (grid) grid[k] = g.n[k];
    if (widths) widths[k] = k < g.dim ? g.w[k] : 0.0;
  }
  if (stencil) {
    stencil[0] = nh;
    stencil[1] = nf;
  }
  return CL_OK;
}

int cl_build(const double* pos_dev, long long n, const cl_box* box, void* stream, cl_list** out) {
  if (!out || !box || n < 0 || n >= 2147483647LL || (n > 0 && !pos_dev)) return CL_ERR_INVALID_ARG;
  *out = nullptr;
  cl_list* c = new (std::nothrow) cl_list;
  if (!c) return CL_ERR_OOM;
  std::memset(c, 0, sizeof(*c));
  c->half = new (std::nothrow) clk::SweepArgs;
  c->full = new (std::nothrow) clk::SweepArgs;
  c->hood = new (std::nothrow) clk::HoodArgs;
  if (!c->half || !c->full || !c->hood) {
    free_all(c);
    delete c;
    return CL_ERR_OOM;
  }
  std::memset(c->half, 0, sizeof(clk::SweepArgs));
  std::memset(c->full, 0, sizeof(clk::SweepArgs));
  c->n = (int)n;
  c->pos = pos_dev;
  c->ncells_alloc = -1;
  int e = CL_OK;
  size_t b = 0;
  const size_t nn = (size_t)n;
  if (!e) e = dev_alloc(&c->slot, nn, &b);
  if (!e) e = dev_alloc(&c->xl, nn, &b);
  if (!e) e = dev_alloc(&c->xs, nn, &b);
  if (!e) e = dev_alloc(&c->cellc, nn, &b);
  if (!e) e = dev_alloc(&c->meta, 4, &b);
  if (!e) e = dev_alloc(&c->partials, (size_t)clk::sweep_partials_needed(c->n), &b);
  if (!e) e = dev_alloc(&c->sums, 32, &b);
  if (!e) e = dev_alloc(&c->work, 8, &b);  // [0] work counter, [2..3] candidate counter, [5] the dense
                                           // cells' work counter, [6] list length, [7] dense cells
  if (!e && box->dim == 3) e = dev_alloc(&c->hforce, nn, &b);
  if (!e && box->dim == 3 && nn > 0 && cudaMemset(c->hforce, 0, sizeof(float4) * nn) != cudaSuccess) e = CL_ERR_CUDA;
  if (!e) e = dev_alloc(&c->u64, 8, &b);
  if (!e) e = dev_alloc(&c->d_off_half, (size_t)clk::kMaxOff, &b);
  if (!e) e = dev_alloc(&c->d_off_full, (size_t)clk::kMaxOff, &b);
  c->bytes = b;
  if (!e) e = set_geometry(c, box);
  cudaStream_t s = (cudaStream_t)stream;
  if (!e && cudaMemsetAsync(c->meta, 0, sizeof(int) * 4, s) != cudaSuccess) e = CL_ERR_CUDA;
  // sums[31]: the final reduction's completion counter, zero between launches
  if (!e && cudaMemsetAsync(c->sums, 0, sizeof(double) * 32, s) != cudaSuccess) e = CL_ERR_CUDA;
  if (!e) e = run_build(c, s);
  if (e) {
    free_all(c);
    delete c;
    return e;
  }
  *out = c;
  return CL_OK;
}

int cl_update(cl_list* c, const double* pos_dev, const cl_box* box, void* stream) {
  if (!c || (c->n > 0 && !pos_dev)) return CL_ERR_INVALID_ARG;
  if (box) {
    int e = set_geometry(c, box);
    if (e) return e;
  }
  c->pos = pos_dev;
  return run_build(c, (cudaStream_t)stream);
}

int cl_map(const cl_list* cc, cl_reduction red, const cl_params* params, cl_result* r, void* stream) {
  if (!cc || !r) return CL_ERR_INVALID_ARG;
  cl_list* c = const_cast<cl_list*>(cc);
  cudaStream_t s = (cudaStream_t)stream;
  const int dim = c->geo.dim;
  switch (red) {
    case CL_RED_COUNT:
      if (!r->count) return CL_ERR_INVALID_ARG;
      if (scalar_staged(c))
        return clk::launch_hood_scalar(*c->half, *c->hood, c->work, 0, r->count, c->partials, hood_cap(c), c->sums,
                                       nullptr, 0, 0.f, nullptr, s, &c->lists_half);
      return clk::launch_count(*c->half, dim, r->count, s);
    case CL_RED_SUM_INV_R:
      if (!r->sum_inv_r) return CL_ERR_INVALID_ARG;
      if (scalar_staged(c))
        return clk::launch_hood_scalar(*c->half, *c->hood, c->work, 1, nullptr, c->partials, hood_cap(c), c->sums,
                                       r->sum_inv_r, 0, 0.f, nullptr, s, &c->lists_half);
      return clk::launch_scalar(*c->half, dim, 0, c->partials, c->sums, r->sum_inv_r, s);
    case CL_RED_SF_ENERGY:
      if (!r->energy) return CL_ERR_INVALID_ARG;
      if (dim == 3 && c->n > 0 && clk::hood_half_fits(*c->half))
        return clk::launch_hood_scalar(*c->half, *c->hood, c->work, 3, nullptr, c->partials, hood_cap(c), c->sums,
                                       r->energy, 0, 0.f, nullptr, s, &c->lists_half);
      if (dim == 3 && c->n > 0)
        return clk::launch_hood(*c->half, nullptr, *c->hood, c->work, 2, c->geo.hinv, nullptr, nullptr, nullptr, nullptr,
                                c->partials, hood_cap(c), c->sums, r->energy, nullptr, nullptr, s, &c->lists_half);
      return clk::launch_scalar(*c->half, dim, 1, c->partials, c->sums, r->energy, s);
    case CL_RED_SF_ENERGY_FORCES_VIRIAL:
      if (!r->forces && c->n > 0) return CL_ERR_INVALID_ARG;
      if (dim == 3 && c->n > 0) {
        c->last_half = clk::half_path_applies(*c->full, c->half, *c->hood, 0) ? 1 : 0;
        return clk::launch_hood(*c->full, c->half, *c->hood, c->work, 0, c->geo.hinv, r->forces, nullptr, nullptr, nullptr,
                                c->partials, hood_cap(c), c->sums, r->energy, r->virial, nullptr, s, &c->lists_half);
      }
      return clk::launch_force(*c->full, dim, 0, c->geo.hinv, r->forces, nullptr, nullptr, nullptr, c->partials,
                               c->sums, r->energy, r->virial, nullptr, s);
    case CL_RED_HIST: {
      if (!params || !r->hist || params->nbins < 1 || params->nbins > clk::kMaxBins) return CL_ERR_INVALID_ARG;
      double rmax = params->rmax > 0 ? params->rmax : c->geo.rc;
      if (scalar_staged(c))
        return clk::launch_hood_scalar(*c->half, *c->hood, c->work, 2, nullptr, c->partials, hood_cap(c), c->sums,
                                       nullptr, params->nbins, (float)rmax, r->hist, s, &c->lists_half);
      return clk::launch_hist(*c->half, dim, params->nbins, (float)rmax, r->hist, s);
    }
    case CL_RED_PAIRLIST:
      return map_pairlist(c, r, s);
    default:
      return CL_ERR_INVALID_ARG;
  }
}

int cl_backward(const cl_list* cc, const double* grad_energy_dev, double* grad_pos_dev, double* grad_box_dev,
                double* virial_dev, void* stream) {
  if (!cc || !grad_energy_dev || (cc->n > 0 && !grad_pos_dev)) return CL_ERR_INVALID_ARG;
  cl_list* c = const_cast<cl_list*>(cc);
  if (c->geo.dim == 3 && c->n > 0) {
    c->last_half = clk::half_path_applies(*c->full, c->half, *c->hood, 1) ? 1 : 0;
    return clk::launch_hood(*c->full, c->half, *c->hood, c->work, 1, c->geo.hinv, nullptr, grad_pos_dev, grad_energy_dev,
                            c->pos, c->partials, hood_cap(c), c->sums, nullptr, virial_dev, grad_box_dev,
                            (cudaStream_t)stream, &c->lists_half);
  }
  return clk::launch_force(*c->full, c->geo.dim, 1, c->geo.hinv, nullptr, grad_pos_dev, grad_energy_dev, c->pos,
                           c->partials, c->sums, nullptr, virial_dev, grad_box_dev, (cudaStream_t)stream);
}

int cl_energy_grad(const cl_list* cc, const double* scale_dev, double* energy_dev, double* grad_pos_dev,
                   double* grad_box_dev, double* virial_dev, void* stream) {
  if (!cc || !scale_dev || !energy_dev || (cc->n > 0 && !grad_pos_dev)) return CL_ERR_INVALID_ARG;
  cl_list* c = const_cast<cl_list*>(cc);
  cudaStream_t s = (cudaStream_t)stream;
  if (c->geo.dim == 3 && c->n > 0) {
    c->last_half = clk::half_path_applies(*c->full, c->half, *c->hood, 3) ? 1 : 0;
    return clk::launch_hood(*c->full, c->half, *c->hood, c->work, 3, c->geo.hinv, nullptr, grad_pos_dev, scale_dev, c->pos,
                            c->partials, hood_cap(c), c->sums, energy_dev, virial_dev, grad_box_dev, s,
                            &c->lists_half);
  }
  // 2D (and the empty list): the energy sweep, then the backward sweep
  int e = clk::launch_scalar(*c->half, c->geo.dim, 1, c->partials, c->sums, energy_dev, s);
  if (e) return e;
  return clk::launch_force(*c->full, c->geo.dim, 1, c->geo.hinv, nullptr, grad_pos_dev, scale_dev, c->pos,
                           c->partials, c->sums, nullptr, virial_dev, grad_box_dev, s);
}

int cl_scale(const double* scale_dev, const double* in_dev, double* out_dev, long long count, void* stream) {
  if (count < 0 || (count > 0 && (!scale_dev || !in_dev || !out_dev))) return CL_ERR_INVALID_ARG;
  return clk::launch_scale(scale_dev, in_dev, out_dev, count, (cudaStream_t)stream);
}

// ---- two sets: queries of set B against the cell list of set A
namespace {

int check_query(const cl_list* c, const double* posb, long long nb) {
  if (!c || nb < 0 || nb >= 2147483647LL || (nb > 0 && !posb)) return CL_ERR_INVALID_ARG;
  return CL_OK;
}

// Per-call workspace of the two-set queries (allocated and freed here).
struct QueryWs {
  int* count = nullptr;
  long long* start = nullptr;  // 64-bit offsets of the cross list
  long long* tiles = nullptr;
  int* meta = nullptr;
  int* err = nullptr;
  int* longs = nullptr;
  unsigned long long* total = nullptr;
  ~QueryWs() {
    cudaFree(longs);
    cudaFree(count);
    cudaFree(start);
    cudaFree(tiles);
    cudaFree(meta);
    cudaFree(err);
    cudaFree(total);
  }
};

int read_err(const int* err_dev, cudaStream_t s) {
  int v = 0;
  if (cudaMemcpyAsync(&v, err_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CL_ERR_CUDA;
  return v ? CL_ERR_NONFINITE : CL_OK;
}

}  // namespace

int cl_cross_count(const cl_list* cc, const double* posb_dev, long long nb, unsigned long long* count_dev,
                   void* stream) {
  int e = check_query(cc, posb_dev, nb);
  if (e || !count_dev) return e ? e : CL_ERR_INVALID_ARG;
  cl_list* c = const_cast<cl_list*>(cc);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(count_dev, 0, sizeof(unsigned long long), s) != cudaSuccess) return CL_ERR_CUDA;
  size_t b = 0;
  QueryWs w;
  if ((e = dev_alloc(&w.err, 1, &b))) return e;
  if (cudaMemsetAsync(w.err, 0, sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  if ((e = clk::launch_cross(0, *c->full, c->geo, posb_dev, nb, 0, nullptr, count_dev, nullptr, nullptr, nullptr,
                             nullptr, nullptr, nullptr, w.err, s)))
    return e;
  return read_err(w.err, s);
}

int cl_cross_pairlist(const cl_list* cc, const double* posb_dev, long long nb, long long capacity, int* pa_dev,
                      int* pb_dev, float* pd_dev, long long* npairs, void* stream) {
  int e = check_query(cc, posb_dev, nb);
  if (e || !npairs || capacity < 0) return e ? e : CL_ERR_INVALID_ARG;
  cl_list* c = const_cast<cl_list*>(cc);
  for (int k = 0; k < c->geo.dim; ++k)
    if (!(2.0 * c->geo.rc <= c->geo.w[k])) return CL_ERR_CUTOFF_TOO_LARGE;  // unique images only
  cudaStream_t s = (cudaStream_t)stream;
  *npairs = 0;
  if (nb == 0) return CL_OK;
  size_t b = 0;
  QueryWs w;
  if ((e = dev_alloc(&w.count, (size_t)nb, &b)) || (e = dev_alloc(&w.start, (size_t)nb + 1, &b)) ||
      (e = dev_alloc(&w.tiles, (size_t)clk::scan_tiles_for(nb), &b)) || (e = dev_alloc(&w.meta, 4, &b)) ||
      (e = dev_alloc(&w.err, 1, &b)) || (e = dev_alloc(&w.longs, (size_t)nb, &b)))
    return e;
  if (cudaMemsetAsync(w.err, 0, sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  if ((e = clk::launch_cross(0, *c->full, c->geo, posb_dev, nb, 0, w.count, nullptr, nullptr, nullptr, nullptr,
                             nullptr, nullptr, nullptr, w.err, s)))
    return e;
  if ((e = clk::launch_scan64(w.count, nb, w.tiles, w.start, w.meta, s))) return e;
  long long total = 0;
  int meta[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(&total, w.start + nb, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(meta, w.meta, sizeof(meta), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CL_ERR_CUDA;
  if ((e = read_err(w.err, s))) return e;
  *npairs = total;
  if ((e = cl_pairlist_fits(total, capacity))) return e;
  if (total == 0) return CL_OK;
  if (!pa_dev || !pb_dev || !pd_dev) return CL_ERR_INVALID_ARG;
  if ((e = clk::launch_cross(1, *c->full, c->geo, posb_dev, nb, 0, nullptr, nullptr, w.start, pa_dev, pb_dev, pd_dev,
                             nullptr, nullptr, w.err, s)))
    return e;
  if ((e = clk::launch_pairs_sort((int)nb, w.count, w.start, pa_dev, pd_dev, w.longs, w.meta + 3, s))) return e;
  return cudaStreamSynchronize(s) == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int cl_cross_knn(const cl_list* cc, const double* posb_dev, long long nb, int k, int* knn_a_dev, float* knn_d_dev,
                 void* stream) {
  int e = check_query(cc, posb_dev, nb);
  if (e || k < 1 || k > CL_KNN_MAX || (nb > 0 && (!knn_a_dev || !knn_d_dev))) return e ? e : CL_ERR_INVALID_ARG;
  cl_list* c = const_cast<cl_list*>(cc);
  cudaStream_t s = (cudaStream_t)stream;
  if (nb == 0) return CL_OK;
  size_t b = 0;
  QueryWs w;
  if ((e = dev_alloc(&w.err, 1, &b))) return e;
  if (cudaMemsetAsync(w.err, 0, sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  if ((e = clk::launch_cross(2, *c->full, c->geo, posb_dev, nb, k, nullptr, nullptr, nullptr, nullptr, nullptr,
                             nullptr, knn_a_dev, knn_d_dev, w.err, s)))
    return e;
  return read_err(w.err, s);
}

int cl_cross_topk(const cl_list* cc, const double* posb_dev, long long nb, int k, int* a_dev, int* b_dev,
                  float* d_dev, long long* nfound, void* stream) {
  int e = check_query(cc, posb_dev, nb);
  if (e || k < 1 || k > CL_KNN_MAX || !a_dev || !b_dev || !d_dev || !nfound) return e ? e : CL_ERR_INVALID_ARG;
  cl_list* c = const_cast<cl_list*>(cc);
  cudaStream_t s = (cudaStream_t)stream;
  *nfound = 0;
  size_t b = 0;
  QueryWs w;
  int* la = nullptr;
  float* ld = nullptr;
  const size_t m = (size_t)(nb > 0 ? nb : 1) * k;
  if ((e = dev_alloc(&w.err, 2, &b)) || (e = dev_alloc(&la, m, &b)) || (e = dev_alloc(&ld, m, &b))) {
    cudaFree(la);
    cudaFree(ld);
    return e;
  }
  if (cudaMemsetAsync(w.err, 0, 2 * sizeof(int), s) != cudaSuccess) e = CL_ERR_CUDA;
  if (!e && nb > 0)
    e = clk::launch_cross(2, *c->full, c->geo, posb_dev, nb, k, nullptr, nullptr, nullptr, nullptr, nullptr,
                          nullptr, la, ld, w.err, s);
  if (!e) e = clk::launch_topk_merge(la, ld, nb, k, a_dev, b_dev, d_dev, w.err + 1, s);
  int found = 0;
  if (!e && cudaMemcpyAsync(&found, w.err + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    e = CL_ERR_CUDA;
  if (!e) e = read_err(w.err, s);
  cudaFree(la);
  cudaFree(ld);
  if (!e) *nfound = found;
  return e;
}

int cl_query(const cl_list* c, int what, long long* value, void* stream) {
  if (!c || !value) return CL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  switch (what) {
    case CL_INFO_N: *value = c->n; return CL_OK;
    case CL_INFO_DIM: *value = c->geo.dim; return CL_OK;
    case CL_INFO_GRID_X: *value = c->geo.n[0]; return CL_OK;
    case CL_INFO_GRID_Y: *value = c->geo.n[1]; return CL_OK;
    case CL_INFO_GRID_Z: *value = c->geo.n[2]; return CL_OK;
    case CL_INFO_NCELLS: *value = c->geo.ncells; return CL_OK;
    case CL_INFO_BYTES: *value = (long long)c->bytes; return CL_OK;
    case CL_INFO_STENCIL_HALF: *value = c->half->noff; return CL_OK;
    case CL_INFO_STENCIL_FULL: *value = c->full->noff; return CL_OK;
    case CL_INFO_WORK_TILES: *value = (c->n + 255) / 256; return CL_OK;
    case CL_INFO_NONEMPTY:
    case CL_INFO_MAX_OCCUPANCY: {
      int m[3];
      if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
      if (cudaMemcpy(m, c->meta, sizeof(m), cudaMemcpyDeviceToHost) != cudaSuccess) return CL_ERR_CUDA;
      *value = what == CL_INFO_NONEMPTY ? m[1] : m[2];
      return CL_OK;
    }
    case CL_INFO_SWEEP_HALF:
      *value = c->last_half;
      return CL_OK;
    case CL_INFO_SWEEP_CANDIDATES: {
      unsigned long long v = 0;
      if (cudaMemcpyAsync(&v, c->work + 2, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CL_ERR_CUDA;
      if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
      *value = (long long)v;
      return CL_OK;
    }
    case CL_INFO_CANDIDATES: {
      int e = clk::launch_candidates(*c->half, c->geo.ncells, c->u64, s);
      if (e) return e;
      unsigned long long v = 0;
      if (cudaMemcpyAsync(&v, c->u64, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CL_ERR_CUDA;
      if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
      *value = (long long)v;
      return CL_OK;
    }
    default: return CL_ERR_INVALID_ARG;
  }
}

int cl_get_view(const cl_list* c, cl_view* v) {
  if (!c || !v) return CL_ERR_INVALID_ARG;
  static_assert(sizeof(cl_offset) == sizeof(clk::Off), "public and internal stencil entries differ");
  v->dim = c->geo.dim;
  v->n = c->n;
  v->nx = c->geo.n[0];
  v->ny = c->geo.n[1];
  v->nz = c->geo.n[2];
  v->cutoff = (float)c->geo.rc;
  v->xs = c->xs;
  v->cellc = c->cellc;
  v->cell_start = c->cell_start;
  v->off_half = reinterpret_cast<const cl_offset*>(c->d_off_half);
  v->noff_half = c->half->noff;
  v->off_full = reinterpret_cast<const cl_offset*>(c->d_off_full);
  v->noff_full = c->full->noff;
  return CL_OK;
}

int cl_status(cl_list* c, void* stream) {
  if (!c) return CL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int flag = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
  if (cudaMemcpy(&flag, c->meta, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CL_ERR_CUDA;
  if (flag) {
    int zero = 0;
    if (cudaMemcpy(c->meta, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return CL_ERR_CUDA;
  }
  return (flag & clk::kErrNonFinite) ? CL_ERR_NONFINITE : CL_OK;
}

void cl_free(cl_list* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  free_all(c);
  delete c;
}

}  // extern "C"
