// cl_cross.cu -- pairs between two sets of particles (Sec. 3.2, Code 8: a cell
// list of x and a second set y; Sec. 4.1: neighbour lists between two sets).
// The cell list is the one of set A (cl_build); every particle b of set B is
// binned on A's grid like k_bin does (FP64 wrap and cell, FP32 coordinate
// relative to the cell centre) and sweeps the FULL stencil of its cell, the
// displacement to a being (xs_a + S_o) - x_b as in the one-set sweep. Every
// (a, b) pair-image within the cutoff is visited once; there is no a < b rule.
//
//   k_cross<COUNT>   per-b counts (and their sum)
//   k_cross<FILL>    writes (a, b, r) into b's segment of the list
//   k_cross_knn      per b the k nearest a within the cutoff (k <= 32)
//   k_topk_merge     the k smallest over all per-b lists (one CTA)
#include <cfloat>

#include "cl_sweep.cuh"

namespace clk {
namespace {

constexpr int kKnnMax = CL_KNN_MAX;

struct QueryArgs {
  const double* pos;  // (nb, dim) FP64
  long long nb;
  int dim, ortho;
  double m[9];        // t = x M (cell units)
  float g[9];         // cell edge vectors (rows)
};

// Cell and centred FP32 coordinate of query point b; false when not finite.
__device__ __forceinline__ bool bin_query(const SweepArgs& A, const QueryArgs& Q, long long b, int& cx, int& cy,
                                          int& cz, float& px, float& py, float& pz) {
  double x[3] = {0.0, 0.0, 0.0};
  bool finite = true;
  for (int k = 0; k < Q.dim; ++k) {
    x[k] = Q.pos[b * Q.dim + k];
    finite = finite && isfinite(x[k]);
  }
  if (!finite) return false;
  const int nk[3] = {A.nx, A.ny, A.nz};
  int c[3] = {0, 0, 0};
  float u[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < Q.dim; ++k) {
    double t;
    if (Q.ortho) {
      t = x[k] * Q.m[k * 3 + k];
    } else {
      t = 0.0;
      for (int q = 0; q < Q.dim; ++q) t = fma(x[q], Q.m[q * 3 + k], t);
    }
    const double f = floor(t);
    long long ci = (long long)f % nk[k];
    if (ci < 0) ci += nk[k];
    c[k] = (int)ci;
    u[k] = (float)(t - f) - 0.5f;
  }
  px = py = pz = 0.f;
  for (int k = 0; k < Q.dim; ++k) {
    px = fmaf(u[k], Q.g[k * 3 + 0], px);
    py = fmaf(u[k], Q.g[k * 3 + 1], py);
    pz = fmaf(u[k], Q.g[k * 3 + 2], pz);
  }
  cx = c[0];
  cy = c[1];
  cz = c[2];
  return true;
}

// Visits every a within the cutoff of query b: f(a_original, r^2).
template <class Fn>
__device__ __forceinline__ void query_sweep(const SweepArgs& A, int cx, int cy, int cz, float px, float py, float pz,
                                           Fn&& f) {
  for (int k = 0; k < A.noff; ++k) {
    const Off& o = A.off[k];
    const int c = stencil_cell(A, k, cx, cy, cz);
    const float sx = o.sx - px, sy = o.sy - py, sz = o.sz - pz;
    const int j1 = A.cell_start[c + 1];
    for (int j = A.cell_start[c]; j < j1; ++j) {
      const float4 q = __ldg(&A.xs[j]);
      const float dx = q.x + sx, dy = q.y + sy, dz = q.z + sz;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (d2 < A.rc2) f(__float_as_int(q.w), d2);
    }
  }
}

__global__ void __launch_bounds__(256) k_cross_count(const __grid_constant__ SweepArgs A,
                                                     const __grid_constant__ QueryArgs Q, int* __restrict__ count,
                                                     unsigned long long* __restrict__ total, int* __restrict__ err) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned n = 0;
  if (b < Q.nb) {
    int cx, cy, cz;
    float px, py, pz;
    if (bin_query(A, Q, b, cx, cy, cz, px, py, pz)) {
      query_sweep(A, cx, cy, cz, px, py, pz, [&](int, float) { ++n; });
    } else {
      atomicOr(err, kErrNonFinite);
    }
    if (count) count[b] = (int)n;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n && total) atomicAdd(total, (unsigned long long)n);
}

__global__ void __launch_bounds__(256) k_cross_fill(const __grid_constant__ SweepArgs A,
                                                    const __grid_constant__ QueryArgs Q, const long long* __restrict__ start,
                                                    int* __restrict__ pa, int* __restrict__ pb,
                                                    float* __restrict__ pd) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= Q.nb) return;
  int cx, cy, cz;
  float px, py, pz;
  if (!bin_query(A, Q, b, cx, cy, cz, px, py, pz)) return;
  long long pos = start[b];
  query_sweep(A, cx, cy, cz, px, py, pz, [&](int a, float d2) {
    pa[pos] = a;
    pb[pos] = (int)b;
    pd[pos] = sqrtf(d2);
    ++pos;
  });
}

// Per query b: the k nearest a within the cutoff, ascending by distance (ties:
// smaller a first); empty slots hold a = -1, r = +inf.
__global__ void __launch_bounds__(128) k_cross_knn(const __grid_constant__ SweepArgs A,
                                                   const __grid_constant__ QueryArgs Q, int k, int* __restrict__ out_a,
                                                   float* __restrict__ out_d, int* __restrict__ err) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= Q.nb) return;
  float bd[kKnnMax];
  int ba[kKnnMax];
  for (int q = 0; q < k; ++q) {
    bd[q] = FLT_MAX;
    ba[q] = -1;
  }
  int cx, cy, cz;
  float px, py, pz;
  if (bin_query(A, Q, b, cx, cy, cz, px, py, pz)) {
    query_sweep(A, cx, cy, cz, px, py, pz, [&](int a, float d2) {
      if (d2 > bd[k - 1] || (d2 == bd[k - 1] && (ba[k - 1] >= 0 && a > ba[k - 1]))) return;
      int q = k - 1;  // insertion: shift the larger entries up
      while (q > 0 && (bd[q - 1] > d2 || (bd[q - 1] == d2 && ba[q - 1] > a))) {
        bd[q] = bd[q - 1];
        ba[q] = ba[q - 1];
        --q;
      }
      bd[q] = d2;
      ba[q] = a;
    });
  } else {
    atomicOr(err, kErrNonFinite);
  }
  for (int q = 0; q < k; ++q) {
    out_a[b * k + q] = ba[q];
    out_d[b * k + q] = ba[q] >= 0 ? sqrtf(bd[q]) : INFINITY;
  }
}

// The k smallest (r, a, b) over nb per-query lists of k (one CTA of 1024
// threads): chunks of 1024 candidates are sorted in shared memory by a bitonic
// network and merged into the running best k.
__global__ void __launch_bounds__(1024) k_topk_merge(const int* __restrict__ la, const float* __restrict__ ld,
                                                     long long nb, int k, int* __restrict__ oa, int* __restrict__ ob,
                                                     float* __restrict__ od, int* __restrict__ found) {
  __shared__ float cd[1024];
  __shared__ long long cid[1024];
  __shared__ float bd[kKnnMax];
  __shared__ long long bid[kKnnMax];
  __shared__ float md[2 * kKnnMax];
  __shared__ long long mid[2 * kKnnMax];
  const int t = threadIdx.x;
  if (t < k) {
    bd[t] = INFINITY;
    bid[t] = -1;
  }
  const long long total = nb * k;
  for (long long base = 0; base < total; base += 1024) {
    const long long e = base + t;
    // candidate id e = b * k + q; empty slots sort last
    cd[t] = (e < total && la[e] >= 0) ? ld[e] : INFINITY;
    cid[t] = (e < total && la[e] >= 0) ? e : LLONG_MAX;
    __syncthreads();
    for (int size = 2; size <= 1024; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const int p = t ^ stride;
        if (p > t) {
          const bool up = (t & size) == 0;
          const bool gt = cd[t] > cd[p] || (cd[t] == cd[p] && cid[t] > cid[p]);
          if (gt == up) {
            const float td = cd[t];
            cd[t] = cd[p];
            cd[p] = td;
            const long long ti = cid[t];
            cid[t] = cid[p];
            cid[p] = ti;
          }
        }
        __syncthreads();
      }
    if (t == 0) {  // merge the k best of the chunk with the running best
      int i = 0, j = 0;
      for (int q = 0; q < k; ++q) {
        const bool take_b = bd[i] < cd[j] || (bd[i] == cd[j] && bid[i] <= cid[j]);
        if (take_b) {
          md[q] = bd[i];
          mid[q] = bid[i];
          ++i;
        } else {
          md[q] = cd[j];
          mid[q] = cid[j];
          ++j;
        }
      }
      for (int q = 0; q < k; ++q) {
        bd[q] = md[q];
        bid[q] = mid[q];
      }
    }
    __syncthreads();
  }
  if (t < k) {
    const bool ok = bid[t] >= 0 && bid[t] != LLONG_MAX && bd[t] < INFINITY;
    oa[t] = ok ? la[bid[t]] : -1;
    ob[t] = ok ? (int)(bid[t] / k) : -1;
    od[t] = ok ? bd[t] : INFINITY;
    if (ok) atomicAdd(found, 1);
  }
}

}  // namespace

int launch_cross(int what, const SweepArgs& A, const Geo& g, const double* posb, long long nb, int k, int* count,
                 unsigned long long* total, const long long* start, int* pa, int* pb, float* pd, int* knn_a, float* knn_d,
                 int* err, cudaStream_t s) {
  QueryArgs Q;
  Q.pos = posb;
  Q.nb = nb;
  Q.dim = g.dim;
  Q.ortho = g.ortho;
  for (int q = 0; q < 9; ++q) {
    Q.m[q] = g.m[q];
    Q.g[q] = g.g[q];
  }
  if (nb <= 0) return CL_OK;
  const long long blocks = (nb + 255) / 256;
  if (what == 0) k_cross_count<<<(unsigned)blocks, 256, 0, s>>>(A, Q, count, total, err);
  else if (what == 1) k_cross_fill<<<(unsigned)blocks, 256, 0, s>>>(A, Q, start, pa, pb, pd);
  else k_cross_knn<<<(unsigned)((nb + 127) / 128), 128, 0, s>>>(A, Q, k, knn_a, knn_d, err);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int launch_topk_merge(const int* la, const float* ld, long long nb, int k, int* oa, int* ob, float* od, int* found,
                      cudaStream_t s) {
  if (cudaMemsetAsync(found, 0, sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  k_topk_merge<<<1, 1024, 0, s>>>(la, ld, nb, k, oa, ob, od, found);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

}  // namespace clk
