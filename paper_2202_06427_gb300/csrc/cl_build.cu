// cl_build.cu -- cell binning on the GPU (the cell-list construction of
// Sec. 2.6 and Sec. 2.8 "integer division of the coordinates").
//
//   k_bin          one thread per particle: FP64 position in cell units
//                  t = x . H^-1 . diag(n), wrap t into [0, n), cell index from
//                  the integer part, centred FP32 local coordinate from the
//                  fractional part; counts particles per cell with an atomic
//                  whose return value is the particle's slot in its cell.
//   k_scan_*       exclusive prefix sum of the per-cell counts: per-tile sums
//                  (and the number of non-empty cells and the largest count),
//                  then per tile the sum of the tiles before it and the
//                  rescan -> cell_start[ncells + 1].
//   k_scatter      moves each particle's (local coordinate, index) into its
//                  cell's range: the per-cell contiguous copy of Sec. 2.6
//                  ("vector of lists ... an immutable copy of the particle
//                  coordinates and index", Sec. 2.8).
// Per particle the build reads its FP64 position once (24 B) and moves 20 B
// through k_bin's output (local coordinate with the packed cell, slot) to the
// sorted arrays (16 B coordinate and index, 4 B packed cell).
//
// FP64 is kept for the position in cell units. On this GPU FP64 issues at
// about 1/74 of the FP32 rate, so per axis the kernel spends one FP64
// multiply (diagonal boxes; three FMAs otherwise) and one conversion: M is
// scaled by 2^32 (exact), and floor(t 2^32) as a 64-bit integer holds the
// cell coordinate in its high word and the fraction in cell units, to 2^-32,
// in its low word. Periodic wrapping is integer work. Positions 2^30 cells or
// more from the origin, and non-finite ones, take the plain FP64 floor path.
#include <cmath>

#include "cl_internal.cuh"

namespace clk {

struct BinArgs {
  const double* pos;
  int n;
  int nx, ny, nz;
  double m[9];      // t = x M
  float g[9];       // cell edge vectors (rows)
  int* slot;        // per original particle: position inside its cell
  float4* xl;       // per original particle: centred local coordinate, w = packed cell
  int* counts;      // per cell
  int* err;         // error latch
};

template <int DIM, bool ORTHO>
__global__ void __launch_bounds__(256) k_bin(const __grid_constant__ BinArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < DIM; ++k) x[k] = a.pos[(size_t)i * DIM + k];
  bool finite = true;
#pragma unroll
  for (int k = 0; k < DIM; ++k) finite = finite && isfinite(x[k]);
  const int nk[3] = {a.nx, a.ny, a.nz};
  int c[3] = {0, 0, 0};
  float u[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    double t;  // position in cell units times 2^32
    if (ORTHO) {
      t = x[k] * a.m[k * 3 + k];
    } else {
      t = 0.0;
#pragma unroll
      for (int q = 0; q < DIM; ++q) t = fma(x[q], a.m[q * 3 + k], t);
    }
    long long ci;
    float frac;  // in [0, 1)
    if (((__double2hiint(t) >> 20) & 0x7ff) < 1023 + 62) {  // |t| < 2^62, finite
      const long long ti = __double2ll_rd(t);
      ci = ti >> 32;
      frac = (float)(unsigned)(ti & 0xffffffffLL) * 0x1p-32f;
      frac = frac < 1.0f ? frac : 0x1.fffffep-1f;  // a fraction that rounds up to 1
    } else {
      const double tc = t * 0x1p-32;
      const double f = floor(tc);
      frac = (float)(tc - f);
      ci = finite ? (long long)f : 0;
    }
    int cm;
    if (ci >= 0 && ci < nk[k]) {
      cm = (int)ci;  // inside the box: the common case
    } else {
      long long r = ci % nk[k];
      if (r < 0) r += nk[k];
      cm = (int)r;
    }
    c[k] = cm;
    u[k] = frac - 0.5f;  // centred, in [-0.5, 0.5]
  }
  float4 o;
  o.x = 0.f; o.y = 0.f; o.z = 0.f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    o.x = fmaf(u[k], a.g[k * 3 + 0], o.x);
    o.y = fmaf(u[k], a.g[k * 3 + 1], o.y);
    if (DIM == 3) o.z = fmaf(u[k], a.g[k * 3 + 2], o.z);
  }
  if (!finite) {
    // park the particle in cell 0 at its sentinel position: every distance
    // test against it fails, and the host learns of it through the latch
    c[0] = c[1] = c[2] = 0;
    o = sentinel_pos(i);
    atomicOr(a.err, kErrNonFinite);
  }
  o.w = __uint_as_float((unsigned)c[0] | ((unsigned)c[1] << 10) | ((unsigned)c[2] << 20));
  const int lin = c[0] + a.nx * (c[1] + a.ny * c[2]);
  a.slot[i] = atomicAdd(&a.counts[lin], 1);
  a.xl[i] = o;
}

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block.
template <class T>
__device__ void block_excl_scan(T v, T* out_excl) {
  __shared__ T wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = warp_incl_scan(v);
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = (lane < kScanThreads / 32) ? wsum[lane] : T(0);
    T wi = warp_incl_scan(w);
    if (lane < kScanThreads / 32) wsum[lane] = wi - w;
  }
  __syncthreads();
  *out_excl = incl - v + wsum[warp];
  __syncthreads();  // wsum is reused by the next call
}

// Per tile: sum of counts, non-empty cells, largest count. T is the offset
// type: int for cell offsets (at most n < 2^31 particles), long long for the
// pair list, whose total may pass 2^31.
template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int* __restrict__ counts, long long ncells,
                                                             T* __restrict__ tile_sum, int* __restrict__ meta) {
  const long long base = (long long)blockIdx.x * kScanTile;
  T s = 0;
  int ne = 0, mx = 0;
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    long long c = base + k;
    if (c < ncells) {
      int v = counts[c];
      s += v;
      ne += (v > 0);
      mx = max(mx, v);
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, off);
    ne += __shfl_down_sync(0xffffffffu, ne, off);
    mx = max(mx, __shfl_down_sync(0xffffffffu, mx, off));
  }
  __shared__ T ssum[kScanThreads / 32];
  __shared__ int sm[2][kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { ssum[warp] = s; sm[0][warp] = ne; sm[1][warp] = mx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    T S = 0;
    int NE = 0, MX = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) { S += ssum[w]; NE += sm[0][w]; MX = max(MX, sm[1][w]); }
    tile_sum[blockIdx.x] = S;
    atomicAdd(&meta[1], NE);
    atomicMax(&meta[2], MX);
  }
}

// Per tile: the sum of the tiles before it (read straight from the tile sums,
// so no separate pass scans them), then the rescan of the tile's counts ->
// cell_start; the last tile also writes cell_start[ncells] = total.
template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_final(const int* __restrict__ counts, long long ncells,
                                                            const T* __restrict__ tile_sum,
                                                            T* __restrict__ cell_start) {
  __shared__ T part[kScanThreads / 32];
  T before = 0;
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += kScanThreads) before += tile_sum[t];
#pragma unroll
  for (int o = 16; o; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = before;
  __syncthreads();
  T off = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) off += part[w];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer;
  int v[kScanPer];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < ncells) ? counts[base + k] : 0;
    s += v[k];
  }
  T excl;
  block_excl_scan(s, &excl);
  T run = off + excl;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < ncells) cell_start[base + k] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) cell_start[ncells] = run;
}

__global__ void __launch_bounds__(256) k_scatter(int n, int nx, int ny, const int* __restrict__ slot,
                                                const float4* __restrict__ xl, const int* __restrict__ cell_start,
                                                float4* __restrict__ xs, unsigned* __restrict__ cellc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 v = xl[i];
  const unsigned cc = __float_as_uint(v.w);
  const int lin = (int)(cc & 1023u) + nx * ((int)((cc >> 10) & 1023u) + ny * (int)(cc >> 20));
  const int p = cell_start[lin] + slot[i];
  v.w = __int_as_float(i);
  xs[p] = v;
  cellc[p] = cc;
}

// ------------------------------------------------------------ host entry --



int scan_tiles_for(long long ncells) { return (int)((ncells + kScanTile - 1) / kScanTile); }

// Enqueue the whole binning pipeline on `s`. Returns CL_OK or CL_ERR_CUDA.
int launch_build(const Geo& g, const BuildBufs& b, cudaStream_t s) {
  const long long nc = g.ncells;
  const int ntiles = scan_tiles_for(nc);
  if (cudaMemsetAsync(b.counts, 0, sizeof(int) * nc, s) != cudaSuccess) return CL_ERR_CUDA;
  if (cudaMemsetAsync(b.meta + 1, 0, sizeof(int) * 2, s) != cudaSuccess) return CL_ERR_CUDA;
  BinArgs a;
  a.pos = b.pos;
  a.n = b.n;
  a.nx = g.n[0]; a.ny = g.n[1]; a.nz = g.n[2];
  for (int k = 0; k < 9; ++k) {
    a.m[k] = std::ldexp(g.m[k], 32);  // exact: t 2^32 = x (M 2^32)
    a.g[k] = g.g[k];
  }
  a.slot = b.slot; a.xl = b.xl; a.counts = b.counts; a.err = b.meta;
  const int blocks = (b.n + 255) / 256;
  if (b.n > 0) {
    if (g.dim == 3) {
      if (g.ortho) k_bin<3, true><<<blocks, 256, 0, s>>>(a);
      else k_bin<3, false><<<blocks, 256, 0, s>>>(a);
    } else {
      if (g.ortho) k_bin<2, true><<<blocks, 256, 0, s>>>(a);
      else k_bin<2, false><<<blocks, 256, 0, s>>>(a);
    }
  }
  k_scan_reduce<int><<<ntiles, kScanThreads, 0, s>>>(b.counts, nc, b.tile_sum, b.meta);
  k_scan_final<int><<<ntiles, kScanThreads, 0, s>>>(b.counts, nc, b.tile_sum, b.cell_start);
  if (b.n > 0)
    k_scatter<<<blocks, 256, 0, s>>>(b.n, g.n[0], g.n[1], b.slot, b.xl, b.cell_start, b.xs, b.cellc);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

}  // namespace clk

namespace clk {

// Exclusive scan of n int counts into 64-bit start[n + 1] (start[n] = total),
// with the same two kernels as the cell offsets; meta receives the number of
// non-zero counts and the largest one. The pair list's offsets and total are
// 64-bit: a list may hold more than 2^31 pairs.
int launch_scan64(const int* counts, long long n, long long* tile_sum, long long* start, int* meta, cudaStream_t s) {
  const int ntiles = scan_tiles_for(n);
  if (cudaMemsetAsync(meta + 1, 0, sizeof(int) * 2, s) != cudaSuccess) return CL_ERR_CUDA;
  if (ntiles == 0) return cudaMemsetAsync(start, 0, sizeof(long long), s) == cudaSuccess ? CL_OK : CL_ERR_CUDA;
  k_scan_reduce<long long><<<ntiles, kScanThreads, 0, s>>>(counts, n, tile_sum, meta);
  k_scan_final<long long><<<ntiles, kScanThreads, 0, s>>>(counts, n, tile_sum, start);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

}  // namespace clk
