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
//   k_cellc        the packed cell of every sorted particle, cell by cell.
//   k_octsort      (launched by the 3D half-shell sweep on its windowed cells)
//                  cells of kOctMin..kOctCap particles ordered by the octant
//                  of their local coordinates (slots updated to match).
// Per particle the build reads its FP64 position once (24 B) and moves 20 B
// through k_bin's output (local coordinate with the packed cell, slot) to the
// sorted arrays (16 B coordinate and index, 4 B packed cell).
//
// The position in cell units is exact integer work where it can be. M is
// scaled by 2^32, and floor(t 2^32) as a 64-bit integer holds the cell
// coordinate in its high word and the fraction in cell units, to 2^-32, in
// its low word. On this GPU FP64 issues at about 1/74 of the FP32 rate, so for
// diagonal boxes the product x M_kk is formed from the two 53-bit mantissas
// with 64-bit integer multiplies (a 106-bit product, shifted and floored
// exactly); for triclinic boxes t is three FP64 FMAs per axis and its floor is
// read from its bits the same way, so no FP64 conversion is issued. Periodic
// wrapping is integer work. Positions 2^30 cells or more from the origin, and
// non-finite ones, take the plain FP64 floor path.
#include <algorithm>
#include <cmath>

#include "cl_internal.cuh"

namespace clk {

struct BinArgs {
  const double* pos;
  int n;
  int nx, ny, nz;
  double m[9];      // t = x M
  unsigned long long mm[3];  // diagonal boxes: M_kk 2^32 = mm[k] 2^me[k], mm[k] in [2^52, 2^53)
  int me[3];
  float g[9];       // cell edge vectors (rows)
  int* slot;        // per original particle: position inside its cell
  float4* xl;       // per original particle: centred local coordinate, w = packed cell
  int* counts;      // per cell
  int* err;         // error latch
};

// floor(x mm 2^me) as a 64-bit integer, exactly, for a finite x and mm in
// [2^52, 2^53): the 53-bit mantissa of x times mm is a 106-bit integer, which
// is shifted right and floored (toward minus infinity for negative x). False
// when x is not finite or the result reaches 2^62 in magnitude.
__device__ __forceinline__ bool floor_mul(double x, unsigned long long mm, int me, long long& out) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ffu);
  if (ex == 0x7ff) return false;
  const bool neg = (b >> 63) != 0;
  unsigned long long mx = b & 0xfffffffffffffull;
  if (ex != 0) mx |= 1ull << 52;
  if (mx == 0) {
    out = 0;
    return true;
  }
  const int k = 1075 - (ex != 0 ? ex : 1) - me;  // x mm 2^me = mx mm 2^-k
  if (k <= 0) return false;                       // at least 2^104
  const unsigned long long lo = mx * mm, hi = __umul64hi(mx, mm);
  unsigned long long q;
  bool rem;
  if (k >= 128) {
    q = 0;
    rem = true;
  } else if (k >= 64) {
    const int r = k - 64;
    q = r ? hi >> r : hi;
    rem = lo != 0 || (r && (hi & ((1ull << r) - 1)) != 0);
  } else {
    if ((hi >> k) != 0) return false;
    q = (lo >> k) | (hi << (64 - k));
    rem = (lo & ((1ull << k) - 1)) != 0;
  }
  if (q >= (1ull << 62)) return false;
  out = neg ? -(long long)q - (rem ? 1 : 0) : (long long)q;
  return true;
}

// One particle: its packed cell and centred local coordinate (o, w = packed
// cell) and its linear cell index.
template <int DIM, bool ORTHO>
__device__ __forceinline__ void bin_one(const BinArgs& a, int i, float4& o, int& lin) {
  double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < DIM; ++k) x[k] = a.pos[(size_t)i * DIM + k];
  bool finite = true;  // from the exponent bits: no FP64 compare
#pragma unroll
  for (int k = 0; k < DIM; ++k) finite = finite && ((__double2hiint(x[k]) >> 20) & 0x7ff) != 0x7ff;
  const int nk[3] = {a.nx, a.ny, a.nz};
  int c[3] = {0, 0, 0};
  float u[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    long long ti;  // floor of the position in cell units times 2^32
    bool exact;
    double t = 0.0;
    if (ORTHO) {
      exact = floor_mul(x[k], a.mm[k], a.me[k], ti);
    } else {
#pragma unroll
      for (int q = 0; q < DIM; ++q) t = fma(x[q], a.m[q * 3 + k], t);
      exact = floor_mul(t, 1ull << 52, -52, ti);
    }
    long long ci;
    float frac;  // in [0, 1)
    if (exact) {
      ci = ti >> 32;
      frac = (float)(unsigned)(ti & 0xffffffffLL) * 0x1p-32f;
      frac = frac < 1.0f ? frac : 0x1.fffffep-1f;  // a fraction that rounds up to 1
    } else {
      if (ORTHO) t = x[k] * a.m[k * 3 + k];
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
  lin = c[0] + a.nx * (c[1] + a.ny * c[2]);
}

// kBinPer particles per thread (strided by the block size, so every load and
// store stays coalesced), their count atomics issued together. Measured at 8M
// particles: one per thread 105 us (k_bin) and 86 us (k_scatter), four per
// thread 110 and 98 us: the kernels are bound by memory throughput, not by
// the atomics' latency.
constexpr int kBinPer = 1;

template <int DIM, bool ORTHO>
__global__ void __launch_bounds__(256) k_bin(const __grid_constant__ BinArgs a) {
  const long long i0 = (long long)blockIdx.x * (blockDim.x * kBinPer) + threadIdx.x;  // 64-bit: n may near 2^31
  float4 o[kBinPer];
  int lin[kBinPer];
#pragma unroll
  for (int u = 0; u < kBinPer; ++u) {
    const long long i = i0 + u * (long long)blockDim.x;
    if (i < a.n) {
      bin_one<DIM, ORTHO>(a, (int)i, o[u], lin[u]);
      a.xl[i] = o[u];
    }
  }
  int sl[kBinPer];
#pragma unroll
  for (int u = 0; u < kBinPer; ++u)
    if (i0 + u * (long long)blockDim.x < a.n) sl[u] = atomicAdd(&a.counts[lin[u]], 1);
#pragma unroll
  for (int u = 0; u < kBinPer; ++u) {
    const long long i = i0 + u * (long long)blockDim.x;
    if (i < a.n) a.slot[i] = sl[u];
  }
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

// Orders the particles of each listed cell of kOctMin..kOctCap particles by
// the octant of their local coordinate (key = (x > 0) | (y > 0) << 1 |
// (z > 0) << 2): a counting sort through shared memory, writing the cell's
// range of xs back in key order and each moved particle's slot. The order of
// particles within a cell is free (every sweep indexes them through xs.w and
// slot), so the cell list stays valid. One CTA per cell, persistent over the
// list; other listed cells are skipped.
__global__ void __launch_bounds__(256) k_octsort(const int* __restrict__ big, const int* __restrict__ nbig,
                                                const int* __restrict__ cell_start, float4* __restrict__ xs,
                                                int* __restrict__ slot) {
  __shared__ float4 buf[kOctCap];
  __shared__ int cnt[8], at[8];
  const int nb = *nbig;
  for (int q = blockIdx.x; q < nb; q += gridDim.x) {
    const int c = big[q];
    const int hs = cell_start[c], nh = cell_start[c + 1] - hs;
    if (nh < kOctMin || nh > kOctCap) continue;  // uniform over the CTA
    if (threadIdx.x < 8) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
      const float4 v = xs[hs + t];
      buf[t] = v;
      atomicAdd(&cnt[(v.x > 0.f ? 1 : 0) | (v.y > 0.f ? 2 : 0) | (v.z > 0.f ? 4 : 0)], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int k = 0; k < 8; ++k) {
        at[k] = run;
        run += cnt[k];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
      const float4 v = buf[t];
      const int p = atomicAdd(&at[(v.x > 0.f ? 1 : 0) | (v.y > 0.f ? 2 : 0) | (v.z > 0.f ? 4 : 0)], 1);
      xs[hs + p] = v;
      slot[__float_as_int(v.w)] = p;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_scatter(int n, int nx, int ny, const int* __restrict__ slot,
                                                const float4* __restrict__ xl, const int* __restrict__ cell_start,
                                                float4* __restrict__ xs) {
  const long long i0 = (long long)blockIdx.x * (blockDim.x * kBinPer) + threadIdx.x;
  float4 v[kBinPer];
  int p[kBinPer];
#pragma unroll
  for (int u = 0; u < kBinPer; ++u) {  // kBinPer particles per thread: the dependent loads overlap
    const long long i = min(i0 + u * (long long)blockDim.x, (long long)n - 1);
    v[u] = xl[i];
    p[u] = slot[i];
  }
#pragma unroll
  for (int u = 0; u < kBinPer; ++u) {
    const unsigned cc = __float_as_uint(v[u].w);
    p[u] += cell_start[(int)(cc & 1023u) + nx * ((int)((cc >> 10) & 1023u) + ny * (int)(cc >> 20))];
  }
#pragma unroll
  for (int u = 0; u < kBinPer; ++u) {
    const long long i = i0 + u * (long long)blockDim.x;
    if (i < n) {
      v[u].w = __int_as_float((int)i);
      xs[p[u]] = v[u];
    }
  }
}

// Packed cell of every sorted particle, written along the sorted array
// (coalesced), where a write per particle from k_scatter would land 4 B at a
// random address. A warp takes 32 consecutive cells (lane l loads cell l's
// range and packed coordinates) and writes them one after the other, all
// lanes over one cell's range.
__global__ void __launch_bounds__(256) k_cellc(long long ncells, int nx, int ny, const int* __restrict__ cell_start,
                                              unsigned* __restrict__ cellc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long c0 = (blockIdx.x * 8LL + warp) * 32; c0 < ncells; c0 += (long long)gridDim.x * 8 * 32) {
    const long long c = c0 + lane;
    int s0 = 0, s1 = 0;
    unsigned cc = 0;
    if (c < ncells) {
      s0 = cell_start[c];
      s1 = cell_start[c + 1];
      const int cx = (int)(c % nx), cy = (int)((c / nx) % ny), cz = (int)(c / ((long long)nx * ny));
      cc = (unsigned)cx | ((unsigned)cy << 10) | ((unsigned)cz << 20);
    }
    unsigned live = __ballot_sync(0xffffffffu, s1 > s0);
    while (live) {
      const int j = __ffs(live) - 1;
      live &= live - 1;
      const int a = __shfl_sync(0xffffffffu, s0, j), b = __shfl_sync(0xffffffffu, s1, j);
      const unsigned v = __shfl_sync(0xffffffffu, cc, j);
      for (int p = a + lane; p < b; p += 32) cellc[p] = v;
    }
  }
}

// ------------------------------------------------------------ host entry --



int launch_octsort(const int* cells, const int* ncells_listed, const int* cell_start, float4* xs, int* slot,
                   cudaStream_t s) {
  k_octsort<<<152 * 4, 256, 0, s>>>(cells, ncells_listed, cell_start, xs, slot);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

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
  for (int k = 0; k < 3; ++k) {  // M_kk 2^32 = f 2^e, f in [0.5, 1): mantissa f 2^53, exponent e - 53
    int e = 0;
    const double f = std::frexp(a.m[k * 3 + k], &e);
    a.mm[k] = (unsigned long long)std::ldexp(f, 53);
    a.me[k] = e - 53;
    if (!(a.m[k * 3 + k] > 0.0)) {  // not a diagonal entry (triclinic boxes do not use it)
      a.mm[k] = 1ull << 52;
      a.me[k] = -52;
    }
  }
  a.slot = b.slot; a.xl = b.xl; a.counts = b.counts; a.err = b.meta;
  const int blocks = (b.n + 256 * kBinPer - 1) / (256 * kBinPer);
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
  if (b.n > 0) {
    k_scatter<<<blocks, 256, 0, s>>>(b.n, g.n[0], g.n[1], b.slot, b.xl, b.cell_start, b.xs);
    const long long cb = std::min<long long>((nc + 255) / 256, 152 * 8);
    k_cellc<<<(int)cb, 256, 0, s>>>(nc, g.n[0], g.n[1], b.cell_start, b.cellc);
  }
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
