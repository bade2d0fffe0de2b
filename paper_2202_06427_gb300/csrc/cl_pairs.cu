// cl_pairs.cu -- the i<j neighbour list (Sec. 4.1: "the lists of pairs of
// particles within a cutoff"), sorted by (i, j), with the FP32 distance.
//
//   k_pairs_cell<COUNT>  one CTA per cell stages the cell's neighbourhood
//                  (the particles of its full stencil that lie within
//                  rc + half a cell diagonal of its centre and whose index is
//                  above the smallest of the cell's own) in shared memory;
//                  one warp per home particle sweeps it and counts the pairs
//                  with j > i (original indices), so every pair is counted
//                  once, by its smaller index, without atomics. A cell whose
//                  neighbourhood does not fit is flagged and listed.
//   (scan)         exclusive prefix sum of the counts in original order:
//                  segment of i = [start[i], start[i] + count[i])
//   k_pairs_cell<FILL>   the same staging, then the staged list's original
//                  indices are radix-sorted, so each particle's pairs with
//                  j > i come out of a suffix of that order in ascending j and
//                  are written in order with coalesced stores
//   k_pairs_count / k_pairs_fill_sorted
//                  the listed cells' particles, one thread (count) or one warp
//                  (fill) per particle straight from the sorted arrays; a
//                  segment longer than kMaxSegment is written unsorted and
//                  listed for k_pairs_sort_long
//   k_pairs_sort   one warp per segment, in place, for the two-set list (its
//                  segments are filled by a per-query sweep); longer segments
//                  are listed for k_pairs_sort_long
//   k_pairs_sort_long  one CTA per listed segment, in place in global memory
//
// Each particle's count and fill run the same arithmetic in the same kernel
// family, so the fill keeps exactly count[i] pairs (the write is clamped to
// count[i] all the same). The sweep visits the pair-images of a particle; the
// list is only defined when each pair has at most one image within rc
// (rc <= w_min / 2), which the host checks before launching.
#include <climits>

#include "cl_sweep.cuh"

namespace clk {


struct RedPairCount {
  static constexpr bool kFull = true;
  struct Acc { int a; int n; };
  __device__ void init(Acc& x) const { x.n = 0; }
  __device__ void hit(Acc& x, float, float, float, float, int j) const { x.n += (j > x.a) ? 1 : 0; }
};

// The particles of the listed cells (cells[0, *ncells)), one thread each.
template <int DIM>
__global__ void __launch_bounds__(256) k_pairs_count(const __grid_constant__ SweepArgs A,
                                                     const int* __restrict__ cells, const int* __restrict__ ncells,
                                                     int* __restrict__ count) {
  const int m = *ncells;
  for (int q = blockIdx.x; q < m; q += gridDim.x) {
    const int c = cells[q];
    const int p1 = A.cell_start[c + 1];
    for (int p = A.cell_start[c] + threadIdx.x; p < p1; p += blockDim.x) {
      RedPairCount red;
      RedPairCount::Acc acc;
      red.init(acc);
      acc.a = __float_as_int(A.xs[p].w);
      float4 pi;
      sweep_particle<DIM>(A, red, acc, p, pi);
      count[acc.a] = acc.n;
    }
  }
}

constexpr int kSortWarps = 4;

// One warp per segment (grid-stride): bitonic sort of up to kMaxSegment keys
// (j, distinct within a segment) with their distances, in shared memory.
// Longer segments are appended to longs[] (counter *nlong) for
// k_pairs_sort_long.
__global__ void __launch_bounds__(32 * kSortWarps) k_pairs_sort(int n, const int* __restrict__ count,
                                                               const long long* __restrict__ start, int* __restrict__ pj,
                                                               float* __restrict__ pd, int* __restrict__ longs,
                                                               int* __restrict__ nlong) {
  __shared__ int sk[kSortWarps][kMaxSegment];
  __shared__ float sv[kSortWarps][kMaxSegment];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* K = sk[warp];
  float* V = sv[warp];
  for (int a = blockIdx.x * kSortWarps + warp; a < n; a += gridDim.x * kSortWarps) {
    const int L = count[a];
    if (L <= 1) continue;
    if (L > kMaxSegment) {
      if (lane == 0) longs[atomicAdd(nlong, 1)] = a;
      continue;
    }
    const long long base = start[a];
    int P = 32;
    while (P < L) P <<= 1;
    for (int k = lane; k < P; k += 32) {
      if (k < L) {
        K[k] = pj[base + k];
        V[k] = pd[base + k];
      } else {
        K[k] = INT_MAX;
        V[k] = 0.f;
      }
    }
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = lane; t < (P >> 1); t += 32) {
          const int lo = 2 * stride * (t / stride) + (t % stride);
          const int hi = lo + stride;
          const bool up = (lo & size) == 0;
          const int ka = K[lo], kb = K[hi];
          if ((ka > kb) == up) {
            K[lo] = kb;
            K[hi] = ka;
            const float va = V[lo];
            V[lo] = V[hi];
            V[hi] = va;
          }
        }
        __syncwarp();
      }
    }
    for (int k = lane; k < L; k += 32) {
      pj[base + k] = K[k];
      pd[base + k] = V[k];
    }
    __syncwarp();
  }
}

// One CTA per listed segment (grid-stride over the *nlong entries): the
// segment sorted by j in place in global memory by a bitonic network whose
// compare-exchanges all put the smaller key first (each merge opens with the
// mirrored pairing i <-> size - 1 - i of its block), padded to a power of two
// with virtual +inf keys past the end, which never move.
__global__ void __launch_bounds__(1024) k_pairs_sort_long(const int* __restrict__ longs,
                                                         const int* __restrict__ nlong,
                                                         const int* __restrict__ count,
                                                         const long long* __restrict__ start, int* __restrict__ pj,
                                                         float* __restrict__ pd) {
  const int m = *nlong;
  for (int q = blockIdx.x; q < m; q += gridDim.x) {
    const int a = longs[q];
    const int L = count[a];
    int* K = pj + start[a];
    float* V = pd + start[a];
    int P = 2;
    while (P < L) P <<= 1;
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
          int lo, hi;
          if (stride == (size >> 1)) {
            const int blk = t / stride, off = t - blk * stride;
            lo = blk * size + off;
            hi = blk * size + size - 1 - off;
          } else {
            lo = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
            hi = lo + stride;
          }
          if (hi < L) {
            const int ka = K[lo], kb = K[hi];
            if (ka > kb) {
              K[lo] = kb;
              K[hi] = ka;
              const float va = V[lo];
              V[lo] = V[hi];
              V[hi] = va;
            }
          }
        }
        __syncthreads();
      }
    }
  }
}

// Shared pieces of the pair-list sweeps. A warp takes the stencil 32 entries
// at a time, one per lane: each lane finds its neighbour cell's particle
// range, a warp scan lays the ranges end to end, and the warp walks the
// concatenation 32 candidates per step (a shuffle binary search finds each
// candidate's entry), so the lanes stay busy however small the cells are. The
// kept pairs of a particle are compacted with a ballot into the warp's
// shared-memory segment, sorted by j in registers (bitonic) and written to
// [start[a], start[a] + count[a]) with coalesced stores. Segments are at most
// kMaxSegment long (the host checks the counts first).
constexpr int kFillWarps = 4;
constexpr int kStageMax = 3072;  // largest staged neighbourhood of one cell (the launch picks its capacity)
constexpr int kSegPad = kMaxSegment + kMaxSegment / 32;

// Segment buffer index with one pad word per 32: conflict-free both for lane i
// at i (coalesced order) and for lane l at l * E + e (blocked order, E <= 32).
__device__ __forceinline__ int seg_at(int i) { return i + (i >> 5); }

// Bitonic sort, ascending by key, of 32 E elements held E per lane in blocked
// order (element lane * E + e). Pairs closer than E apart are in one lane's
// registers; farther ones are exchanged with a shuffle.
template <int E>
__device__ __forceinline__ void sort_blocked(int (&k)[E], float (&v)[E], int lane) {
#pragma unroll
  for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= E) {
        const int ls = stride / E;
        const bool lower = (lane & ls) == 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const bool up = ((lane * E + e) & size) == 0;
          const int ok = __shfl_xor_sync(0xffffffffu, k[e], ls);
          const float ov = __shfl_xor_sync(0xffffffffu, v[e], ls);
          const bool take = (lower == up) ? (ok < k[e]) : (ok > k[e]);
          k[e] = take ? ok : k[e];
          v[e] = take ? ov : v[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if ((e & stride) == 0) {
            const int f = e | stride;
            const bool up = ((lane * E + e) & size) == 0;
            const bool sw = up ? (k[e] > k[f]) : (k[e] < k[f]);
            const int tk = k[e];
            const float tv = v[e];
            k[e] = sw ? k[f] : k[e];
            v[e] = sw ? v[f] : v[e];
            k[f] = sw ? tk : k[f];
            v[f] = sw ? tv : v[f];
          }
        }
      }
    }
  }
}

template <int E>
__device__ __forceinline__ void sort_segment_regs(int* K, float* V, int L, int lane) {
  int k[E];
  float v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = lane * E + e;
    k[e] = i < L ? K[seg_at(i)] : INT_MAX;
    v[e] = i < L ? V[seg_at(i)] : 0.f;
  }
  sort_blocked<E>(k, v, lane);
  __syncwarp();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = lane * E + e;
    if (i < L) {
      K[seg_at(i)] = k[e];
      V[seg_at(i)] = v[e];
    }
  }
  __syncwarp();
}

// Segments longer than 16 per lane: the same network in shared memory.
__device__ void sort_segment_smem(int* K, float* V, int L, int lane) {
  int P = 32;
  while (P < L) P <<= 1;
  for (int i = L + lane; i < P; i += 32) {
    K[seg_at(i)] = INT_MAX;
    V[seg_at(i)] = 0.f;
  }
  __syncwarp();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = lane; t < (P >> 1); t += 32) {
        const int lo = 2 * stride * (t / stride) + (t % stride);
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const int ka = K[seg_at(lo)], kb = K[seg_at(hi)];
        if ((ka > kb) == up) {
          K[seg_at(lo)] = kb;
          K[seg_at(hi)] = ka;
          const float va = V[seg_at(lo)];
          V[seg_at(lo)] = V[seg_at(hi)];
          V[seg_at(hi)] = va;
        }
      }
      __syncwarp();
    }
  }
}


// Stencil entries k0 + lane of cell (cx, cy, cz): the lane's range [j0, j0 +
// len) of sorted particles, its shift (stencil shift + (bx, by, bz)) and, over
// the warp, the exclusive offsets of the ranges laid end to end and their total.
struct Chunk {
  int j0, len, excl, total;
  float sx, sy, sz;
};

template <int DIM>
__device__ __forceinline__ Chunk chunk_ranges(const SweepArgs& A, const float4* stab, int k0, int lane, int cx,
                                              int cy, int cz, float bx, float by, float bz, int lim = 32) {
  Chunk ch;
  ch.j0 = 0;
  ch.len = 0;
  ch.sx = ch.sy = ch.sz = 0.f;
  const int k = k0 + lane;
  if (lane < lim && k < A.noff) {  // lim: the entries this warp takes (lanes 0..lim-1)
    const float4 e = stab[k];
    const unsigned d = __float_as_uint(e.w);
    int x2 = cx + (int)(d & 1023u);
    x2 -= (x2 >= A.nx) ? A.nx : 0;
    int y2 = cy + (int)((d >> 10) & 1023u);
    y2 -= (y2 >= A.ny) ? A.ny : 0;
    int z2 = 0;
    if (DIM == 3) {
      z2 = cz + (int)(d >> 20);
      z2 -= (z2 >= A.nz) ? A.nz : 0;
    }
    const int c = x2 + A.nx * (y2 + A.ny * z2);
    ch.j0 = __ldg(A.cell_start + c);
    ch.len = __ldg(A.cell_start + c + 1) - ch.j0;
    ch.sx = e.x + bx;
    ch.sy = e.y + by;
    ch.sz = e.z + bz;
  }
  int inc = ch.len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    inc += lane >= o ? u : 0;
  }
  ch.total = __shfl_sync(0xffffffffu, inc, 31);
  ch.excl = inc - ch.len;
  return ch;
}

// Candidate t of the chunk: its sorted index and the shift of its entry.
__device__ __forceinline__ int chunk_candidate(const Chunk& ch, int t, float& ax, float& ay, float& az) {
  int l = 0;  // last entry whose range starts at or before t
#pragma unroll
  for (int b = 16; b >= 1; b >>= 1) {
    const int u = __shfl_sync(0xffffffffu, ch.excl, l + b);
    l += (u <= t) ? b : 0;
  }
  ax = __shfl_sync(0xffffffffu, ch.sx, l);
  ay = __shfl_sync(0xffffffffu, ch.sy, l);
  az = __shfl_sync(0xffffffffu, ch.sz, l);
  return __shfl_sync(0xffffffffu, ch.j0, l) + (t - __shfl_sync(0xffffffffu, ch.excl, l));
}

__device__ __forceinline__ void stencil_to_smem(const SweepArgs& A, float4* stab) {
  for (int k = threadIdx.x; k < A.noff; k += blockDim.x) {
    const Off& o = A.off[k];
    stab[k] = make_float4(o.sx, o.sy, o.sz,
                          __uint_as_float((unsigned)o.dx | ((unsigned)o.dy << 10) | ((unsigned)o.dz << 20)));
  }
}

// Sorts the warp's segment of nw kept pairs by j and writes it at base.
__device__ __forceinline__ void segment_out(int* K, float* V, int nw, int a, long long base, int lane, int* pi_out,
                                            int* pj_out, float* pd_out) {
  if (nw <= 1) {
  } else if (nw <= 32) {
    sort_segment_regs<1>(K, V, nw, lane);
  } else if (nw <= 64) {
    sort_segment_regs<2>(K, V, nw, lane);
  } else if (nw <= 128) {
    sort_segment_regs<4>(K, V, nw, lane);
  } else if (nw <= 256) {
    sort_segment_regs<8>(K, V, nw, lane);
  } else if (nw <= 512) {
    sort_segment_regs<16>(K, V, nw, lane);
  } else {
    sort_segment_smem(K, V, nw, lane);
  }
  for (int i = lane; i < nw; i += 32) {
    pi_out[base + i] = a;
    pj_out[base + i] = K[seg_at(i)];
    pd_out[base + i] = V[seg_at(i)];
  }
  __syncwarp();
}

// The listed cells' particles, one warp per particle, straight from the sorted
// arrays: the candidate's distance is x_j + (s_o - x_i), equal in IEEE
// arithmetic to x_j - (x_i - s_o) of k_pairs_count (same fused multiply-adds).
template <int DIM>
__global__ void __launch_bounds__(32 * kFillWarps, 6) k_pairs_fill_sorted(const __grid_constant__ SweepArgs A,
                                                                          const int* __restrict__ cells,
                                                                          const int* __restrict__ ncells,
                                                                          const int* __restrict__ count,
                                                                          const long long* __restrict__ start,
                                                                          int* __restrict__ pi_out,
                                                                          int* __restrict__ pj_out,
                                                                          float* __restrict__ pd_out,
                                                                          int* __restrict__ longs,
                                                                          int* __restrict__ nlong) {
  extern __shared__ float4 stab[];  // per entry: (s_x, s_y, s_z, dx | dy << 10 | dz << 20)
  __shared__ int sk[kFillWarps][kSegPad];
  __shared__ float sv[kFillWarps][kSegPad];
  stencil_to_smem(A, stab);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int* K = sk[warp];
  float* V = sv[warp];
  const int mc = *ncells;
  for (int q = blockIdx.x; q < mc; q += gridDim.x) {
    const int cq = cells[q];
    const int pend = A.cell_start[cq + 1];
    for (int p = A.cell_start[cq] + warp; p < pend; p += kFillWarps) {
      const float4 pi = A.xs[p];
      const int a = __float_as_int(pi.w);
      const unsigned cc = A.cellc[p];
      const int cx = (int)(cc & 1023u), cy = (int)((cc >> 10) & 1023u), cz = (int)(cc >> 20);
      const int cnt_a = __ldg(count + a);
      const long long base = __ldg(start + a);
      const bool big = cnt_a > kMaxSegment;  // written unsorted, sorted by k_pairs_sort_long
      int L = 0;
      for (int k0 = 0; k0 < A.noff; k0 += 32) {
        const Chunk ch = chunk_ranges<DIM>(A, stab, k0, lane, cx, cy, cz, -pi.x, -pi.y, -pi.z);
        for (int t0 = 0; t0 < ch.total; t0 += 32) {
          const int t = t0 + lane;
          float ax, ay, az;
          const int j = chunk_candidate(ch, t, ax, ay, az);
          bool keep = false;
          int jo = 0;
          float d2 = 0.f;
          if (t < ch.total) {
            const float4 q = __ldg(&A.xs[j]);
            jo = __float_as_int(q.w);
            const float dx = q.x + ax, dy = q.y + ay;
            const float dz = DIM == 3 ? q.z + az : 0.f;
            d2 = DIM == 3 ? fmaf(dx, dx, fmaf(dy, dy, dz * dz)) : fmaf(dx, dx, dy * dy);
            keep = jo > a && d2 < A.rc2;
          }
          const unsigned m = __ballot_sync(0xffffffffu, keep);
          if (keep) {
            const int e = L + __popc(m & lt);
            if (big) {
              if (e < cnt_a) {
                pi_out[base + e] = a;
                pj_out[base + e] = jo;
                pd_out[base + e] = d2 * rsqrt_nr(d2);
              }
            } else if (e < kMaxSegment) {
              K[seg_at(e)] = jo;
              V[seg_at(e)] = d2 * rsqrt_nr(d2);
            }
          }
          L += __popc(m);
        }
      }
      __syncwarp();
      if (big) {
        if (lane == 0) longs[atomicAdd(nlong, 1)] = a;
      } else {
        segment_out(K, V, min(min(L, kMaxSegment), cnt_a), a, base, lane, pi_out, pj_out, pd_out);
      }
    }
  }
}

// Stable LSD radix sort (8-bit digits) of the staged list's original indices,
// the whole CTA (W warps) taking part: the slots 0..S-1 into st are sorted by
// the key jo - kmin, read through the slot (no key array, so that four CTAs
// fit per SM). Each warp ranks a fixed span of positions in order with
// __match_any_sync, and the (digit, warp) offsets come from one exclusive scan
// per pass, so equal digits keep their order. Returns the buffer that holds
// the sorted slots.
template <int W>
__device__ __forceinline__ void stage_radix(const float4* st, int S, unsigned short* s0, unsigned short* s1,
                                            unsigned short* cnt,
                                            int* scal, unsigned short*& slots, int& kmin) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) {
    scal[1] = INT_MAX;
    scal[2] = 0;
  }
  __syncthreads();
  int lo = INT_MAX, hi = 0;
  for (int i = threadIdx.x; i < S; i += blockDim.x) {
    const int jo = __float_as_int(st[i].w);
    lo = min(lo, jo);
    hi = max(hi, jo);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if (lane == 0) {
    atomicMin(scal + 1, lo);
    atomicMax(scal + 2, hi);
  }
  __syncthreads();
  kmin = scal[1];
  const unsigned range = (unsigned)(scal[2] - kmin);
  for (int i = threadIdx.x; i < S; i += blockDim.x) s0[i] = (unsigned short)i;
  __syncthreads();
  const int bits = range ? 32 - __clz(range) : 0;
  const int span = (((S + W - 1) / W) + 31) & ~31;
  const int b0 = min(S, warp * span), b1 = min(S, b0 + span);
  for (int sh = 0; sh < bits; sh += 8) {
    for (int i = threadIdx.x; i < 256 * W; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int r = b0; r < b1; r += 32) {
      const int i = r + lane;
      const bool ok = i < b1;
      const int d = ok ? (int)(((unsigned)(__float_as_int(st[s0[i]].w) - kmin) >> sh) & 255u) : 256 + lane;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      if (ok && lane == __ffs(peers) - 1) cnt[d * W + warp] += (unsigned short)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {  // exclusive scan of cnt in (digit, warp) order; 8 entries per thread
      const int per = 256 * W / blockDim.x;
      int loc = 0;
      for (int e = 0; e < per; ++e) loc += cnt[threadIdx.x * per + e];
      int inc = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        inc += lane >= o ? u : 0;
      }
      if (lane == 31) scal[4 + warp] = inc;
      __syncthreads();
      int off = inc - loc;
      for (int w = 0; w < warp; ++w) off += scal[4 + w];
      for (int e = 0; e < per; ++e) {
        const int v = cnt[threadIdx.x * per + e];
        cnt[threadIdx.x * per + e] = (unsigned short)off;
        off += v;
      }
    }
    __syncthreads();
    for (int r = b0; r < b1; r += 32) {
      const int i = r + lane;
      const bool ok = i < b1;
      const unsigned key = ok ? (unsigned)(__float_as_int(st[s0[i]].w) - kmin) : 0u;
      const int d = ok ? (int)((key >> sh) & 255u) : 256 + lane;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int base = ok ? cnt[d * W + warp] : 0;
      __syncwarp();
      if (ok) {
        if (lane == __ffs(peers) - 1) cnt[d * W + warp] = (unsigned short)(base + __popc(peers));
        const int pos = base + __popc(peers & lt);
        s1[pos] = s0[i];
      }
      __syncwarp();
    }
    __syncthreads();
    unsigned short* ts = s0;
    s0 = s1;
    s1 = ts;
  }
  slots = s0;
}

// Squared distances of a staged entry q to two home particles (nx, ny, nz:
// their negated coordinates), both in packed FP32: per lane the same rounding
// as fmaf(dx, dx, fmaf(dy, dy, dz * dz)) with dx = q.x - x. The count and the
// fill pass both decide j within rc from this one expression.
template <int DIM>
__device__ __forceinline__ float2 pair_d2(const float4& q, float2 nx, float2 ny, float2 nz, float2& dx, float2& dy,
                                          float2& dz) {
  dx = __fadd2_rn(make_float2(q.x, q.x), nx);
  dy = __fadd2_rn(make_float2(q.y, q.y), ny);
  if (DIM == 3) {
    dz = __fadd2_rn(make_float2(q.z, q.z), nz);
    return __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  }
  dz = make_float2(0.f, 0.f);
  return __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
}

// One CTA of W warps per cell (grid-stride over the cells). The stencil
// entries are shared among the warps 32 at a time; each warp appends the
// particles of its entries that lie within sqrt(ball2) of the cell centre,
// shifted to the cell's frame (x_j + s_o), to the staged list. Then warp w
// sweeps home particles w, w + W, ... against it (distance (x_j + s_o) - x_i).
// Particles whose original index is not above the smallest of the cell's own
// are not staged: no pair with j > i of this cell needs them.
// COUNT: count[a] = pairs with j > a; a cell whose list does not fit gets
// flag 1 (else 0) and is listed in fcells. FILL: flagged cells are skipped; the staged list is ordered
// by original index (radix sort of its indices), so a particle's pairs with
// j > a come from a suffix of that order in ascending j and are written in
// order, coalesced, as the ballot finds them.
template <int DIM, bool FILL>
__global__ void __launch_bounds__(256, 5) k_pairs_cell(const __grid_constant__ SweepArgs A,
                                                                               float ball2, int cap,
                                                                               unsigned char* __restrict__ flag,
                                                                               int* __restrict__ fcells,
                                                                               int* __restrict__ nfcells,
                                                                               int* __restrict__ count,
                                                                               const long long* __restrict__ start,
                                                                               int* __restrict__ pi_out,
                                                                               int* __restrict__ pj_out,
                                                                               float* __restrict__ pd_out) {
  constexpr int W = 8;
  extern __shared__ float4 smem[];
  float4* st = smem;           // staged neighbourhood: (x, y, z in the cell's frame, original index)
  float4* stab = st + cap;     // stencil: (s_x, s_y, s_z, dx | dy << 10 | dz << 20)
  int* scal = reinterpret_cast<int*>(stab + A.noff);  // [0] staged count, [1..2] index range, [4..] warp sums
  unsigned short* cnt = reinterpret_cast<unsigned short*>(scal + 16);  // FILL: radix counters and slots
  unsigned short* rs0 = cnt + 256 * W;
  unsigned short* rs1 = rs0 + cap;
  stencil_to_smem(A, stab);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int ncells = A.nx * A.ny * A.nz;
  for (int c = blockIdx.x; c < ncells; c += gridDim.x) {
    const int h0 = __ldg(A.cell_start + c), h1 = __ldg(A.cell_start + c + 1);
    if (h1 == h0) continue;
    if (FILL && flag[c]) continue;
    const int cx = c % A.nx, cy = (c / A.nx) % A.ny, cz = c / (A.nx * A.ny);
    if (threadIdx.x == 0) scal[0] = 0;
    // the smallest original index among the cell's particles (each warp on
    // its own): a staged particle of index <= amin pairs with none of them
    // under j > i, so neither pass stages it
    int amin = INT_MAX;
    for (int p = h0 + lane; p < h1; p += 32) amin = min(amin, __float_as_int(__ldg(&A.xs[p].w)));
    amin = __reduce_min_sync(0xffffffffu, amin);
    __syncthreads();
    // the stencil dealt evenly to the warps (E entries each per round, at most
    // 32): at 32 per warp the 125 entries of a full stencil at lcell 2 would
    // keep four of the eight warps waiting while the others stage
    const int E = min(32, (A.noff + W - 1) / W);
    for (int k0 = warp * E; k0 < A.noff; k0 += E * W) {
      const Chunk ch = chunk_ranges<DIM>(A, stab, k0, lane, cx, cy, cz, 0.f, 0.f, 0.f, E);
      for (int t0 = 0; t0 < ch.total; t0 += 32) {
        const int t = t0 + lane;
        float ax, ay, az;
        const int j = chunk_candidate(ch, t, ax, ay, az);
        bool keep = false;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < ch.total) {
          const float4 q = __ldg(&A.xs[j]);
          v.x = q.x + ax;
          v.y = q.y + ay;
          v.z = DIM == 3 ? q.z + az : 0.f;
          v.w = q.w;
          keep = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z)) < ball2 && __float_as_int(q.w) > amin;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(scal, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
          const int e = base + __popc(m & lt);
          if (e < cap) st[e] = v;
        }
      }
    }
    __syncthreads();
    const int S = scal[0];
    if (S <= cap) {
      unsigned short* slots = rs0;
      int kmin = 0;
      if (FILL) stage_radix<W>(st, S, rs0, rs1, cnt, scal, slots, kmin);
      if (!FILL) {
        // COUNT: two home particles per warp share each staged load; the
        // distance of each (particle, candidate) is computed as in the fill pass.
        for (int p = h0 + 2 * warp; p < h1; p += 2 * W) {
          const bool two = p + 1 < h1;
          const float4 pa = A.xs[p];
          const float4 pb = two ? A.xs[p + 1] : pa;
          const int a0 = __float_as_int(pa.w), a1 = two ? __float_as_int(pb.w) : INT_MAX;
          const float2 nx = make_float2(-pa.x, -pb.x), ny = make_float2(-pa.y, -pb.y),
                       nz = make_float2(-pa.z, -pb.z);
          int L0 = 0, L1 = 0;  // per lane, summed over the warp at the end
#pragma unroll 2
          for (int t = lane; t < S; t += 32) {
            const float4 q = st[t];
            const int jo = __float_as_int(q.w);
            float2 dx, dy, dz;
            const float2 d2 = pair_d2<DIM>(q, nx, ny, nz, dx, dy, dz);
            L0 += (jo > a0 && d2.x < A.rc2) ? 1 : 0;
            L1 += (jo > a1 && d2.y < A.rc2) ? 1 : 0;
          }
          L0 = __reduce_add_sync(0xffffffffu, L0);
          L1 = __reduce_add_sync(0xffffffffu, L1);
          if (lane == 0) {
            count[a0] = L0;
            if (two) count[a1] = L1;
          }
        }
      }
      if (FILL) {
        // FILL: two home particles per warp; the sweep starts at the earlier of
        // their suffixes (entries before a particle's own suffix fail j > i) and
        // each particle's kept pairs are written in order from its own ballot.
        for (int p = h0 + 2 * warp; p < h1; p += 2 * W) {
          const bool two = p + 1 < h1;
          const float4 pa = A.xs[p];
          const float4 pb = two ? A.xs[p + 1] : pa;
          const int a0 = __float_as_int(pa.w), a1 = two ? __float_as_int(pb.w) : INT_MAX;
          int f0 = 0, f1 = S;  // first position (in index order) with index > a0, a1
          {
            const unsigned ka = a0 >= kmin ? (unsigned)(a0 - kmin) : 0u;
            int lo = 0, hi = S;
            while (a0 >= kmin && lo < hi) {
              const int mid = (lo + hi) >> 1;
              if ((unsigned)(__float_as_int(st[slots[mid]].w) - kmin) > ka) hi = mid;
              else lo = mid + 1;
            }
            f0 = a0 >= kmin ? lo : 0;
          }
          if (two) {
            const unsigned kb = a1 >= kmin ? (unsigned)(a1 - kmin) : 0u;
            int lo = 0, hi = S;
            while (a1 >= kmin && lo < hi) {
              const int mid = (lo + hi) >> 1;
              if ((unsigned)(__float_as_int(st[slots[mid]].w) - kmin) > kb) hi = mid;
              else lo = mid + 1;
            }
            f1 = a1 >= kmin ? lo : 0;
          }
          const int c0 = __ldg(count + a0), c1 = two ? __ldg(count + a1) : 0;
          const long long b0 = __ldg(start + a0), b1 = two ? __ldg(start + a1) : 0;
          const float2 nx = make_float2(-pa.x, -pb.x), ny = make_float2(-pa.y, -pb.y),
                       nz = make_float2(-pa.z, -pb.z);
          int L0 = 0, L1 = 0;
#pragma unroll 2
          for (int t0 = min(f0, f1); t0 < S; t0 += 32) {
            const int t = t0 + lane;
            bool k0 = false, k1 = false;
            int jo = 0;
            float d20 = 0.f, d21 = 0.f;
            if (t < S) {
              const float4 q = st[(int)slots[t]];
              jo = __float_as_int(q.w);
              float2 dx, dy, dz;
              const float2 d2 = pair_d2<DIM>(q, nx, ny, nz, dx, dy, dz);
              d20 = d2.x;
              d21 = d2.y;
              k0 = jo > a0 && d20 < A.rc2;
              k1 = jo > a1 && d21 < A.rc2;
            }
            const unsigned m0 = __ballot_sync(0xffffffffu, k0), m1 = __ballot_sync(0xffffffffu, k1);
            if (k0) {
              const int e = L0 + __popc(m0 & lt);
              if (e < c0) {
                pi_out[b0 + e] = a0;
                pj_out[b0 + e] = jo;
                pd_out[b0 + e] = d20 * rsqrt_nr(d20);
              }
            }
            if (k1) {
              const int e = L1 + __popc(m1 & lt);
              if (e < c1) {
                pi_out[b1 + e] = a1;
                pj_out[b1 + e] = jo;
                pd_out[b1 + e] = d21 * rsqrt_nr(d21);
              }
            }
            L0 += __popc(m0);
            L1 += __popc(m1);
          }
        }
      }
    }
    if (!FILL && threadIdx.x == 0) {
      flag[c] = S > cap ? 1 : 0;
      if (S > cap) fcells[atomicAdd(nfcells, 1)] = c;
    }
    __syncthreads();
  }
}

size_t pairs_cell_smem(int noff, bool fill, int cap) {
  const size_t head = (size_t)(cap + noff) * sizeof(float4) + 16 * sizeof(int);
  return fill ? head + 256 * 8 * sizeof(unsigned short) + 2 * (size_t)cap * sizeof(unsigned short) : head;
}

template <int DIM, bool FILL>
static int launch_cell(const SweepArgs& A, float ball2, int cap, unsigned char* flag, int* fcells, int* nfcells,
                       int* count, const long long* start, int* pi, int* pj, float* pd, cudaStream_t s) {
  static DevCache ready;  // shared-memory limit raised on this device
  if (cap < 32 || cap > kStageMax) return CL_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CL_ERR_CUDA;
  if (!ready.get(dev)) {
    if (cudaFuncSetAttribute(k_pairs_cell<DIM, FILL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pairs_cell_smem(kMaxOff, FILL, kStageMax)) != cudaSuccess)
      return CL_ERR_CUDA;
    ready.put(dev, 1);
  }
  const size_t smem = pairs_cell_smem(A.noff, FILL, cap);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pairs_cell<DIM, FILL>, 256, smem) !=
          cudaSuccess ||
      per < 1)
    return CL_ERR_CUDA;
  long long blocks = (long long)sms * per;
  const long long ncells = (long long)A.nx * A.ny * A.nz;
  if (blocks > ncells) blocks = ncells;
  k_pairs_cell<DIM, FILL><<<(int)blocks, 256, smem, s>>>(A, ball2, cap, flag, fcells, nfcells, count,
                                                                      start, pi, pj, pd);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int launch_pairs_count(const SweepArgs& A, int dim, float ball2, int cap, unsigned char* flag, int* fcells,
                       int* nfcells, int* count, cudaStream_t s) {
  if (A.n <= 0) return CL_OK;
  if (cudaMemsetAsync(nfcells, 0, sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  const int e = dim == 3 ? launch_cell<3, false>(A, ball2, cap, flag, fcells, nfcells, count, nullptr, nullptr,
                                                 nullptr, nullptr, s)
                         : launch_cell<2, false>(A, ball2, cap, flag, fcells, nfcells, count, nullptr, nullptr,
                                                 nullptr, nullptr, s);
  if (e) return e;
  if (dim == 3) k_pairs_count<3><<<152 * 4, 256, 0, s>>>(A, fcells, nfcells, count);
  else k_pairs_count<2><<<152 * 4, 256, 0, s>>>(A, fcells, nfcells, count);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

static int launch_sort_long(const int* longs, const int* nlong, const int* count, const long long* start, int* pj,
                            float* pd, cudaStream_t s) {
  k_pairs_sort_long<<<152, 1024, 0, s>>>(longs, nlong, count, start, pj, pd);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int launch_pairs_fill(const SweepArgs& A, int dim, float ball2, int cap, const unsigned char* flag, const int* fcells,
                      const int* nfcells, const int* count, const long long* start, int* pi, int* pj, float* pd, int* longs,
                      int* nlong, cudaStream_t s) {
  if (A.n <= 0) return CL_OK;
  unsigned char* fl = const_cast<unsigned char*>(flag);  // only read by the fill pass
  int* cn = const_cast<int*>(count);                     // likewise
  const int e = dim == 3 ? launch_cell<3, true>(A, ball2, cap, fl, nullptr, nullptr, cn, start, pi, pj, pd, s)
                         : launch_cell<2, true>(A, ball2, cap, fl, nullptr, nullptr, cn, start, pi, pj, pd, s);
  if (e) return e;
  const size_t dyn = (size_t)A.noff * sizeof(float4);
  if (cudaMemsetAsync(nlong, 0, sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  if (dim == 3)
    k_pairs_fill_sorted<3><<<152 * 6, 32 * kFillWarps, dyn, s>>>(A, fcells, nfcells, count, start, pi, pj, pd, longs,
                                                                nlong);
  else
    k_pairs_fill_sorted<2><<<152 * 6, 32 * kFillWarps, dyn, s>>>(A, fcells, nfcells, count, start, pi, pj, pd, longs,
                                                                nlong);
  if (cudaGetLastError() != cudaSuccess) return CL_ERR_CUDA;
  return launch_sort_long(longs, nlong, count, start, pj, pd, s);
}

int launch_pairs_sort(int n, const int* count, const long long* start, int* pj, float* pd, int* longs, int* nlong,
                      cudaStream_t s) {
  if (n <= 0) return CL_OK;
  if (cudaMemsetAsync(nlong, 0, sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  int blocks = (n + kSortWarps - 1) / kSortWarps;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_pairs_sort<<<blocks, 32 * kSortWarps, 0, s>>>(n, count, start, pj, pd, longs, nlong);
  if (cudaGetLastError() != cudaSuccess) return CL_ERR_CUDA;
  return launch_sort_long(longs, nlong, count, start, pj, pd, s);
}

}  // namespace clk
