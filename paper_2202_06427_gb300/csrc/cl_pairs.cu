// cl_pairs.cu -- the i<j neighbour list (Sec. 4.1: "the lists of pairs of
// particles within a cutoff"), sorted by (i, j), with the FP32 distance.
//
//   k_pairs_count  full-shell sweep; the thread of particle i counts its
//                  pairs with j > i (original indices), so every pair is
//                  counted once, by its smaller index, without atomics
//   (scan)         exclusive prefix sum of the counts in original order:
//                  segment of i = [start[i], start[i] + count[i])
//   k_pairs_fill   the same sweep writes (i, j, r) into i's segment, in the
//                  order the stencil visits the neighbour cells
//   k_pairs_sort   one warp per segment: bitonic sort by j in shared memory
//
// The sweep visits the pair-images of a particle; the list is only defined
// when each pair has at most one image within rc (rc <= w_min / 2), which the
// host checks before launching.
#include <climits>

#include "cl_sweep.cuh"

namespace clk {

struct RedPairCount {
  static constexpr bool kFull = true;
  struct Acc { int a; int n; };
  __device__ void init(Acc& x) const { x.n = 0; }
  __device__ void hit(Acc& x, float, float, float, float, int j) const { x.n += (j > x.a) ? 1 : 0; }
};

struct RedPairFill {
  static constexpr bool kFull = true;
  int* pi;
  int* pj;
  float* pd;
  struct Acc { int a; int pos; };
  __device__ void init(Acc&) const {}
  __device__ void hit(Acc& x, float, float, float, float d2, int j) const {
    if (j > x.a) {
      pi[x.pos] = x.a;
      pj[x.pos] = j;
      pd[x.pos] = d2 * rsqrt_nr(d2);
      x.pos++;
    }
  }
};

template <int DIM>
__global__ void __launch_bounds__(256) k_pairs_count(const __grid_constant__ SweepArgs A, int* __restrict__ count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= A.n) return;
  RedPairCount red;
  RedPairCount::Acc acc;
  red.init(acc);
  acc.a = __float_as_int(A.xs[p].w);
  float4 pi;
  sweep_particle<DIM>(A, red, acc, p, pi);
  count[acc.a] = acc.n;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_pairs_fill(const __grid_constant__ SweepArgs A, const int* __restrict__ start,
                                                    int* pi_out, int* pj_out, float* pd_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= A.n) return;
  RedPairFill red;
  red.pi = pi_out;
  red.pj = pj_out;
  red.pd = pd_out;
  RedPairFill::Acc acc;
  acc.a = __float_as_int(A.xs[p].w);
  acc.pos = start[acc.a];
  float4 pi;
  sweep_particle<DIM>(A, red, acc, p, pi);
}

constexpr int kSortWarps = 4;

// One warp per segment (grid-stride): bitonic sort of up to kMaxSegment keys
// (j, distinct within a segment) with their distances, in shared memory.
__global__ void __launch_bounds__(32 * kSortWarps) k_pairs_sort(int n, const int* __restrict__ count,
                                                               const int* __restrict__ start, int* __restrict__ pj,
                                                               float* __restrict__ pd) {
  __shared__ int sk[kSortWarps][kMaxSegment];
  __shared__ float sv[kSortWarps][kMaxSegment];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* K = sk[warp];
  float* V = sv[warp];
  for (int a = blockIdx.x * kSortWarps + warp; a < n; a += gridDim.x * kSortWarps) {
    const int L = count[a];
    if (L <= 1 || L > kMaxSegment) continue;  // the host refuses lists with longer segments
    const int base = start[a];
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

static int blocks_of(int n) { return n > 0 ? (n + 255) / 256 : 1; }

int launch_pairs_count(const SweepArgs& A, int dim, int* count, cudaStream_t s) {
  if (A.n > 0) {
    if (dim == 3) k_pairs_count<3><<<blocks_of(A.n), 256, 0, s>>>(A, count);
    else k_pairs_count<2><<<blocks_of(A.n), 256, 0, s>>>(A, count);
  }
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int launch_pairs_fill(const SweepArgs& A, int dim, const int* start, int* pi, int* pj, float* pd, cudaStream_t s) {
  if (A.n > 0) {
    if (dim == 3) k_pairs_fill<3><<<blocks_of(A.n), 256, 0, s>>>(A, start, pi, pj, pd);
    else k_pairs_fill<2><<<blocks_of(A.n), 256, 0, s>>>(A, start, pi, pj, pd);
  }
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int launch_pairs_sort(int n, const int* count, const int* start, int* pj, float* pd, cudaStream_t s) {
  if (n > 0) {
    int blocks = (n + kSortWarps - 1) / kSortWarps;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_pairs_sort<<<blocks, 32 * kSortWarps, 0, s>>>(n, count, start, pj, pd);
  }
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

}  // namespace clk
