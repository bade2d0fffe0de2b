// cl_sweep.cu -- the neighbour-cell sweep (Sec. 2.8: "a loop over the cells
// is performed, and the interactions of the particle of each cell with the
// particles of the neighboring cells are computed") with the reduction fused
// into the loop, and the fixed-order FP64 final reduction of the per-CTA
// partial outputs (Sec. 2.8: each worker updates its own copy of the output;
// the copies are summed at the end).
//
// Mapping: one thread per cell-sorted particle i. The thread walks the
// stencil of its cell (own cell first), and for every neighbour cell scans
// that cell's contiguous range of the sorted array. Threads of a warp hold
// consecutive sorted particles, mostly of one cell, so they read the same
// neighbour particles at the same time (one broadcast load serves the warp).
//
// Half shell (count, sum 1/r, energy, histogram): lexicographically positive
// offsets plus the own cell with j after i in sorted order; each pair-image
// once. Full shell (forces, virial, backward): all offsets; each pair-image
// twice, once from each end, so a thread owns the force on its particle and
// writes it once, without atomics.
//
// Precision: pair math in FP32 on cell-centred coordinates; per-thread FP32
// partial sums (a few hundred terms); FP64 from the warp level up; partials
// per CTA reduced in a fixed order.
#include <algorithm>
#include <cmath>

#include "cl_sweep.cuh"

namespace clk {

// Particle p of the sweep, or A.n (none) when flag is given and p's cell is
// not flagged: a neighbourhood sweep took that cell (3D).
__device__ __forceinline__ int flagged_particle(const SweepArgs& A, const unsigned char* __restrict__ flag, int p) {
  if (!flag || p >= A.n) return p;
  const unsigned cc = A.cellc[p];
  const int c = (int)(cc & 1023u) + A.nx * ((int)((cc >> 10) & 1023u) + A.ny * (int)(cc >> 20));
  return flag[c] ? p : A.n;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_sweep_count(const __grid_constant__ SweepArgs A, unsigned long long* out,
                                                     const unsigned char* __restrict__ flag) {
  RedCount red;
  RedCount::Acc acc;
  red.init(acc);
  float4 pi;
  sweep_particle<DIM>(A, red, acc, flagged_particle(A, flag, blockIdx.x * blockDim.x + threadIdx.x), pi);
  unsigned v = acc.n;
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}

// Scalar FP64 partial per CTA: sum 1/r (kind 0) or shifted-force energy (kind 1).
template <int DIM, int KIND>
__global__ void __launch_bounds__(256) k_sweep_scalar(const __grid_constant__ SweepArgs A, double* partials,
                                                      const unsigned char* __restrict__ flag) {
  float4 pi;
  double v[1];
  const int p = flagged_particle(A, flag, blockIdx.x * blockDim.x + threadIdx.x);
  if (KIND == 0) {
    RedSumInvR red;
    RedSumInvR::Acc acc;
    red.init(acc);
    sweep_particle<DIM>(A, red, acc, p, pi);
    v[0] = (double)acc.s;
  } else {
    RedEnergy red;
    red.irc = A.irc;
    RedEnergy::Acc acc;
    red.init(acc);
    sweep_particle<DIM>(A, red, acc, p, pi);
    v[0] = (double)acc.e;
  }
  block_sum_store<1>(v, partials + blockIdx.x);
}

template <int DIM>
__global__ void __launch_bounds__(256) k_sweep_hist(const __grid_constant__ SweepArgs A, int nbins, float rmax,
                                                    unsigned long long* __restrict__ hist,
                                                    const unsigned char* __restrict__ flag) {
  extern __shared__ unsigned sh[];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0u;
  __syncthreads();
  RedHist red;
  red.nbins = nbins;
  red.rmax = rmax;
  red.scale = (float)nbins / rmax;
  red.sh = sh;
  RedHist::Acc acc;
  float4 pi;
  sweep_particle<DIM>(A, red, acc, flagged_particle(A, flag, blockIdx.x * blockDim.x + threadIdx.x), pi);
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

// Full shell: forces (FP32, original order), and per CTA the energy (x1/2) and
// the symmetric accumulator of the virial. MODE 0: forward forces; MODE 1:
// backward, grad_pos = -g F in FP64 plus X = sum x_raw (x) F for the box gradient.
template <int DIM, int MODE>
__global__ void __launch_bounds__(256) k_sweep_force(const __grid_constant__ SweepArgs A, float* __restrict__ forces,
                                                     double* __restrict__ grad, const double* __restrict__ gE,
                                                     const double* __restrict__ pos, double* __restrict__ partials) {
  RedForce<DIM, MODE == 0> red;
  red.irc = A.irc;
  red.irc2 = A.irc2;
  typename RedForce<DIM, MODE == 0>::Acc acc;
  red.init(acc);
  float4 pi;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = sweep_particle<DIM>(A, red, acc, p, pi);
  constexpr int NW = (DIM == 3) ? kVirN3 : kVirN2;
  constexpr int NV = (MODE == 0) ? 1 + NW : NW + DIM * DIM;
  double v[NV];
  // symmetric components in the order xx, xy, (xz), yy, (yz), (zz)
  if (DIM == 3) {
    v[0] = acc.w[0]; v[1] = acc.w[1]; v[2] = acc.w[2]; v[3] = acc.w[3]; v[4] = acc.w[4]; v[5] = acc.w[5];
  } else {
    v[0] = acc.w[0]; v[1] = acc.w[1]; v[2] = acc.w[3];
  }
  if (MODE == 0) {
    v[NW] = 0.5 * (double)acc.e;
    if (live) {
      const int i = __float_as_int(pi.w);
#pragma unroll
      for (int a = 0; a < DIM; ++a) forces[(size_t)i * DIM + a] = acc.f[a];
    }
  } else {
#pragma unroll
    for (int k = NW; k < NV; ++k) v[k] = 0.0;
    if (live) {
      const int i = __float_as_int(pi.w);
      const double g = *gE;
#pragma unroll
      for (int a = 0; a < DIM; ++a) grad[(size_t)i * DIM + a] = -g * (double)acc.f[a];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double xa = pos[(size_t)i * DIM + a];
#pragma unroll
        for (int b = 0; b < DIM; ++b) v[NW + a * DIM + b] = xa * (double)acc.f[b];
      }
    }
  }
  block_sum_store<NV>(v, partials + (size_t)blockIdx.x * NV);
}

// Packed 3D counterparts of the energy and force sweeps (same outputs).
__global__ void __launch_bounds__(256) k_sweep2_energy(const __grid_constant__ SweepArgs A, double* partials) {
  Red2Energy red;
  red.irc = A.irc;
  Red2Energy::Acc acc;
  red.init(acc);
  float4 pi;
  sweep_particle2(A, red, acc, blockIdx.x * blockDim.x + threadIdx.x, pi);
  double v[1] = {(double)acc.e.x + (double)acc.e.y};
  block_sum_store<1>(v, partials + blockIdx.x);
}

// Packed 3D counterparts of the count, sum 1/r and histogram sweeps.
__global__ void __launch_bounds__(256) k_sweep2_count(const __grid_constant__ SweepArgs A, unsigned long long* out,
                                                      const unsigned char* __restrict__ flag) {
  Red2Count red;
  Red2Count::Acc acc;
  red.init(acc);
  float4 pi;
  sweep_particle2(A, red, acc, flagged_particle(A, flag, blockIdx.x * blockDim.x + threadIdx.x), pi);
  unsigned v = acc.n;
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}

__global__ void __launch_bounds__(256) k_sweep2_suminvr(const __grid_constant__ SweepArgs A, double* partials,
                                                        const unsigned char* __restrict__ flag) {
  Red2SumInvR red;
  Red2SumInvR::Acc acc;
  red.init(acc);
  float4 pi;
  sweep_particle2(A, red, acc, flagged_particle(A, flag, blockIdx.x * blockDim.x + threadIdx.x), pi);
  double v[1] = {(double)acc.s.x + (double)acc.s.y};
  block_sum_store<1>(v, partials + blockIdx.x);
}

__global__ void __launch_bounds__(256) k_sweep2_hist(const __grid_constant__ SweepArgs A, int nbins, float scale2,
                                                     float xlim, unsigned long long* __restrict__ hist,
                                                     const unsigned char* __restrict__ flag) {
  extern __shared__ unsigned sh[];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0u;
  __syncthreads();
  Red2Hist red;
  red.scale2 = scale2;
  red.xlim = xlim;
  red.sh = sh;
  Red2Hist::Acc acc;
  float4 pi;
  sweep_particle2(A, red, acc, flagged_particle(A, flag, blockIdx.x * blockDim.x + threadIdx.x), pi);
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

// Histogram parameters of the packed sweeps: scale^2 = (nbins / rmax)^2 and
// the bin-coordinate limit min(nbins, rc nbins / rmax).
static void hist_params(const SweepArgs& A, int nbins, float rmax, float* scale2, float* xlim) {
  const double sc = (double)nbins / (double)rmax;
  *scale2 = (float)(sc * sc);
  *xlim = (float)std::min((double)nbins, std::sqrt((double)A.rc2) * sc);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_sweep2_force(const __grid_constant__ SweepArgs A, float* __restrict__ forces,
                                                      double* __restrict__ grad, const double* __restrict__ gE,
                                                      const double* __restrict__ pos, double* __restrict__ partials) {
  Red2Force<MODE == 0> red;
  red.irc = A.irc;
  red.irc2 = A.irc2;
  typename Red2Force<MODE == 0>::Acc acc;
  red.init(acc);
  float4 pi;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = sweep_particle2(A, red, acc, p, pi);
  const float F[3] = {-acc.tx, -acc.ty, -acc.tz};
  constexpr int NV = (MODE == 0) ? 1 + kVirN3 : kVirN3 + 9;
  double v[NV];
  // the symmetric accumulator of the scalar kernels is sum fs r(x)r = -(sum fsn r(x)r)
  float v6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (live) red.virial(acc, pi.x, pi.y, pi.z, v6);
#pragma unroll
  for (int k = 0; k < 6; ++k) v[k] = -(double)v6[k];
  if (MODE == 0) {
    v[kVirN3] = 0.5 * ((double)acc.e.x + (double)acc.e.y);
    if (live) {
      const int i = __float_as_int(pi.w);
#pragma unroll
      for (int a = 0; a < 3; ++a) forces[(size_t)i * 3 + a] = F[a];
    }
  } else {
#pragma unroll
    for (int k = kVirN3; k < NV; ++k) v[k] = 0.0;
    if (live) {
      const int i = __float_as_int(pi.w);
      const double g = *gE;
#pragma unroll
      for (int a = 0; a < 3; ++a) grad[(size_t)i * 3 + a] = -g * (double)F[a];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double xa = pos[(size_t)i * 3 + a];
#pragma unroll
        for (int b = 0; b < 3; ++b) v[kVirN3 + a * 3 + b] = xa * (double)F[b];
      }
    }
  }
  block_sum_store<NV>(v, partials + (size_t)blockIdx.x * NV);
}

// ----------------------------------------------------------- final reduce

struct FinalArgs {
  int mode;          // 0 sum 1/r, 1 energy, 2 forward forces (energy + virial), 3 backward, 4 energy + backward
  int dim;
  double hinv[9];    // 3x3
  double* out_scalar;
  double* out_virial;   // dim*dim or null
  double* out_gradbox;  // dim*dim or null
  const double* gE;
};

// Turns the summed partials into the caller's outputs (one thread).
__device__ void final_assemble(const FinalArgs& F, const double* sums) {
  const int d = F.dim;
  if (F.mode <= 1) {
    *F.out_scalar = sums[0];
    return;
  }
  const int NW = (d == 3) ? kVirN3 : kVirN2;
  double S[3][3];
  if (d == 3) {
    const int map[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) S[a][b] = sums[map[a][b]];
  } else {
    S[0][0] = sums[0]; S[0][1] = S[1][0] = sums[1]; S[1][1] = sums[2];
  }
  double W[3][3];
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) W[a][b] = -0.5 * S[a][b];
  if (F.out_virial)
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) F.out_virial[a * d + b] = W[a][b];
  if (F.mode == 2) {
    if (F.out_scalar) *F.out_scalar = sums[NW];
    return;
  }
  if (F.mode == 4 && F.out_scalar) *F.out_scalar = sums[NW + d * d];
  // dE/dH at fixed positions = H^-T (X - W), X = sum_i x_i (x) F_i
  const double g = *F.gE;
  if (F.out_gradbox) {
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += F.hinv[k * 3 + a] * (sums[NW + k * d + b] - W[k][b]);
        F.out_gradbox[a * d + b] = g * s;
      }
  }
}

// Sums partials[nblocks][nv] in a fixed order into sums[nv]: CTA k sums
// component k (strided per thread, then a fixed tree). The last CTA to finish
// (a completion counter in the last word of sums, which holds 32 doubles,
// zero between launches and reset by that CTA) turns the sums into the
// caller's outputs, so the final step takes one launch.
__global__ void __launch_bounds__(256) k_final_sum(const double* __restrict__ partials, int nblocks, int nv,
                                                   double* __restrict__ sums, const __grid_constant__ FinalArgs F) {
  __shared__ double sm[256];
  __shared__ bool last;
  const int k = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 256) s += partials[(size_t)b * nv + k];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[k] = sm[0];
    __threadfence();
    unsigned long long* done = reinterpret_cast<unsigned long long*>(sums + 31);
    last = atomicAdd(done, 1ull) == (unsigned long long)(nv - 1);
    if (last) {
      *done = 0ull;
      double tot[32];  // the other CTAs' sums, past L1
      for (int q = 0; q < nv; ++q) tot[q] = __ldcg(sums + q);
      final_assemble(F, tot);
    }
  }
}

int finish_reduction(int final_mode, int dim, const double* hinv, int nblocks, int nv, const double* partials,
                     double* sums, double* scalar, double* virial, double* gradbox, const double* gE,
                     cudaStream_t s) {
  FinalArgs F;
  memset(&F, 0, sizeof(F));
  F.mode = final_mode;
  F.dim = dim;
  if (hinv)
    for (int k = 0; k < 9; ++k) F.hinv[k] = hinv[k];
  F.out_scalar = scalar;
  F.out_virial = virial;
  F.out_gradbox = gradbox;
  F.gE = gE;
  if (nv < 1 || nv > 31) return CL_ERR_INVALID_ARG;  // sums[31] is the completion counter
  k_final_sum<<<nv, 256, 0, s>>>(partials, nblocks, nv, sums, F);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

__global__ void __launch_bounds__(256) k_scale(const double* __restrict__ g, const double* __restrict__ in,
                                              double* __restrict__ out, long long count) {
  const double s = *g;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count; k += (long long)gridDim.x * blockDim.x)
    out[k] = s * in[k];
}

int launch_scale(const double* g, const double* in, double* out, long long count, cudaStream_t s) {
  if (count <= 0) return CL_OK;
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scale<<<(int)blocks, 256, 0, s>>>(g, in, out, count);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

// Candidate pairs the half-shell sweep tests: for each cell c,
// n_c (n_c - 1)/2 + n_c sum_{o != 0} n_{c+o}.
__global__ void __launch_bounds__(256) k_candidates(const __grid_constant__ SweepArgs A, long long ncells,
                                                    unsigned long long* out) {
  unsigned long long acc = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncells;
       c += (long long)gridDim.x * blockDim.x) {
    const long long nc = A.cell_start[c + 1] - A.cell_start[c];
    if (nc == 0) continue;
    const int cx = (int)(c % A.nx), cy = (int)((c / A.nx) % A.ny), cz = (int)(c / ((long long)A.nx * A.ny));
    unsigned long long s = 0;
    for (int k = 1; k < A.noff; ++k) {
      const Off o = A.off[k];
      int x2 = cx + o.dx; x2 -= (x2 >= A.nx) ? A.nx : 0;
      int y2 = cy + o.dy; y2 -= (y2 >= A.ny) ? A.ny : 0;
      int z2 = cz + o.dz; z2 -= (z2 >= A.nz) ? A.nz : 0;
      const long long c2 = x2 + (long long)A.nx * (y2 + (long long)A.ny * z2);
      s += (unsigned long long)(A.cell_start[c2 + 1] - A.cell_start[c2]);
    }
    acc += (unsigned long long)nc * s + (unsigned long long)(nc * (nc - 1) / 2);
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// ------------------------------------------------------------ host entry --

static int blocks_for(int n) { return n > 0 ? (n + 255) / 256 : 1; }

// Per-CTA partials (16 doubles each) for the one-thread-per-particle sweeps, and
// for the persistent neighbourhood sweep (at most kMaxPersistent CTAs)
// followed by its one-thread-per-particle companion.
constexpr int kMaxPersistent = 4096;
int sweep_partials_needed(int n) { return (blocks_for(n) + kMaxPersistent) * 16; }

int launch_count(const SweepArgs& A, int dim, unsigned long long* out, cudaStream_t s) {
  if (cudaMemsetAsync(out, 0, sizeof(unsigned long long), s) != cudaSuccess) return CL_ERR_CUDA;
  if (A.n > 0) {
    if (dim == 3) k_sweep2_count<<<blocks_for(A.n), 256, 0, s>>>(A, out, nullptr);
    else k_sweep_count<2><<<blocks_for(A.n), 256, 0, s>>>(A, out, nullptr);
  }
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int launch_scalar(const SweepArgs& A, int dim, int kind, double* partials, double* sums, double* out,
                  cudaStream_t s) {
  const int nb = blocks_for(A.n);
  if (A.n > 0) {
    if (dim == 3) {
      if (kind == 0) k_sweep2_suminvr<<<nb, 256, 0, s>>>(A, partials, nullptr);
      else k_sweep2_energy<<<nb, 256, 0, s>>>(A, partials);
    } else {
      if (kind == 0) k_sweep_scalar<2, 0><<<nb, 256, 0, s>>>(A, partials, nullptr);
      else k_sweep_scalar<2, 1><<<nb, 256, 0, s>>>(A, partials, nullptr);
    }
  } else {
    if (cudaMemsetAsync(partials, 0, sizeof(double), s) != cudaSuccess) return CL_ERR_CUDA;
  }
  return finish_reduction(kind, dim, nullptr, A.n > 0 ? nb : 1, 1, partials, sums, out, nullptr, nullptr, nullptr, s);
}

int launch_hist(const SweepArgs& A, int dim, int nbins, float rmax, unsigned long long* hist, cudaStream_t s) {
  if (cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * nbins, s) != cudaSuccess) return CL_ERR_CUDA;
  const size_t smem = sizeof(unsigned) * nbins;
  if (A.n > 0) {
    if (dim == 3) {
      float scale2, xlim;
      hist_params(A, nbins, rmax, &scale2, &xlim);
      k_sweep2_hist<<<blocks_for(A.n), 256, smem, s>>>(A, nbins, scale2, xlim, hist, nullptr);
    }
    else {
      k_sweep_hist<2><<<blocks_for(A.n), 256, smem, s>>>(A, nbins, rmax, hist, nullptr);
    }
  }
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int flagged_blocks(int n) { return blocks_for(n); }

int launch_count_flagged(const SweepArgs& A, const unsigned char* flag, unsigned long long* out, cudaStream_t s) {
  if (A.n > 0) k_sweep2_count<<<blocks_for(A.n), 256, 0, s>>>(A, out, flag);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int launch_suminvr_flagged(const SweepArgs& A, const unsigned char* flag, double* partials, cudaStream_t s) {
  if (A.n > 0) k_sweep2_suminvr<<<blocks_for(A.n), 256, 0, s>>>(A, partials, flag);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

int launch_hist_flagged(const SweepArgs& A, const unsigned char* flag, int nbins, float rmax,
                        unsigned long long* hist, cudaStream_t s) {
  if (A.n > 0) {
    float scale2, xlim;
    hist_params(A, nbins, rmax, &scale2, &xlim);
    k_sweep2_hist<<<blocks_for(A.n), 256, sizeof(unsigned) * nbins, s>>>(A, nbins, scale2, xlim, hist, flag);
  }
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

// mode 0: forward (forces, energy, virial); mode 1: backward (grad_pos, grad_box, virial).
int launch_force(const SweepArgs& A, int dim, int mode, const double* hinv, float* forces, double* grad,
                 const double* gE, const double* pos, double* partials, double* sums, double* energy,
                 double* virial, double* gradbox, cudaStream_t s) {
  const int nb = blocks_for(A.n);
  const int NW = dim == 3 ? kVirN3 : kVirN2;
  const int NV = mode == 0 ? 1 + NW : NW + dim * dim;
  if (A.n > 0) {
    if (dim == 3) {
      if (mode == 0) k_sweep2_force<0><<<nb, 256, 0, s>>>(A, forces, grad, gE, pos, partials);
      else k_sweep2_force<1><<<nb, 256, 0, s>>>(A, forces, grad, gE, pos, partials);
    } else {
      if (mode == 0) k_sweep_force<2, 0><<<nb, 256, 0, s>>>(A, forces, grad, gE, pos, partials);
      else k_sweep_force<2, 1><<<nb, 256, 0, s>>>(A, forces, grad, gE, pos, partials);
    }
  } else {
    if (cudaMemsetAsync(partials, 0, sizeof(double) * NV, s) != cudaSuccess) return CL_ERR_CUDA;
  }
  return finish_reduction(mode == 0 ? 2 : 3, dim, hinv, A.n > 0 ? nb : 1, NV, partials, sums, energy, virial, gradbox,
                          gE, s);
}

int launch_candidates(const SweepArgs& A, long long ncells, unsigned long long* out, cudaStream_t s) {
  if (cudaMemsetAsync(out, 0, sizeof(unsigned long long), s) != cudaSuccess) return CL_ERR_CUDA;
  long long blocks = (ncells + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_candidates<<<(int)blocks, 256, 0, s>>>(A, ncells, out);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

}  // namespace clk
