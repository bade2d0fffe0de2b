/*
 * cellmap_pairfns.cuh -- ready-made device functors for the compile-time hook
 * of cellmap_functor.cuh: the mapped functions of the paper's examples.
 *
 *   MassPotential      Code 5 (second example): sum of m_i m_j / r over the
 *                      pair-images within the cutoff, masses per particle.
 *   LennardJones       Code 6: 4 eps ((s^2/d2)^6 - (s^2/d2)^3), not shifted.
 *   LennardJonesForces Code 7: the forces F = -dE/dx of the Code 6 energy, and
 *                      the energy, full shell (each particle's force written
 *                      once by its own thread).
 *   VelocityHistogram  Code 10: for each pair-image, bin k = ceil(r / binstep)
 *                      (1-based, bins closed on the right); when k <= nbins the
 *                      pair adds 1 to counts[k-1] and |v_i - v_j| to vsum[k-1].
 *
 * Each is instantiated with cellmap::map(cl, functor, stream) in the caller's
 * CUDA translation unit; libcellmap exports C entry points built from them
 * (cl_map_mass, cl_map_lj, cl_map_velocity_hist in cellmap.h). Per-particle
 * arrays (masses, velocities, forces) are indexed by the original particle
 * index. Scalar outputs are FP64 (they must be zeroed first): each thread's
 * FP32 sum is added in FP64 over the lanes of its warp that finish together,
 * and one lane adds that to the output with an atomic (one atomic per warp
 * and output instead of one per particle: the outputs are a few adjacent
 * addresses that every thread hits). Pair terms are FP32.
 */
#ifndef CELLMAP_PAIRFNS_CUH
#define CELLMAP_PAIRFNS_CUH

#include "cellmap_functor.cuh"

namespace cellmap {
namespace pairfn {

namespace detail {

// Sum of v over the lanes that call this together (FP64), added to *out by
// the lowest of them. Any subset of a warp may call it; each lane's value is
// added once.
__device__ __forceinline__ void warp_add(double* out, double v) {
  const unsigned m = __activemask();
  double s = 0.0;
  for (unsigned r = m; r; r &= r - 1) s += __shfl_sync(m, v, __ffs(r) - 1);
  if ((int)(threadIdx.x & 31) == __ffs(m) - 1 && s != 0.0) atomicAdd(out, s);
}

__device__ __forceinline__ void warp_add(unsigned long long* out, unsigned v) {
  const unsigned m = __activemask();
  const unsigned s = __reduce_add_sync(m, v);
  if ((int)(threadIdx.x & 31) == __ffs(m) - 1 && s != 0u) atomicAdd(out, (unsigned long long)s);
}

}  // namespace detail

struct MassPotential {
  static constexpr bool kFullShell = false;
  const float* mass;  // per particle
  double* out;
  struct Acc { float s; };
  __device__ void init(Acc& a) const { a.s = 0.f; }
  __device__ void pair(Acc& a, int i, int j, float, float, float, float d2) const {
    a.s = fmaf(__ldg(mass + i) * __ldg(mass + j), rsqrtf(d2), a.s);
  }
  __device__ void finish(const Acc& a, int) const { detail::warp_add(out, (double)a.s); }
};

struct LennardJones {
  static constexpr bool kFullShell = false;
  float eps4, s2;  // 4 eps, sigma^2
  double* out;
  struct Acc { float e; };
  __device__ void init(Acc& a) const { a.e = 0.f; }
  __device__ void pair(Acc& a, int, int, float, float, float, float d2) const {
    const float q = s2 / d2, q3 = q * q * q;
    a.e = fmaf(eps4, q3 * q3 - q3, a.e);
  }
  __device__ void finish(const Acc& a, int) const { detail::warp_add(out, (double)a.e); }
};

// F_i = sum_j u'(r) r_ij / r with r_ij = x_j - x_i: u'(r)/r = -24 eps (2 q6^2 - q6)/d2,
// q6 = (s^2/d2)^3. The energy is counted from both ends and halved.
struct LennardJonesForces {
  static constexpr bool kFullShell = true;
  float eps4, eps24, s2;
  float* forces;       // (n, dim) FP32, original order
  int dim;
  double* energy;      // optional
  struct Acc { float fx, fy, fz, e; };
  __device__ void init(Acc& a) const { a.fx = a.fy = a.fz = a.e = 0.f; }
  __device__ void pair(Acc& a, int, int, float dx, float dy, float dz, float d2) const {
    const float y2 = 1.0f / d2;
    const float q = s2 * y2, q3 = q * q * q;
    const float g = -eps24 * (2.0f * q3 * q3 - q3) * y2;
    a.fx = fmaf(g, dx, a.fx);
    a.fy = fmaf(g, dy, a.fy);
    a.fz = fmaf(g, dz, a.fz);
    a.e = fmaf(eps4, q3 * q3 - q3, a.e);
  }
  __device__ void finish(const Acc& a, int i) const {
    forces[(size_t)i * dim + 0] = a.fx;
    forces[(size_t)i * dim + 1] = a.fy;
    if (dim == 3) forces[(size_t)i * 3 + 2] = a.fz;
    if (energy) detail::warp_add(energy, 0.5 * (double)a.e);
  }
};

// NB: compile-time bound on the number of bins. The bins are indexed by the
// pair's bin, so they live in the thread's local memory (L1), one load and one
// store per counted pair instead of a compare chain over every bin; v_i is
// loaded once per particle (at its first counted pair) and kept in Acc; r and
// |v_i - v_j| come from the hardware reciprocal square root (relative error
// about 1e-7).
template <int NB>
struct VelocityHistogram {
  static constexpr bool kFullShell = false;
  const float* vel;   // (n, dim) FP32, original order
  int dim, nbins;     // nbins <= NB
  float inv_binstep;
  unsigned long long* counts;
  double* vsum;
  struct Acc {
    int i;           // particle whose velocity vi holds (-1: none yet)
    float vi[3];
    unsigned c[NB];
    float v[NB];
  };
  __device__ void init(Acc& a) const {
    a.i = -1;
    for (int b = 0; b < nbins; ++b) {
      a.c[b] = 0u;
      a.v[b] = 0.f;
    }
  }
  __device__ void pair(Acc& a, int i, int j, float, float, float, float d2) const {
    const float r = d2 > 0.f ? d2 * rsqrtf(d2) : 0.f;
    const int k = (int)ceilf(r * inv_binstep);  // 1-based bin
    if (k < 1 || k > nbins) return;
    if (a.i != i) {
      a.i = i;
      a.vi[0] = __ldg(vel + (size_t)i * dim);
      a.vi[1] = __ldg(vel + (size_t)i * dim + 1);
      a.vi[2] = dim == 3 ? __ldg(vel + (size_t)i * dim + 2) : 0.f;
    }
    const float* vj = vel + (size_t)j * dim;
    const float t0 = a.vi[0] - __ldg(vj), t1 = a.vi[1] - __ldg(vj + 1);
    const float t2 = dim == 3 ? a.vi[2] - __ldg(vj + 2) : 0.f;
    const float s = fmaf(t0, t0, fmaf(t1, t1, t2 * t2));
    a.c[k - 1] += 1u;
    a.v[k - 1] += s > 0.f ? s * rsqrtf(s) : 0.f;
  }
  __device__ void finish(const Acc& a, int) const {
    for (int b = 0; b < nbins; ++b) {
      detail::warp_add(counts + b, a.c[b]);
      detail::warp_add(vsum + b, (double)a.v[b]);
    }
  }
};

}  // namespace pairfn
}  // namespace cellmap

#endif /* CELLMAP_PAIRFNS_CUH */
