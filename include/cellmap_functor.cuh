/*
 * cellmap_functor.cuh -- compile-time device-functor hook: map a user
 * function over every pair-image within the cutoff of a built cell list.
 *
 * This is the library's counterpart of the paper's mapped function
 * (Sec. 2.3, Code 2: f(x, y, i, j, d2, output) returns the updated output)
 * and of its custom reduction (Sec. 3.2, Code 8: reduce=). The functor is a
 * C++ type compiled into the caller's own CUDA translation unit, so the pair
 * arithmetic inlines into the sweep like the built-in reductions:
 *
 *   struct MyFunctor {
 *     static constexpr bool kFullShell = false;  // false: each pair-image once (half shell)
 *                                                // true : from both ends (owner-writes, no atomics)
 *     struct Acc { ... };                        // per-thread output, lives in registers
 *     __device__ void init(Acc&) const;
 *     // i, j: original 0-based indices; (dx, dy, dz) = x_j - x_i under the
 *     // periodic image, FP32, dz = 0 in 2D; d2 = squared distance < cutoff^2
 *     __device__ void pair(Acc&, int i, int j, float dx, float dy, float dz, float d2) const;
 *     // once per particle i after its pairs: fold Acc into the global output
 *     // (a plain store of per-particle data, or an atomic reduction)
 *     __device__ void finish(const Acc&, int i) const;
 *   };
 *   int rc = cellmap::map(cl, MyFunctor{...}, stream);
 *
 * One thread per cell-sorted particle walks the stencil of its cell (own
 * cell first, then neighbour cells in the order of the stencil) and calls
 * pair() for every neighbour closer than the cutoff. With kFullShell = false
 * a pair-image is visited once, from the end whose offset is
 * lexicographically positive (or from the smaller sorted position inside one
 * cell); with kFullShell = true it is visited from both ends, which lets
 * finish() write per-particle outputs without atomics (Code 7's forces).
 *
 * Requires cellmap.h, the CUDA runtime, and a build for sm_103a; link
 * against libcellmap.so for cl_get_view.
 */
#ifndef CELLMAP_FUNCTOR_CUH
#define CELLMAP_FUNCTOR_CUH

#include <cuda_runtime.h>

#include "cellmap.h"

namespace cellmap {

namespace detail {

template <class F, int DIM>
__device__ __forceinline__ void scan(const F& f, typename F::Acc& acc, const float4* __restrict__ xs, int i,
                                     int j0, int j1, int skip, float ax, float ay, float az, float rc2) {
  for (int j = j0; j < j1; ++j) {
    if (j == skip) continue;
    const float4 q = xs[j];
    const float dx = q.x - ax, dy = q.y - ay;
    const float dz = DIM == 3 ? q.z - az : 0.f;
    const float d2 = DIM == 3 ? fmaf(dx, dx, fmaf(dy, dy, dz * dz)) : fmaf(dx, dx, dy * dy);
    if (d2 < rc2) f.pair(acc, i, __float_as_int(q.w), dx, dy, dz, d2);
  }
}

template <class F, int DIM>
__global__ void __launch_bounds__(256) map_kernel(const cl_view v, const F f) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= v.n) return;
  const float4* __restrict__ xs = static_cast<const float4*>(v.xs);
  const float rc2 = v.cutoff * v.cutoff;
  const float4 pi = xs[p];
  const int i = __float_as_int(pi.w);
  const unsigned cc = v.cellc[p];
  const int cx = (int)(cc & 1023u), cy = (int)((cc >> 10) & 1023u), cz = (int)(cc >> 20);
  const cl_offset* off = F::kFullShell ? v.off_full : v.off_half;
  const int noff = F::kFullShell ? v.noff_full : v.noff_half;
  typename F::Acc acc;
  f.init(acc);
  {
    const int c = cx + v.nx * (cy + v.ny * cz);
    const int s0 = F::kFullShell ? v.cell_start[c] : p + 1;
    scan<F, DIM>(f, acc, xs, i, s0, v.cell_start[c + 1], p, pi.x, pi.y, pi.z, rc2);
  }
  for (int k = 1; k < noff; ++k) {
    const cl_offset o = off[k];
    int x2 = cx + o.dx;
    x2 -= (x2 >= v.nx) ? v.nx : 0;
    int y2 = cy + o.dy;
    y2 -= (y2 >= v.ny) ? v.ny : 0;
    int z2 = cz + o.dz;
    z2 -= (z2 >= v.nz) ? v.nz : 0;
    const int c = x2 + v.nx * (y2 + v.ny * z2);
    scan<F, DIM>(f, acc, xs, i, v.cell_start[c], v.cell_start[c + 1], -1, pi.x - o.sx, pi.y - o.sy, pi.z - o.sz,
                 rc2);
  }
  f.finish(acc, i);
}

}  // namespace detail

/* Launch the functor sweep on `stream`. Returns CL_OK, or the error of
 * cl_get_view, or CL_ERR_CUDA when the launch fails. Asynchronous. */
template <class F>
int map(const cl_list* cl, const F& f, cudaStream_t stream) {
  cl_view v;
  int e = cl_get_view(cl, &v);
  if (e != CL_OK) return e;
  if (v.n == 0) return CL_OK;
  const int blocks = (v.n + 255) / 256;
  if (v.dim == 3) detail::map_kernel<F, 3><<<blocks, 256, 0, stream>>>(v, f);
  else detail::map_kernel<F, 2><<<blocks, 256, 0, stream>>>(v, f);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

}  // namespace cellmap

#endif /* CELLMAP_FUNCTOR_CUH */
