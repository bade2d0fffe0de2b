// cl_open.cu -- cell lists without periodic boundaries (the neighbour-list
// benchmark of Sec. 4.1, Fig. 2, which the paper runs by giving the periodic
// method a bounding box large enough that no periodic image comes within the
// cutoff). The extent of the particles is reduced on the GPU; the box is
// orthorhombic with side = extent + cutoff (+ a margin) per axis, so that for
// any two particles every image but the direct one is at least rc away.
#include <cmath>
#include <cstring>

#include "cl_internal.cuh"

namespace clk {
namespace {

// Per-axis min and max of n points (dim columns), FP64, one CTA per 256 x 8
// points, atomics on the order-preserving integer image of the doubles.
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(256) k_extent(const double* __restrict__ x, long long n, int dim,
                                                unsigned long long* __restrict__ mm, int* __restrict__ bad) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool finite = true;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    for (int k = 0; k < dim; ++k) {
      const double v = x[i * dim + k];
      if (!isfinite(v)) {
        finite = false;
        continue;
      }
      lo[k] = fmin(lo[k], v);
      hi[k] = fmax(hi[k], v);
    }
  for (int k = 0; k < dim; ++k) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
    if ((threadIdx.x & 31) == 0 && lo[k] <= hi[k]) {
      atomicMin(mm + 2 * k, ordered_bits(lo[k]));
      atomicMax(mm + 2 * k + 1, ordered_bits(hi[k]));
    }
  }
  if (!finite) atomicOr(bad, 1);
}

double from_ordered(unsigned long long b) {
  const unsigned long long v = (b >> 63) ? (b & 0x7fffffffffffffffull) : ~b;
  double d;
  std::memcpy(&d, &v, sizeof(d));
  return d;
}

}  // namespace

int open_box(const double* const* sets, const long long* ns, int nsets, int dim, double cutoff, int lcell,
             cudaStream_t s, cl_box* box) {
  if (dim != 2 && dim != 3) return CL_ERR_INVALID_ARG;
  if (!(cutoff > 0) || !std::isfinite(cutoff)) return CL_ERR_INVALID_ARG;
  unsigned long long* mm = nullptr;
  if (cudaMalloc((void**)&mm, sizeof(unsigned long long) * 6 + sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return CL_ERR_OOM;
  }
  int* bad = reinterpret_cast<int*>(mm + 6);
  unsigned long long init[6];
  for (int k = 0; k < 3; ++k) {
    init[2 * k] = ~0ull;
    init[2 * k + 1] = 0ull;
  }
  int e = CL_OK;
  if (cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess)
    e = CL_ERR_CUDA;
  long long ntot = 0;
  for (int q = 0; q < nsets && !e; ++q) {
    if (ns[q] <= 0) continue;
    ntot += ns[q];
    long long blocks = (ns[q] + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_extent<<<(int)blocks, 256, 0, s>>>(sets[q], ns[q], dim, mm, bad);
    if (cudaGetLastError() != cudaSuccess) e = CL_ERR_CUDA;
  }
  unsigned long long out[6];
  int nonfinite = 0;
  if (!e && (cudaMemcpyAsync(out, mm, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaMemcpyAsync(&nonfinite, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess))
    e = CL_ERR_CUDA;
  cudaFree(mm);
  if (e) return e;
  if (nonfinite) return CL_ERR_NONFINITE;
  std::memset(box, 0, sizeof(*box));
  box->dim = dim;
  box->cutoff = cutoff;
  box->lcell = lcell;
  for (int k = 0; k < dim; ++k) {
    double ext = 0.0;
    if (ntot > 0) ext = from_ordered(out[2 * k + 1]) - from_ordered(out[2 * k]);
    // side > extent + rc, so every image but the direct one is >= rc away; the
    // relative margin keeps the periodic grid away from the extreme points
    const double side = (ext + cutoff) * (1.0 + 1e-6) + 1e-9 * (std::fabs(from_ordered(out[2 * k])) + 1.0);
    box->h[k * dim + k] = ntot > 0 ? side : 2.0 * cutoff;
  }
  return CL_OK;
}

}  // namespace clk

extern "C" int cl_box_nonperiodic(const double* pos_dev, long long n, const double* pos2_dev, long long n2, int dim,
                                  double cutoff, int lcell, void* stream, cl_box* box_out) {
  if (!box_out || n < 0 || n2 < 0 || (n > 0 && !pos_dev) || (n2 > 0 && !pos2_dev)) return CL_ERR_INVALID_ARG;
  const double* sets[2] = {pos_dev, pos2_dev};
  const long long ns[2] = {n, n2};
  return clk::open_box(sets, ns, 2, dim, cutoff, lcell, (cudaStream_t)stream, box_out);
}
