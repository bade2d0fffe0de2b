// User code compiled against include/cellmap_functor.cuh by tests/test_gpu_functor.py:
// two mapped functions of the paper's kind (Code 2), each with its own reduction.
#include "cellmap_functor.cuh"

// Number of neighbours of every particle (both ends of each pair-image).
struct NeighbourCount {
  static constexpr bool kFullShell = true;
  int* counts;
  struct Acc { int n; };
  __device__ void init(Acc& a) const { a.n = 0; }
  __device__ void pair(Acc& a, int, int, float, float, float, float) const { a.n++; }
  __device__ void finish(const Acc& a, int i) const { counts[i] = a.n; }
};

// Lennard-Jones energy, 4 eps ((s^2/d2)^6 - (s^2/d2)^3) (Code 6), each pair once.
struct LennardJones {
  static constexpr bool kFullShell = false;
  float eps4, s2;
  double* out;
  struct Acc { float e; };
  __device__ void init(Acc& a) const { a.e = 0.f; }
  __device__ void pair(Acc& a, int, int, float, float, float, float d2) const {
    const float q = s2 / d2, q3 = q * q * q;
    a.e += eps4 * (q3 * q3 - q3);
  }
  __device__ void finish(const Acc& a, int) const { atomicAdd(out, (double)a.e); }
};

extern "C" int fx_neighbour_counts(const cl_list* cl, int* counts, void* stream) {
  NeighbourCount f;
  f.counts = counts;
  return cellmap::map(cl, f, (cudaStream_t)stream);
}

extern "C" int fx_lj_energy(const cl_list* cl, double eps, double sigma, double* out, void* stream) {
  LennardJones f;
  f.eps4 = (float)(4.0 * eps);
  f.s2 = (float)(sigma * sigma);
  f.out = out;
  if (cudaMemsetAsync(out, 0, sizeof(double), (cudaStream_t)stream) != cudaSuccess) return CL_ERR_CUDA;
  return cellmap::map(cl, f, (cudaStream_t)stream);
}
