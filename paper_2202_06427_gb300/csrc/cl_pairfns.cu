// cl_pairfns.cu -- C entry points for the mapped functions of the paper's
// examples (Code 5, 6, 7, 10), built from the ready-made device functors of
// cellmap_pairfns.cuh on the compile-time hook of cellmap_functor.cuh: one
// thread per cell-sorted particle over its stencil, as a user's own functor
// would run.
#include "cellmap_pairfns.cuh"

namespace {

template <int NB>
int velocity_hist_nb(const cl_list* cl, const float* vel, int dim, double binstep, int nbins,
                     unsigned long long* counts, double* vsum, cudaStream_t s) {
  cellmap::pairfn::VelocityHistogram<NB> f;
  f.vel = vel;
  f.dim = dim;
  f.nbins = nbins;
  f.inv_binstep = (float)(1.0 / binstep);
  f.counts = counts;
  f.vsum = vsum;
  return cellmap::map(cl, f, s);
}

}  // namespace

extern "C" int cl_map_mass(const cl_list* cl, const float* mass_dev, double* out_dev, void* stream) {
  if (!cl || !out_dev) return CL_ERR_INVALID_ARG;
  cl_view v;
  int e = cl_get_view(cl, &v);
  if (e) return e;
  if (v.n > 0 && !mass_dev) return CL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(out_dev, 0, sizeof(double), s) != cudaSuccess) return CL_ERR_CUDA;
  cellmap::pairfn::MassPotential f;
  f.mass = mass_dev;
  f.out = out_dev;
  return cellmap::map(cl, f, s);
}

extern "C" int cl_map_lj(const cl_list* cl, double eps, double sigma, double* energy_dev, float* forces_dev,
                         void* stream) {
  if (!cl || !energy_dev || !(sigma > 0) || !isfinite(eps) || !isfinite(sigma)) return CL_ERR_INVALID_ARG;
  cl_view v;
  int e = cl_get_view(cl, &v);
  if (e) return e;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(energy_dev, 0, sizeof(double), s) != cudaSuccess) return CL_ERR_CUDA;
  if (!forces_dev) {
    cellmap::pairfn::LennardJones f;
    f.eps4 = (float)(4.0 * eps);
    f.s2 = (float)(sigma * sigma);
    f.out = energy_dev;
    return cellmap::map(cl, f, s);
  }
  cellmap::pairfn::LennardJonesForces f;
  f.eps4 = (float)(4.0 * eps);
  f.eps24 = (float)(24.0 * eps);
  f.s2 = (float)(sigma * sigma);
  f.forces = forces_dev;
  f.dim = v.dim;
  f.energy = energy_dev;
  if (v.n > 0 && cudaMemsetAsync(forces_dev, 0, sizeof(float) * (size_t)v.n * v.dim, s) != cudaSuccess)
    return CL_ERR_CUDA;
  return cellmap::map(cl, f, s);
}

extern "C" int cl_map_velocity_hist(const cl_list* cl, const float* vel_dev, double binstep, int nbins,
                                    unsigned long long* counts_dev, double* vsum_dev, void* stream) {
  if (!cl || !counts_dev || !vsum_dev || !(binstep > 0) || nbins < 1 || nbins > CL_VHIST_MAX_BINS)
    return CL_ERR_INVALID_ARG;
  cl_view v;
  int e = cl_get_view(cl, &v);
  if (e) return e;
  if (v.n > 0 && !vel_dev) return CL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(counts_dev, 0, sizeof(unsigned long long) * nbins, s) != cudaSuccess ||
      cudaMemsetAsync(vsum_dev, 0, sizeof(double) * nbins, s) != cudaSuccess)
    return CL_ERR_CUDA;
  if (nbins <= 16) return velocity_hist_nb<16>(cl, vel_dev, v.dim, binstep, nbins, counts_dev, vsum_dev, s);
  return velocity_hist_nb<CL_VHIST_MAX_BINS>(cl, vel_dev, v.dim, binstep, nbins, counts_dev, vsum_dev, s);
}
