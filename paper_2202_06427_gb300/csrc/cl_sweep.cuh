// cl_sweep.cuh -- device building blocks of the neighbour-cell sweep, shared
// by the reductions of cl_sweep.cu and the neighbour list of cl_pairs.cu.
#pragma once

#include "cl_internal.cuh"

namespace clk {

// Entries of the symmetric virial accumulator (xx, xy, xz, yy, yz, zz / xx, xy, yy).
constexpr int kVirN3 = 6, kVirN2 = 3;

// 1/sqrt(d2) to FP32 accuracy: hardware estimate plus one Newton-Raphson
// step, y1 = y0 + y0 (1 - d2 y0^2) / 2.
__device__ __forceinline__ float rsqrt_nr(float d2) {
  const float y = rsqrtf(d2);
  const float e = fmaf(-d2 * y, y, 1.0f);
  return fmaf(0.5f * y, e, y);
}

// ---------------------------------------------------------------- reductions
// Each reduction: per-thread accumulator, hit() for a pair within the cutoff
// (displacement r = x_j - x_i under the image of the offset), and an
// epilogue. "Half" reductions see each pair-image once, "full" ones twice.

struct RedCount {
  static constexpr bool kFull = false;
  struct Acc { unsigned n; };
  __device__ void init(Acc& a) const { a.n = 0; }
  __device__ void hit(Acc& a, float, float, float, float, int) const { a.n++; }
};

struct RedSumInvR {
  static constexpr bool kFull = false;
  struct Acc { float s; };
  __device__ void init(Acc& a) const { a.s = 0.f; }
  __device__ void hit(Acc& a, float, float, float, float d2, int) const { a.s += rsqrt_nr(d2); }
};

// u(r) = 1/r - 1/rc + (r - rc)/rc^2 = (1 - r/rc)^2 / r
struct RedEnergy {
  static constexpr bool kFull = false;
  float irc;
  struct Acc { float e; };
  __device__ void init(Acc& a) const { a.e = 0.f; }
  __device__ void hit(Acc& a, float, float, float, float d2, int) const {
    const float y = rsqrt_nr(d2);
    const float t = fmaf(-d2 * y, irc, 1.0f);
    a.e = fmaf(t * t, y, a.e);
  }
};

struct RedHist {
  static constexpr bool kFull = false;
  float scale;     // nbins / rmax
  float rmax;
  int nbins;
  unsigned* sh;    // shared-memory histogram
  struct Acc {};
  __device__ void init(Acc&) const {}
  __device__ void hit(Acc&, float, float, float, float d2, int) const {
    const float r = d2 * rsqrt_nr(d2);
    if (r < rmax) {
      int b = (int)(r * scale);
      b = b < nbins ? b : nbins - 1;
      atomicAdd(&sh[b], 1u);
    }
  }
};

// Forces, virial and (optionally) energy; full shell. F_i = sum_j u'(r)/r r,
// W accumulates sum fs r (x) r over ordered pairs (the virial is -1/2 of it).
template <int DIM, bool ENERGY>
struct RedForce {
  static constexpr bool kFull = true;
  float irc, irc2;
  struct Acc { float f[3]; float w[6]; float e; };
  __device__ void init(Acc& a) const {
    a.f[0] = a.f[1] = a.f[2] = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) a.w[k] = 0.f;
    a.e = 0.f;
  }
  __device__ void hit(Acc& a, float dx, float dy, float dz, float d2, int) const {
    const float y = rsqrt_nr(d2);
    const float fs = fmaf(-y, y, irc2) * y;  // u'(r)/r
    const float ax = fs * dx, ay = fs * dy;
    a.f[0] += ax;
    a.f[1] += ay;
    a.w[0] = fmaf(ax, dx, a.w[0]);
    a.w[1] = fmaf(ax, dy, a.w[1]);
    a.w[3] = fmaf(ay, dy, a.w[3]);
    if (DIM == 3) {
      const float az = fs * dz;
      a.f[2] += az;
      a.w[2] = fmaf(ax, dz, a.w[2]);
      a.w[4] = fmaf(ay, dz, a.w[4]);
      a.w[5] = fmaf(az, dz, a.w[5]);
    }
    if (ENERGY) {
      const float t = fmaf(-d2 * y, irc, 1.0f);
      a.e = fmaf(t * t, y, a.e);
    }
  }
};

// --------------------------------------------------------- block reduction

template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* __restrict__ out) {
  __shared__ double sm[8][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------- the sweep

template <int DIM, class R, class Acc>
__device__ __forceinline__ void scan_range(const float4* __restrict__ xs, int j0, int j1, float ax, float ay, float az,
                                           float rc2, const R& red, Acc& acc) {
  for (int j = j0; j < j1; ++j) {
    const float4 q = __ldg(&xs[j]);
    const float dx = q.x - ax, dy = q.y - ay;
    float d2;
    float dz = 0.f;
    if (DIM == 3) {
      dz = q.z - az;
      d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    } else {
      d2 = fmaf(dx, dx, dy * dy);
    }
    if (d2 < rc2) red.hit(acc, dx, dy, dz, d2, __float_as_int(q.w));
  }
}

// Visits every pair-image of sorted particle p (half or full shell) and
// accumulates into acc. Returns false for threads past the end.
// ARGS: SweepArgs (stencil in the kernel parameters) or any struct with the
// same fields (xs, cellc, cell_start, n, nx, ny, nz, rc2, noff, off[]).
template <int DIM, class R, class ARGS>
__device__ __forceinline__ bool sweep_particle(const ARGS& A, const R& red, typename R::Acc& acc, int p,
                                               float4& pi) {
  if (p >= A.n) return false;
  pi = A.xs[p];
  const unsigned cc = A.cellc[p];
  const int cx = (int)(cc & 1023u), cy = (int)((cc >> 10) & 1023u), cz = (int)(cc >> 20);
  {
    const int c = cx + A.nx * (cy + A.ny * cz);
    const int s0 = A.cell_start[c], s1 = A.cell_start[c + 1];
    if (R::kFull) scan_range<DIM>(A.xs, s0, p, pi.x, pi.y, pi.z, A.rc2, red, acc);
    scan_range<DIM>(A.xs, p + 1, s1, pi.x, pi.y, pi.z, A.rc2, red, acc);
  }
  for (int k = 1; k < A.noff; ++k) {
    const Off o = A.off[k];
    int x2 = cx + o.dx;
    x2 -= (x2 >= A.nx) ? A.nx : 0;
    int y2 = cy + o.dy;
    y2 -= (y2 >= A.ny) ? A.ny : 0;
    int z2 = 0;
    if (DIM == 3) {
      z2 = cz + o.dz;
      z2 -= (z2 >= A.nz) ? A.nz : 0;
    }
    const int c = x2 + A.nx * (y2 + A.ny * z2);
    scan_range<DIM>(A.xs, A.cell_start[c], A.cell_start[c + 1], pi.x - o.sx, pi.y - o.sy, pi.z - o.sz, A.rc2, red,
                    acc);
  }
  return true;
}

// ------------------------------------------------- packed (f32x2) sweep, 3D
// Two neighbour candidates per iteration in packed FP32 (one instruction
// computes both lanes of a float2): the same FMA-pipe work as the scalar loop
// in half the issue slots. xy2/zz2 hold particles (j, j+1) at element j; the
// second slot is masked when j+1 leaves the range.

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// 1/sqrt(d2) in both lanes from the hardware estimate alone. Measured on this
// GPU over d2 in [0.05, 144]: mean relative error -6.5e-9, largest 1.25e-7, so
// the bias it leaves in energy and virial sums is below 1e-7 relative.
__device__ __forceinline__ float2 rsqrt2(float2 d2) { return make_float2(rsqrtf(d2.x), rsqrtf(d2.y)); }

// Shifted-force energy (1 - r/rc)^2 / r of the pairs in the cutoff.
struct Red2Energy {
  static constexpr bool kFull = false;
  static constexpr bool kCull = true;  // skip cells beyond rc (sweep_particle2)
  float irc;
  struct Acc { float2 e; };
  __device__ void init(Acc& a) const { a.e = f2(0.f); }
  __device__ void hit2(Acc& a, float2, float2, float2, float2 d2, bool h0, bool h1) const {
    const float2 y = rsqrt2(d2);
    const float2 t = __ffma2_rn(__fmul2_rn(d2, y), f2(-irc), f2(1.0f));
    float2 u = __fmul2_rn(__fmul2_rn(t, t), y);
    u.x = h0 ? u.x : 0.f;
    u.y = h1 ? u.y : 0.f;
    a.e = __fadd2_rn(a.e, u);
  }
};

// Pair count, sum 1/r and distance histogram (half shell), packed. The
// histogram takes x = r nbins / rmax = sqrt(d2 scale^2) from the hardware
// square root (relative error about 1e-7) and counts the pair in bin floor(x)
// when x < xlim = min(nbins, rc scale); floor(x) is read from the low mantissa
// bits of x + 2^23 added with rounding toward zero (exact for 0 <= x < 2^23),
// which keeps the conversion off the special-function unit.
__device__ __forceinline__ float sqrt_approx(float v) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

struct Red2Count {
  static constexpr bool kFull = false;
  static constexpr bool kCull = true;
  struct Acc { unsigned n; };
  __device__ void init(Acc& a) const { a.n = 0; }
  __device__ void hit2(Acc& a, float2, float2, float2, float2, bool h0, bool h1) const {
    a.n += (h0 ? 1u : 0u) + (h1 ? 1u : 0u);
  }
};

struct Red2SumInvR {
  static constexpr bool kFull = false;
  static constexpr bool kCull = true;
  struct Acc { float2 s; };
  __device__ void init(Acc& a) const { a.s = f2(0.f); }
  __device__ void hit2(Acc& a, float2, float2, float2, float2 d2, bool h0, bool h1) const {
    float2 y = rsqrt2(d2);
    y.x = h0 ? y.x : 0.f;
    y.y = h1 ? y.y : 0.f;
    a.s = __fadd2_rn(a.s, y);
  }
};

struct Red2Hist {
  static constexpr bool kFull = false;
  static constexpr bool kCull = false;  // measured slower with the cell test (0.853 against 0.832 ms, 1M triclinic)
  float scale2, xlim;
  unsigned* sh;  // shared-memory histogram
  struct Acc {};
  __device__ void init(Acc&) const {}
  __device__ void hit2(Acc&, float2, float2, float2, float2 d2, bool h0, bool h1) const {
    const float2 s2 = __fmul2_rn(d2, f2(scale2));
    const float2 x = make_float2(sqrt_approx(s2.x), sqrt_approx(s2.y));
    const float2 t = __fadd2_rz(x, f2(8388608.0f));
    if (h0 && x.x < xlim) atomicAdd(&sh[__float_as_int(t.x) - 0x4B000000], 1u);
    if (h1 && x.y < xlim) atomicAdd(&sh[__float_as_int(t.y) - 0x4B000000], 1u);
  }
};

// Forces and virial (optionally energy), full shell, with the opposite sign:
// fsn = -u'(r)/r = y^3 - y/rc^2 and Gn = sum fsn r = -F_i. The virial needs no
// per-pair work: writing r = x_j + S_o - x_i (cell-local coordinates, S_o the
// shift of neighbour cell o) and pairing each ordered pair-image (i, j, o) with
// its reverse (j, i, -o), whose r is -r,
//   sum over ordered pairs of fsn r (x) r
//     = sum_i [ sum_o S_o (x) Gn_i(o)  -  2 x_i (x) Gn_i ],
// where Gn_i(o) is the part of Gn_i from neighbour cell o. So the sweep keeps a
// per-cell partial force (packed, two lanes) and folds S_o (x) Gn_i(o) into a
// 3x3 accumulator once per cell visit.
template <bool ENERGY>
struct Red2Force {
  static constexpr bool kFull = true;
  static constexpr bool kCull = true;
  float irc, irc2;
  struct Acc {
    float2 gx, gy, gz;  // partial Gn of the current neighbour cell
    float tx, ty, tz;   // Gn so far
    float m[9];         // sum_o S_o (x) Gn(o)
    float2 e;
  };
  __device__ void init(Acc& a) const {
    a.gx = a.gy = a.gz = a.e = f2(0.f);
    a.tx = a.ty = a.tz = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) a.m[k] = 0.f;
  }
  __device__ void hit2(Acc& a, float2 dx, float2 dy, float2 dz, float2 d2, bool h0, bool h1) const {
    const float2 y = rsqrt2(d2);
    float2 fsn = __fmul2_rn(__ffma2_rn(y, y, f2(-irc2)), y);
    fsn.x = h0 ? fsn.x : 0.f;
    fsn.y = h1 ? fsn.y : 0.f;
    a.gx = __ffma2_rn(fsn, dx, a.gx);
    a.gy = __ffma2_rn(fsn, dy, a.gy);
    a.gz = __ffma2_rn(fsn, dz, a.gz);
    if (ENERGY) {
      const float2 t = __ffma2_rn(__fmul2_rn(d2, y), f2(-irc), f2(1.0f));
      float2 u = __fmul2_rn(__fmul2_rn(t, t), y);
      u.x = h0 ? u.x : 0.f;
      u.y = h1 ? u.y : 0.f;
      a.e = __fadd2_rn(a.e, u);
    }
  }
  // end of one neighbour cell with shift (sx, sy, sz)
  __device__ void cell_done(Acc& a, float sx, float sy, float sz) const {
    const float gx = a.gx.x + a.gx.y, gy = a.gy.x + a.gy.y, gz = a.gz.x + a.gz.y;
    a.m[0] = fmaf(sx, gx, a.m[0]);
    a.m[1] = fmaf(sx, gy, a.m[1]);
    a.m[2] = fmaf(sx, gz, a.m[2]);
    a.m[3] = fmaf(sy, gx, a.m[3]);
    a.m[4] = fmaf(sy, gy, a.m[4]);
    a.m[5] = fmaf(sy, gz, a.m[5]);
    a.m[6] = fmaf(sz, gx, a.m[6]);
    a.m[7] = fmaf(sz, gy, a.m[7]);
    a.m[8] = fmaf(sz, gz, a.m[8]);
    a.tx += gx;
    a.ty += gy;
    a.tz += gz;
    a.gx = a.gy = a.gz = f2(0.f);
  }
  // per-particle share of sum fsn r (x) r, symmetrised: xx, xy, xz, yy, yz, zz
  __device__ void virial(const Acc& a, float px, float py, float pz, float* v6) const {
    const float M[9] = {fmaf(-2.f * px, a.tx, a.m[0]), fmaf(-2.f * px, a.ty, a.m[1]), fmaf(-2.f * px, a.tz, a.m[2]),
                        fmaf(-2.f * py, a.tx, a.m[3]), fmaf(-2.f * py, a.ty, a.m[4]), fmaf(-2.f * py, a.tz, a.m[5]),
                        fmaf(-2.f * pz, a.tx, a.m[6]), fmaf(-2.f * pz, a.ty, a.m[7]), fmaf(-2.f * pz, a.tz, a.m[8])};
    v6[0] = M[0];
    v6[1] = 0.5f * (M[1] + M[3]);
    v6[2] = 0.5f * (M[2] + M[6]);
    v6[3] = M[4];
    v6[4] = 0.5f * (M[5] + M[7]);
    v6[5] = M[8];
  }
};

// Reductions without per-cell work.
template <class R, class Acc>
__device__ __forceinline__ void cell_done_of(const R&, Acc&, float, float, float) {}
template <bool E>
__device__ __forceinline__ void cell_done_of(const Red2Force<E>& r, typename Red2Force<E>::Acc& a, float sx, float sy,
                                             float sz) {
  r.cell_done(a, sx, sy, sz);
}

// Candidates j in [j0, j1) against one particle, two at a time (the second
// read is clamped to the range and masked). (sx, sy, sz) = S_o - x_i, so that
// the displacement is x_j + S_o - x_i = x_j + s.
template <class R, class Acc>
__device__ __forceinline__ void scan_pairs(const float4* __restrict__ xs, int j0, int j1, float sx, float sy,
                                           float sz, float rc2, const R& red, Acc& acc) {
  const float2 s2x = f2(sx), s2y = f2(sy), s2z = f2(sz);
#pragma unroll 2
  for (int j = j0; j < j1; j += 2) {
    const float4 a = __ldg(&xs[j]);
    const float4 b = __ldg(&xs[min(j + 1, j1 - 1)]);
    const float2 dx = __fadd2_rn(make_float2(a.x, b.x), s2x);
    const float2 dy = __fadd2_rn(make_float2(a.y, b.y), s2y);
    const float2 dz = __fadd2_rn(make_float2(a.z, b.z), s2z);
    float2 d2 = __fmul2_rn(dz, dz);
    d2 = __ffma2_rn(dy, dy, d2);
    d2 = __ffma2_rn(dx, dx, d2);
    const bool h0 = d2.x < rc2;
    const bool h1 = (d2.y < rc2) && (j + 1 < j1);
    if (h0 || h1) red.hit2(acc, dx, dy, dz, d2, h0, h1);
  }
}

// Neighbour cell of stencil entry k for the cell (cx, cy, cz).
template <class ARGS>
__device__ __forceinline__ int stencil_cell(const ARGS& A, int k, int cx, int cy, int cz) {
  const Off& o = A.off[k];
  int x2 = cx + o.dx;
  x2 -= (x2 >= A.nx) ? A.nx : 0;
  int y2 = cy + o.dy;
  y2 -= (y2 >= A.ny) ? A.ny : 0;
  int z2 = cz + o.dz;
  z2 -= (z2 >= A.nz) ? A.nz : 0;
  return x2 + A.nx * (y2 + A.ny * z2);
}

// Packed counterpart of sweep_particle (3D only). A neighbour cell whose
// Cartesian bounding box (centre S_o, half-widths ex, ey, ez, padded by 1e-3
// rc) lies at least rc from the particle holds no pair within the cutoff and
// is skipped (reducers with kCull).
template <class R, class ARGS = SweepArgs>
__device__ __forceinline__ bool sweep_particle2(const ARGS& A, const R& red, typename R::Acc& acc, int p,
                                                float4& pi) {
  if (p >= A.n) return false;
  pi = A.xs[p];
  const unsigned cc = A.cellc[p];
  const int cx = (int)(cc & 1023u), cy = (int)((cc >> 10) & 1023u), cz = (int)(cc >> 20);
  {
    const int c = cx + A.nx * (cy + A.ny * cz);
    const int s0 = A.cell_start[c], s1 = A.cell_start[c + 1];
    if (R::kFull) scan_pairs(A.xs, s0, p, -pi.x, -pi.y, -pi.z, A.rc2, red, acc);
    scan_pairs(A.xs, p + 1, s1, -pi.x, -pi.y, -pi.z, A.rc2, red, acc);
    cell_done_of(red, acc, 0.f, 0.f, 0.f);
  }
  const bool cull = R::kCull && A.ex > 0.f;
  for (int k = 1; k < A.noff; ++k) {
    const Off& o = A.off[k];
    if (cull) {
      const float bx = fmaxf(fabsf(pi.x - o.sx) - A.ex, 0.f), by = fmaxf(fabsf(pi.y - o.sy) - A.ey, 0.f),
                  bz = fmaxf(fabsf(pi.z - o.sz) - A.ez, 0.f);
      if (fmaf(bx, bx, fmaf(by, by, bz * bz)) >= A.rc2) continue;
    }
    const int c = stencil_cell(A, k, cx, cy, cz);
    scan_pairs(A.xs, A.cell_start[c], A.cell_start[c + 1], o.sx - pi.x, o.sy - pi.y, o.sz - pi.z, A.rc2,
               red, acc);
    cell_done_of(red, acc, o.sx, o.sy, o.sz);
  }
  return true;
}

}  // namespace clk
