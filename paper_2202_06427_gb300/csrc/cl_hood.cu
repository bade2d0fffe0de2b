// cl_hood.cu -- neighbourhood sweep of the shifted-force pair energy, forces
// and virial in 3D: the loop over cells of Sec. 2.8 with the reduction fused,
// organised around shared memory instead of one thread per particle.
//
// One CTA takes one home cell at a time (persistent CTAs, atomic work counter).
//  1. Staging. The particles of every neighbour cell of the stencil are copied
//     into shared memory, shifted into the frame of the home cell's centre
//     (x' = x + S_o, once per staged particle), and only those with
//     |x'| < rc + d_max are kept, d_max being the largest distance of a home
//     particle from the centre: by the triangle inequality nothing farther is
//     within rc of any home particle. A warp stages one neighbour cell at a time
//     with coalesced loads and compacts the kept particles with a ballot.
//  2. Sweep. A warp takes two home particles at a time; its lanes run over the
//     staged array, two staged particles per lane in packed f32x2 arithmetic
//     (staged pairs are stored interleaved), so one loaded neighbour serves four
//     candidate pairs.
//  3. The own cell is staged apart, in sorted order, so that a particle's pair
//     with itself (and, for the half shell, pairs already counted) is masked by
//     index.
// Against the cell stencil, whose volume is (2 m + 1)^3 cells, the candidates
// per home particle shrink to the ball of radius rc + d_max: about 2.6 per pair
// within the cutoff instead of 4.0 at two cells per cutoff length.
//
// Virial. For ordered pair-images (i, j) whose lattice image T is zero the
// reverse pair-image (j, i) also has T = 0, so with X the wrapped absolute
// positions (cell centre plus local coordinate),
//   sum over T = 0 pairs of fsn r (x) r = -2 sum_i X_i (x) Gn_i^(T=0),
// Gn_i^(T=0) = sum over j with T = 0 of fsn r (fsn = -u'(r)/r). Neighbours
// across the periodic boundary (T != 0) are staged in a segment of their own,
// growing from the far end of the buffer, and add fsn r (x) r directly. Every
// path of this file computes the same per-particle share, so their sums agree.
//
// Home cells that do not pay for the staging (fewer than kMinHome particles)
// are swept afterwards by a companion kernel, one thread per particle over the
// stencil (k_hood_rest), as are all cells when the stencil is larger than the
// table; cells that do not fit (more than kHome particles, or more than kCap
// staged neighbours) by the dense-cell sweep (k_hood_dense), one
// thread per home particle against windows of the staged neighbourhood. All
// three compute the same per-particle virial share and write per-CTA partials
// to one buffer.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "cl_sweep.cuh"

namespace clk {

namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kHome = 128;             // home particles of the fast path (one per thread)
constexpr int kMinHome = 8;            // fewer home particles: the per-particle companion is cheaper
constexpr int kCap = 2560;             // staged neighbour entries (even)
constexpr int kTab = 1 + kWarps * 32;  // stencil entries the fast path takes (32 per warp)
constexpr int kHCap = 1536;            // staged entries of the half-shell path
// Padding entries sit at (kFar, kFar, kFar) and a missing second home particle
// of a group at -kFar: far from everything and from each other (the stand-ins
// of non-finite inputs lie within [1e15, 2e15) per axis), with squared
// distances that stay finite in FP32.
constexpr float kFar = 3e15f;

// Per-CTA partials: mode 0: S6, E; mode 1: S6, X9; mode 2: E; mode 3: S6, X9, E;
// scalar modes 4 (count), 5 (sum 1/r), 6 (histogram): one value (sum 1/r, else 0).
__host__ __device__ constexpr int hood_nv(int mode) {
  return mode == 0 ? 1 + kVirN3 : (mode == 1 ? kVirN3 + 9 : (mode == 3 ? kVirN3 + 10 : 1));
}

struct Smem {
  float4 xy[kCap / 2 + 16];  // staged pairs (x_2k, x_2k+1, y_2k, y_2k+1); 32 trash entries at the end
  float2 zz[kCap / 2 + 16];  // (z_2k, z_2k+1)
  float4 oxy[kHome / 2]; // own cell in sorted order, same layout
  float2 ozz[kHome / 2];
  int hid[kHome];        // original index of the home particle
  float acc[kHome][6];   // Gn of the neighbours across the boundary (T != 0) and of the others (T = 0)
  float4 otab[kTab];     // stencil entry: (shift x, y, z, unwrapped offset as int bits)
  unsigned short rowk[kTab + 1];  // rows of the stencil: entries [rowk[r], rowk[r + 1])
  int nrows;
  float wmax[kWarps];
  int nf, nb;            // staged entries with T = 0 (from the front) and T != 0 (from the back)
  int item;
  unsigned long long ncand;  // candidate pairs this CTA evaluated
  double out[kWarps][16];    // per-warp sums: share of sum fsn r (x) r (6), X (9), energy (1)
};

__device__ __forceinline__ void unpack_off(int v, int& ox, int& oy, int& oz) {
  ox = (int)(signed char)(v & 0xff);
  oy = (int)(signed char)((v >> 8) & 0xff);
  oz = (int)(signed char)((v >> 16) & 0xff);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of N values at once (N a power of two, at most 32): at each
// butterfly step a lane keeps the half of its values selected by its lane bit
// and adds its partner's copy of that half, so N - 1 + (5 - log2 N) shuffles
// replace 5 N. On return v[0] of lane l holds the sum of value l >> (5 - log2 N)
// (every lane holds one of them).
template <int N>
__device__ __forceinline__ void warp_reduce_multi(float (&v)[N]) {
  const int lane = threadIdx.x & 31;
  int off = 16;
#pragma unroll
  for (int n = N; n > 1; n >>= 1, off >>= 1) {
    const bool upper = lane & off;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const float send = upper ? v[i] : v[n / 2 + i];
      const float keep = upper ? v[n / 2 + i] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
#pragma unroll
  for (; off; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
}

__device__ __forceinline__ float own_x(const Smem& S, int t) {
  return reinterpret_cast<const float*>(S.oxy)[(t >> 1) * 4 + (t & 1)];
}
__device__ __forceinline__ float own_y(const Smem& S, int t) {
  return reinterpret_cast<const float*>(S.oxy)[(t >> 1) * 4 + 2 + (t & 1)];
}
__device__ __forceinline__ float own_z(const Smem& S, int t) {
  return reinterpret_cast<const float*>(S.ozz)[(t >> 1) * 2 + (t & 1)];
}

// Per-lane accumulators of one home particle (packed over the lane's two
// staged neighbours).
struct HAcc {
  float2 gx, gy, gz;
};

// One home particle against the two staged neighbours (qx, qy, qz) of a lane.
// (ix, iy, iz) = minus the home particle's coordinates in both halves. Inside
// the staged ball about a third of the candidates are within the cutoff, so
// every warp-step has hits: the pair terms are computed for every candidate.
// Both factors of the shifted-force terms change sign at the cutoff,
//   fsn = y (y^2 - 1/rc^2) and t = 1 - r/rc (u = t^2 y),  y = 1/r,
// so the cutoff is applied by clamping them at zero. With MASK (own cell) the
// index masks m0, m1 and the cutoff test d2 < rc^2 zero y instead, which zeroes
// both terms (and keeps the particle's pair with itself, y = inf, out).
template <bool ENERGY, bool FORCE, bool VIR, bool MASK>
__device__ __forceinline__ void hood_pair(float2 qx, float2 qy, float2 qz, float2 ix, float2 iy, float2 iz, bool m0,
                                          bool m1, float rc2, float irc, float irc2, HAcc& a, float2& e, float2* w) {
  const float2 dx = __fadd2_rn(qx, ix), dy = __fadd2_rn(qy, iy), dz = __fadd2_rn(qz, iz);
  float2 d2 = __fmul2_rn(dz, dz);
  d2 = __ffma2_rn(dy, dy, d2);
  d2 = __ffma2_rn(dx, dx, d2);
  float2 y = rsqrt2(d2);
  if (MASK) {
    y.x = (m0 && d2.x < rc2) ? y.x : 0.f;
    y.y = (m1 && d2.y < rc2) ? y.y : 0.f;
  }
  if (FORCE) {
    float2 fsn = __fmul2_rn(__ffma2_rn(y, y, f2(-irc2)), y);
    if (!MASK) {
      fsn.x = fmaxf(fsn.x, 0.f);
      fsn.y = fmaxf(fsn.y, 0.f);
    }
    if (VIR) {
      const float2 tx = __fmul2_rn(fsn, dx), ty = __fmul2_rn(fsn, dy), tz = __fmul2_rn(fsn, dz);
      a.gx = __fadd2_rn(a.gx, tx);
      a.gy = __fadd2_rn(a.gy, ty);
      a.gz = __fadd2_rn(a.gz, tz);
      w[0] = __ffma2_rn(tx, dx, w[0]);
      w[1] = __ffma2_rn(tx, dy, w[1]);
      w[2] = __ffma2_rn(tx, dz, w[2]);
      w[3] = __ffma2_rn(ty, dy, w[3]);
      w[4] = __ffma2_rn(ty, dz, w[4]);
      w[5] = __ffma2_rn(tz, dz, w[5]);
    } else {
      a.gx = __ffma2_rn(fsn, dx, a.gx);
      a.gy = __ffma2_rn(fsn, dy, a.gy);
      a.gz = __ffma2_rn(fsn, dz, a.gz);
    }
  }
  if (ENERGY) {
    float2 t = __ffma2_rn(__fmul2_rn(d2, y), f2(-irc), f2(1.0f));
    if (!MASK) {
      t.x = fmaxf(t.x, 0.f);
      t.y = fmaxf(t.y, 0.f);
    }
    e = __ffma2_rn(__fmul2_rn(t, t), y, e);
  }
}

// Lanes over staged pairs [k0, k1) against the two home particles of a group.
template <bool ENERGY, bool FORCE, bool VIR>
__device__ __forceinline__ void hood_scan(const float4* __restrict__ xy, const float2* __restrict__ zz, int k0, int k1,
                                          const float2 (&I)[6], float rc2, float irc, float irc2, HAcc& a0, HAcc& a1,
                                          float2& e, float2* w) {
  const int lane = threadIdx.x & 31;
#pragma unroll 2
  for (int k = k0 + lane; k < k1; k += 32) {
    const float4 q = xy[k];
    const float2 z = zz[k];
    const float2 qx = make_float2(q.x, q.y), qy = make_float2(q.z, q.w);
    hood_pair<ENERGY, FORCE, VIR, false>(qx, qy, z, I[0], I[1], I[2], true, true, rc2, irc, irc2, a0, e, w);
    hood_pair<ENERGY, FORCE, VIR, false>(qx, qy, z, I[3], I[4], I[5], true, true, rc2, irc, irc2, a1, e, w);
  }
}

// Own cell in home order: entries 2k, 2k+1 of pair k; home particles t0, t1.
// Full shell: every entry but the particle itself; half shell: entries after it.
template <bool ENERGY, bool FORCE, bool HALF>
__device__ __forceinline__ void hood_own(const float4* __restrict__ xy, const float2* __restrict__ zz, int npairs,
                                         int t0, int t1, const float2 (&I)[6], float rc2, float irc, float irc2,
                                         HAcc& a0, HAcc& a1, float2& e) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k < npairs; k += 32) {
    const float4 q = xy[k];
    const float2 z = zz[k];
    const float2 qx = make_float2(q.x, q.y), qy = make_float2(q.z, q.w);
    const int e0 = 2 * k, e1 = 2 * k + 1;
    const bool m00 = HALF ? e0 > t0 : e0 != t0, m01 = HALF ? e1 > t0 : e1 != t0;
    const bool m10 = HALF ? e0 > t1 : e0 != t1, m11 = HALF ? e1 > t1 : e1 != t1;
    hood_pair<ENERGY, FORCE, false, true>(qx, qy, z, I[0], I[1], I[2], m00, m01, rc2, irc, irc2, a0, e, nullptr);
    hood_pair<ENERGY, FORCE, false, true>(qx, qy, z, I[3], I[4], I[5], m10, m11, rc2, irc, irc2, a1, e, nullptr);
  }
}

// Scalar reductions of the half-shell staged sweep, per candidate pair:
// MODE 4 count, 5 sum 1/r, 6 distance histogram (each pair-image within the
// cutoff once). Unlike the energy, whose terms vanish at the cutoff, these
// test d2 < rc^2 explicitly. 1/r is the hardware reciprocal square root
// (relative error about 1e-7, as in the energy sweep). The histogram takes
// x = r nbins / rmax = sqrt(d2 scale^2) from the hardware square root and
// counts the pair in bin floor(x) when x < xlim = min(nbins, rc scale), with
// shared-memory atomics; floor(x) comes from adding 2^23 rounded toward zero
// (for 0 <= x < 2^23 the sum's low mantissa bits are floor(x)), which keeps
// the float-to-int conversion off the special-function unit. The histogram is
// kept in hcopies copies (stride hstride = 1 mod 32, so one bin of different
// copies lies in different banks), lane l adding to copy l mod hcopies; the
// copies are summed at the end.
struct ScalarRed {
  float rc2, scale2, xlim;
  float irc;       // MODE 2 (shifted-force energy): 1 / rc
  unsigned* hist;  // shared memory: this lane's copy
};

__host__ __device__ constexpr int hist_stride(int nbins) { return nbins + ((33 - nbins % 32) % 32); }

__device__ __forceinline__ void hist_hit(const ScalarRed& R, bool m, float s2) {
  const float x = sqrt_approx(s2);
  const int b = __float_as_int(__fadd_rz(x, 8388608.0f)) - 0x4B000000;
  if (m && x < R.xlim) atomicAdd(&R.hist[b], 1u);
}

template <int MODE, bool MASK>
__device__ __forceinline__ void scalar_pair(float2 qx, float2 qy, float2 qz, float2 ix, float2 iy, float2 iz, bool m0,
                                            bool m1, const ScalarRed& R, unsigned& n, float2& acc) {
  const float2 dx = __fadd2_rn(qx, ix), dy = __fadd2_rn(qy, iy), dz = __fadd2_rn(qz, iz);
  float2 d2 = __fmul2_rn(dz, dz);
  d2 = __ffma2_rn(dy, dy, d2);
  d2 = __ffma2_rn(dx, dx, d2);
  if (MODE == 2) {  // shifted-force energy, the cutoff applied by clamping as in hood_pair
    float2 y = rsqrt2(d2);
    if (MASK) {
      y.x = (m0 && d2.x < R.rc2) ? y.x : 0.f;
      y.y = (m1 && d2.y < R.rc2) ? y.y : 0.f;
    }
    float2 t = __ffma2_rn(__fmul2_rn(d2, y), f2(-R.irc), f2(1.0f));
    t.x = fmaxf(t.x, 0.f);
    t.y = fmaxf(t.y, 0.f);
    acc = __ffma2_rn(__fmul2_rn(t, t), y, acc);
    return;
  }
  bool h0 = false, h1 = false;
  if (MODE != 6) {
    h0 = d2.x < R.rc2 && (!MASK || m0);
    h1 = d2.y < R.rc2 && (!MASK || m1);
  }
  if (MODE == 4) n += (h0 ? 1u : 0u) + (h1 ? 1u : 0u);
  if (MODE == 5) {
    float2 y = rsqrt2(d2);
    y.x = h0 ? y.x : 0.f;
    y.y = h1 ? y.y : 0.f;
    acc = __fadd2_rn(acc, y);
  }
  if (MODE == 6) {
    const float2 s2 = __fmul2_rn(d2, f2(R.scale2));
    hist_hit(R, !MASK || m0, s2.x);
    hist_hit(R, !MASK || m1, s2.y);
  }
}

template <int MODE>
__device__ __forceinline__ void scalar_scan(const float4* __restrict__ xy, const float2* __restrict__ zz, int k0,
                                            int k1, const float2 (&I)[6], const ScalarRed& R, unsigned& n,
                                            float2& acc) {
  const int lane = threadIdx.x & 31;
#pragma unroll 2
  for (int k = k0 + lane; k < k1; k += 32) {
    const float4 q = xy[k];
    const float2 z = zz[k];
    const float2 qx = make_float2(q.x, q.y), qy = make_float2(q.z, q.w);
    scalar_pair<MODE, false>(qx, qy, z, I[0], I[1], I[2], true, true, R, n, acc);
    scalar_pair<MODE, false>(qx, qy, z, I[3], I[4], I[5], true, true, R, n, acc);
  }
}

// Own cell, half shell: entries after the home particle.
template <int MODE>
__device__ __forceinline__ void scalar_own(const float4* __restrict__ xy, const float2* __restrict__ zz, int npairs,
                                           int t0, int t1, const float2 (&I)[6], const ScalarRed& R, unsigned& n,
                                           float2& acc) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k < npairs; k += 32) {
    const float4 q = xy[k];
    const float2 z = zz[k];
    const float2 qx = make_float2(q.x, q.y), qy = make_float2(q.z, q.w);
    const int e0 = 2 * k, e1 = 2 * k + 1;
    scalar_pair<MODE, true>(qx, qy, z, I[0], I[1], I[2], e0 > t0, e1 > t0, R, n, acc);
    scalar_pair<MODE, true>(qx, qy, z, I[3], I[4], I[5], e0 > t1, e1 > t1, R, n, acc);
  }
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Rows of the stencil. Entries 1.. of the stencil are ordered by (oz, oy, ox)
// with ox fastest, so a maximal run of entries with the same (oy, oz) and
// consecutive ox is a row of neighbour cells; cells are linearised x-fastest,
// so at one home cell the particles of a row are ONE contiguous range of the
// sorted arrays, or a few where the row crosses the periodic boundary in x
// (segments, each with its own lattice image along x). The own cell (entry 0)
// is in no row.
__device__ __forceinline__ int floordiv_i(int a, int b) {  // b > 0
  if (a >= 0 && a < b) return 0;  // inside the box: the common case, no division
  const int q = a / b;
  return q - ((a % b != 0) && (a < 0) ? 1 : 0);
}

// Row table of the stencil in S.otab (entries 1 .. min(noff, kTab) - 1), built
// by one thread.
__device__ void build_rows(const SweepArgs& A, Smem& S) {
  const int ne = A.noff < kTab ? A.noff : kTab;
  int nr = 0, pox = 0, poy = 0, poz = 0;
  for (int k = 1; k < ne; ++k) {
    int ox, oy, oz;
    unpack_off(__float_as_int(S.otab[k].w), ox, oy, oz);
    if (k == 1 || oy != poy || oz != poz || ox != pox + 1) S.rowk[nr++] = (unsigned short)k;
    pox = ox;
    poy = oy;
    poz = oz;
  }
  S.rowk[nr] = (unsigned short)(ne > 1 ? ne : 1);
  S.nrows = nr;
}

// One contiguous particle range of a row at a home cell: sorted particles
// [p0, p1); a particle in wrapped cell column xj has stencil entry ebase + xj;
// back = 1 when its lattice image is not zero (T != 0 neighbours are staged
// apart for the virial).
struct RowSeg {
  int p0, p1, ebase, back;
  bool valid;  // the row has a segment of that number
};

// Segment number `which` of row r at home cell (cx, cy, cz).
template <bool FORCE>
__device__ __forceinline__ RowSeg row_segment(const SweepArgs& A, const Smem& S, int r, int which, int cx, int cy,
                                              int cz) {
  RowSeg g;
  g.p0 = g.p1 = g.ebase = g.back = 0;
  g.valid = false;
  const int e0 = S.rowk[r], e1 = S.rowk[r + 1];
  int ox0, oy, oz, ox1, t1, t2;
  unpack_off(__float_as_int(S.otab[e0].w), ox0, oy, oz);
  unpack_off(__float_as_int(S.otab[e1 - 1].w), ox1, t1, t2);
  int y2 = cy + oy, z2 = cz + oz;
  const int ty = floordiv_i(y2, A.ny), tz = floordiv_i(z2, A.nz);
  y2 -= ty * A.ny;
  z2 -= tz * A.nz;
  int ox = ox0;
  for (int k = 0; ox <= ox1; ++k) {
    const int x = cx + ox;
    const int tx = floordiv_i(x, A.nx);
    const int xw = x - tx * A.nx;
    const int len = min(ox1 - ox + 1, A.nx - xw);  // cells up to the row's end or the box edge
    if (k == which) {
      const int ca = xw + A.nx * (y2 + A.ny * z2);
      g.p0 = A.cell_start[ca];
      g.p1 = A.cell_start[ca + len];
      g.ebase = e0 - ox0 + tx * A.nx - cx;
      g.back = (FORCE && (tx | ty | tz) != 0) ? 1 : 0;
      g.valid = true;
      break;
    }
    ox += len;
  }
  return g;
}

// Entry e of the staged pair layout: x at 2e - (e & 1), y two floats later, z at e.
__device__ __forceinline__ void stage_put(Smem& S, int e, float x, float y, float z) {
  float* const xyf = reinterpret_cast<float*>(S.xy);
  const int ix = 2 * e - (e & 1);
  xyf[ix] = x;
  xyf[ix + 2] = y;
  reinterpret_cast<float*>(S.zz)[e] = z;
}

// Staged-buffer entry of a particle: rank r among the kept T = 0 entries (from
// the front) or T != 0 entries (from the back); lanes that keep nothing, and
// ranks beyond the buffer (an overflowing cell, handed to the dense-cell sweep
// afterwards), write to the lane's trash entry past the end.
__device__ __forceinline__ int stage_slot(bool keep, bool back, int r, int lane) {
  const int e = back ? kCap - 1 - r : r;
  return (keep && e >= 0 && e < kCap) ? e : kCap + lane;
}

constexpr int kStageBatch = 4;  // 32-particle chunks of a segment loaded before any is used

// Staging by warp w of rows w, w + kWarps, ..., 32 segments at a time: lane l
// describes segment l & 1 of row w + kWarps (m0 + l / 2) (rows with more
// segments, which only very small grids have, are walked one by one
// afterwards). The warp then takes the segments in turn, lanes over
// consecutive particles (coalesced), kStageBatch chunks loaded before any is
// used and one shared-memory atomic per segment and batch; loads, shifts,
// tests and writes are predicated rather than branched. Each particle is
// shifted into the home frame by its own stencil entry (found from its cell
// column) and kept when |x'| < top; kept particles are compacted with ballots,
// T = 0 entries from the front of the buffer and T != 0 entries from the back.
// Overflow (nf + nb + 2 > kCap) is detected afterwards.
template <bool FORCE>
__device__ __forceinline__ void stage_rows(const SweepArgs& A, Smem& S, int cx, int cy, int cz, float top2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int nrows = S.nrows;
  const int nmine = nrows > warp ? (nrows - 1 - warp) / kWarps + 1 : 0;
  for (int m0 = 0; m0 < nmine; m0 += 16) {
    const int m = m0 + (lane >> 1);
    RowSeg sg;
    sg.p0 = sg.p1 = sg.ebase = sg.back = 0;
    bool more = false;
    if (m < nmine) {
      const int r = warp + kWarps * m;
      sg = row_segment<FORCE>(A, S, r, lane & 1, cx, cy, cz);
      if (!sg.valid) sg.p0 = sg.p1 = 0;
      if (lane & 1) more = row_segment<FORCE>(A, S, r, 2, cx, cy, cz).valid;
    }
    unsigned live = __ballot_sync(0xffffffffu, sg.p1 > sg.p0);  // non-empty segments
    while (live) {
      const int src = __ffs(live) - 1;
      live &= live - 1;
      const int p0 = __shfl_sync(0xffffffffu, sg.p0, src);
      const int p1 = __shfl_sync(0xffffffffu, sg.p1, src);
      const int eb = __shfl_sync(0xffffffffu, sg.ebase, src);
      const bool back = __shfl_sync(0xffffffffu, sg.back, src) != 0;
      for (int pb = p0; pb < p1; pb += 32 * kStageBatch) {
        float4 v[kStageBatch];
        unsigned c[kStageBatch];
#pragma unroll
        for (int u = 0; u < kStageBatch; ++u) {
          const int p = min(pb + 32 * u + lane, p1 - 1);  // clamped: the tail re-reads the last particle
          v[u] = A.xs[p];
          c[u] = A.cellc[p];
        }
        unsigned mk[kStageBatch];
        int n = 0;
#pragma unroll
        for (int u = 0; u < kStageBatch; ++u) {
          const float4 sh = S.otab[eb + (int)(c[u] & 1023u)];
          v[u].x += sh.x;
          v[u].y += sh.y;
          v[u].z += sh.z;
          const bool keep = pb + 32 * u + lane < p1 &&
                            fmaf(v[u].x, v[u].x, fmaf(v[u].y, v[u].y, v[u].z * v[u].z)) < top2;
          mk[u] = __ballot_sync(0xffffffffu, keep);
          n += __popc(mk[u]);
        }
        int base = 0;
        if (lane == 0 && n) base = atomicAdd(back ? &S.nb : &S.nf, n);
        base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
        for (int u = 0; u < kStageBatch; ++u) {
          const bool keep = (mk[u] >> lane) & 1u;
          stage_put(S, stage_slot(keep, back, base + __popc(mk[u] & lt), lane), v[u].x, v[u].y, v[u].z);
          base += __popc(mk[u]);
        }
      }
    }
    // rows of more than two segments (grids narrower than the row): the rest, one by one
    unsigned mm = __ballot_sync(0xffffffffu, more);
    while (mm) {
      const int src = __ffs(mm) - 1;
      mm &= mm - 1;
      const int rr = warp + kWarps * (m0 + (src >> 1));
      for (int which = 2;; ++which) {
        const RowSeg g = row_segment<FORCE>(A, S, rr, which, cx, cy, cz);
        if (!g.valid) break;
        for (int pb = g.p0; pb < g.p1; pb += 32) {
          const int p = min(pb + lane, g.p1 - 1);
          float4 v = A.xs[p];
          const float4 sh = S.otab[g.ebase + (int)(A.cellc[p] & 1023u)];
          v.x += sh.x;
          v.y += sh.y;
          v.z += sh.z;
          const bool keep = pb + lane < g.p1 && fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z)) < top2;
          const unsigned mk = __ballot_sync(0xffffffffu, keep);
          int base = 0;
          if (lane == 0 && mk) base = atomicAdd(g.back ? &S.nb : &S.nf, __popc(mk));
          base = __shfl_sync(0xffffffffu, base, 0);
          stage_put(S, stage_slot(keep, g.back != 0, base + __popc(mk & lt), lane), v.x, v.y, v.z);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- fallback
// One thread per home particle over the stencil on the shifted-pair arrays,
// with the same per-particle virial share as the fast path.
template <bool ENERGY, bool FORCE>
struct RedFallback {
  static constexpr bool kFull = FORCE;
  float irc, irc2;
  struct Acc {
    float2 gx, gy, gz;  // current neighbour cell
    float tx, ty, tz;   // Gn
    float ax, ay, az;   // Gn^(T=0)
    float2 w[6];        // direct fsn r (x) r of T != 0 cells
    float2 e;
    bool wrap;
  };
  __device__ void init(Acc& a) const {
    a.gx = a.gy = a.gz = a.e = f2(0.f);
    a.tx = a.ty = a.tz = a.ax = a.ay = a.az = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) a.w[k] = f2(0.f);
    a.wrap = false;
  }
  __device__ void hit2(Acc& a, float2 dx, float2 dy, float2 dz, float2 d2, bool h0, bool h1) const {
    const float2 y = rsqrt2(d2);
    if (FORCE) {
      float2 fsn = __fmul2_rn(__ffma2_rn(y, y, f2(-irc2)), y);
      fsn.x = h0 ? fsn.x : 0.f;
      fsn.y = h1 ? fsn.y : 0.f;
      if (a.wrap) {
        const float2 tx = __fmul2_rn(fsn, dx), ty = __fmul2_rn(fsn, dy), tz = __fmul2_rn(fsn, dz);
        a.gx = __fadd2_rn(a.gx, tx);
        a.gy = __fadd2_rn(a.gy, ty);
        a.gz = __fadd2_rn(a.gz, tz);
        a.w[0] = __ffma2_rn(tx, dx, a.w[0]);
        a.w[1] = __ffma2_rn(tx, dy, a.w[1]);
        a.w[2] = __ffma2_rn(tx, dz, a.w[2]);
        a.w[3] = __ffma2_rn(ty, dy, a.w[3]);
        a.w[4] = __ffma2_rn(ty, dz, a.w[4]);
        a.w[5] = __ffma2_rn(tz, dz, a.w[5]);
      } else {
        a.gx = __ffma2_rn(fsn, dx, a.gx);
        a.gy = __ffma2_rn(fsn, dy, a.gy);
        a.gz = __ffma2_rn(fsn, dz, a.gz);
      }
    }
    if (ENERGY) {
      const float2 t = __ffma2_rn(__fmul2_rn(d2, y), f2(-irc), f2(1.0f));
      float2 u = __fmul2_rn(__fmul2_rn(t, t), y);
      u.x = h0 ? u.x : 0.f;
      u.y = h1 ? u.y : 0.f;
      a.e = __fadd2_rn(a.e, u);
    }
  }
  __device__ void cell_done(Acc& a) const {
    const float gx = a.gx.x + a.gx.y, gy = a.gy.x + a.gy.y, gz = a.gz.x + a.gz.y;
    a.tx += gx;
    a.ty += gy;
    a.tz += gz;
    if (!a.wrap) {
      a.ax += gx;
      a.ay += gy;
      a.az += gz;
    }
    a.gx = a.gy = a.gz = f2(0.f);
  }
};

// Per-thread outputs of the sweep: energy (Kahan-compensated FP32), the share
// of sum fsn r (x) r (xx, xy, xz, yy, yz, zz) and X = sum x_raw (x) F (backward).
struct ThreadOut {
  float es, ec;
  float v[6];
  float x[9];
  __device__ void add_energy(float t) {
    const float y = t - ec;
    const float s = es + y;
    ec = (s - es) - y;
    es = s;
  }
};

// Per-particle epilogue: force, virial share -2 X (x) Gn^(T=0), and X.
// The same per-particle outputs as hood_particle_out, returned as terms:
// o[0..5] share of sum fsn r (x) r, o[6..14] x_raw (x) F (gradient modes).
template <int MODE>
__device__ __forceinline__ void particle_terms(float* o, int i, float px, float py, float pz, const float* c,
                                               float gx, float gy, float gz, float ax, float ay, float az,
                                               float* __restrict__ forces, double* __restrict__ grad, float g,
                                               const double* __restrict__ pos) {
  const float X[3] = {c[0] + px, c[1] + py, c[2] + pz};
  o[0] = -2.f * X[0] * ax;
  o[1] = -(X[0] * ay + X[1] * ax);
  o[2] = -(X[0] * az + X[2] * ax);
  o[3] = -2.f * X[1] * ay;
  o[4] = -(X[1] * az + X[2] * ay);
  o[5] = -2.f * X[2] * az;
  const float F[3] = {-gx, -gy, -gz};
  if (MODE == 0 || MODE == 2) {
#pragma unroll
    for (int a = 0; a < 3; ++a) forces[(size_t)i * 3 + a] = F[a];
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) grad[(size_t)i * 3 + a] = (double)(-g * F[a]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float xa = (float)pos[(size_t)i * 3 + a];
#pragma unroll
      for (int b = 0; b < 3; ++b) o[6 + a * 3 + b] = xa * F[b];
    }
  }
}

template <int MODE>
__device__ __forceinline__ void hood_particle_out(ThreadOut& T, int i, float px, float py, float pz, const float* c,
                                                  float gx, float gy, float gz, float ax, float ay, float az,
                                                  float* __restrict__ forces, double* __restrict__ grad, float g,
                                                  const double* __restrict__ pos) {
  const float X[3] = {c[0] + px, c[1] + py, c[2] + pz};
  const float A[3] = {ax, ay, az};
  // symmetric part of -2 X (x) A
  T.v[0] -= 2.f * X[0] * A[0];
  T.v[1] -= X[0] * A[1] + X[1] * A[0];
  T.v[2] -= X[0] * A[2] + X[2] * A[0];
  T.v[3] -= 2.f * X[1] * A[1];
  T.v[4] -= X[1] * A[2] + X[2] * A[1];
  T.v[5] -= 2.f * X[2] * A[2];
  const float F[3] = {-gx, -gy, -gz};
  if (MODE == 0 || MODE == 2) {
#pragma unroll
    for (int a = 0; a < 3; ++a) forces[(size_t)i * 3 + a] = F[a];
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) grad[(size_t)i * 3 + a] = (double)(-g * F[a]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float xa = (float)pos[(size_t)i * 3 + a];
#pragma unroll
      for (int b = 0; b < 3; ++b) T.x[a * 3 + b] = fmaf(xa, F[b], T.x[a * 3 + b]);
    }
  }
}

// One particle p (sorted position) of cell (cx, cy, cz) over the stencil on
// the shifted-pair arrays, with the same per-particle virial share as the
// neighbourhood sweep. Returns the candidate pairs evaluated.
template <int MODE>
__device__ unsigned long long particle_sweep(const SweepArgs& A, const HoodArgs& H, int p, int cx, int cy, int cz,
                                             ThreadOut& T, float* __restrict__ forces, double* __restrict__ grad,
                                             float g, const double* __restrict__ pos) {
  constexpr bool FORCE = MODE != 2, ENERGY = MODE != 1;
  unsigned long long ncand = 0;
  RedFallback<ENERGY, FORCE> red;
  red.irc = A.irc;
  red.irc2 = A.irc2;
  const float4 pi = A.xs[p];
  typename RedFallback<ENERGY, FORCE>::Acc acc;
  red.init(acc);
  {
    const int c = cx + A.nx * (cy + A.ny * cz);
    const int s0 = A.cell_start[c], s1 = A.cell_start[c + 1];
    if (FORCE) scan_pairs(A.xs, s0, p, -pi.x, -pi.y, -pi.z, A.rc2, red, acc);
    scan_pairs(A.xs, p + 1, s1, -pi.x, -pi.y, -pi.z, A.rc2, red, acc);
    red.cell_done(acc);
    ncand += (unsigned long long)(FORCE ? s1 - s0 - 1 : s1 - p - 1);
  }
  for (int k = 1; k < A.noff; ++k) {
    const Off& o = A.off[k];
    const int c = stencil_cell(A, k, cx, cy, cz);
    if (FORCE) {
      int ox, oy, oz;
      unpack_off(H.opk[0][k], ox, oy, oz);
      acc.wrap = (cx + ox < 0) || (cx + ox >= A.nx) || (cy + oy < 0) || (cy + oy >= A.ny) || (cz + oz < 0) ||
                 (cz + oz >= A.nz);
    }
    const int j0 = A.cell_start[c], j1 = A.cell_start[c + 1];
    scan_pairs(A.xs, j0, j1, o.sx - pi.x, o.sy - pi.y, o.sz - pi.z, A.rc2, red, acc);
    red.cell_done(acc);
    ncand += (unsigned long long)(j1 - j0);
  }
  if (ENERGY) T.add_energy(acc.e.x + acc.e.y);
  if (FORCE) {
    float cc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      cc[a] = fmaf((float)cx + 0.5f, H.gf[a], fmaf((float)cy + 0.5f, H.gf[3 + a], ((float)cz + 0.5f) * H.gf[6 + a]));
#pragma unroll
    for (int k = 0; k < 6; ++k) T.v[k] += acc.w[k].x + acc.w[k].y;
    hood_particle_out<MODE>(T, __float_as_int(pi.w), pi.x, pi.y, pi.z, cc, acc.tx, acc.ty, acc.tz, acc.ax, acc.ay,
                            acc.az, forces, grad, g, pos);
  }
  return ncand;
}

// Work lists: cells with kMinHome..kHome particles (and a stencil that fits
// the table) go to the neighbourhood sweep (list, work[6] of them); cells with
// more than kHome particles are flagged 2 and listed for the dense-cell sweep
// (dense, *ndense of them); the other non-empty cells (fewer particles, or a
// stencil larger than the table) are flagged 1 for the per-particle companion.
// A cell whose staged neighbourhood overflows is moved to the dense list by
// the sweep itself.
// Particles in the neighbour cells (cx + ox, cy + oy, cz + oz), ox0 <= ox <= ox1
// (wrapped): one contiguous range unless the run crosses the box edge in x.
__device__ __forceinline__ int run_count(const int* __restrict__ cell_start, int nx, int ny, int nz, int cx, int cy,
                                         int cz, int ox0, int ox1, int oy, int oz) {
  int y2 = cy + oy, z2 = cz + oz;
  if ((unsigned)y2 >= (unsigned)ny) y2 = (y2 % ny + ny) % ny;  // wrap only off the box: no division inside it
  if ((unsigned)z2 >= (unsigned)nz) z2 = (z2 % nz + nz) % nz;
  const int row = nx * (y2 + ny * z2);
  const int xa = cx + ox0, xb = cx + ox1;
  if (xa >= 0 && xb < nx) return cell_start[row + xb + 1] - cell_start[row + xa];
  int n = 0;
  for (int x = xa; x <= xb; ++x) {
    const int xw = (x % nx + nx) % nx;
    n += cell_start[row + xw + 1] - cell_start[row + xw];
  }
  return n;
}

// Work lists: cells with kMinHome..kHome particles (and a stencil that fits
// the table) go to the neighbourhood sweep (list, work[6] of them); cells with
// more than kHome particles are flagged 2 and listed for the dense-cell sweep
// (dense, *ndense of them); the other non-empty cells (fewer particles, or a
// stencil larger than the table) are flagged 1 for the per-particle companion.
// A cell whose staged neighbourhood overflows is moved to the dense list by
// the sweep itself. With half != 0 (the half-shell sweep takes the launch)
// every non-empty cell is listed: on list when it holds at most kHome
// particles and its half stencil's cells (opk_half, noff_half entries) at most
// kHCap, on dense (the windowed cells) otherwise.
__global__ void __launch_bounds__(256) k_hood_list(const int* __restrict__ cell_start, int ncells, int noff,
                                                   int* __restrict__ work, int* __restrict__ list,
                                                   unsigned char* __restrict__ flag, int* __restrict__ dense,
                                                   int* __restrict__ ndense, const __grid_constant__ HoodArgs H,
                                                   int noff_half, int nx, int ny, int nz) {
  const int half = H.half;
  const int* opk_half = H.opk[1];
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
  bool take = false, big = false;
  if (h < ncells) {
    const int nh = cell_start[h + 1] - cell_start[h];
    take = (half ? nh >= 1 : nh >= kMinHome) && nh <= kHome && noff <= kTab;
    big = half ? (nh > 0 && !take) : nh > kHome;
    flag[h] = (nh > 0 && !take) ? (big ? 2 : 1) : 0;
    if (half && take) {
      const int cx = h % nx, cy = (h / nx) % ny, cz = h / (nx * ny);
      int cnt = 0;
      if (H.nrows_half > 0) {  // the rows from the host: independent loads
#pragma unroll 4
        for (int r = 0; r < H.nrows_half; ++r)
          cnt += run_count(cell_start, nx, ny, nz, cx, cy, cz, H.rows_half[r][0], H.rows_half[r][1],
                           H.rows_half[r][2], H.rows_half[r][3]);
      } else {
        int r0 = 0, px = 0, py = 0, pz = 0;
        for (int k = 1; k <= noff_half; ++k) {
          int ox = 0, oy = 0, oz = 0;
          if (k < noff_half) unpack_off(opk_half[k], ox, oy, oz);
          if (k > 1 && (k == noff_half || oy != py || oz != pz || ox != px + 1)) {
            cnt += run_count(cell_start, nx, ny, nz, cx, cy, cz, r0, px, py, pz);
            r0 = ox;
          }
          if (k == 1) r0 = ox;
          px = ox;
          py = oy;
          pz = oz;
        }
      }
      if (cnt > kHCap) {
        take = false;
        big = true;
      }
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, take), mb = __ballot_sync(0xffffffffu, big);
  int base = 0, bbase = 0;
  if ((threadIdx.x & 31) == 0) {
    if (m) base = atomicAdd(work + 6, __popc(m));
    if (mb) bbase = atomicAdd(ndense, __popc(mb));
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  bbase = __shfl_sync(0xffffffffu, bbase, 0);
  if (take) list[base + __popc(m & lt)] = h;
  if (big) dense[bbase + __popc(mb & lt)] = h;
}

// Per-CTA partials from the per-thread outputs (layout of the other sweeps).
template <int MODE>
__device__ __forceinline__ void store_partials(const ThreadOut& T, double* __restrict__ out) {
  constexpr bool GRAD = MODE == 1 || MODE == 3;
  constexpr int NV = hood_nv(MODE);
  double v[NV];
  if (MODE == 2) {
    v[0] = (double)T.es - (double)T.ec;
  } else {
    // the accumulator of the other sweeps is sum fs r (x) r = -(sum fsn r (x) r)
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = -(double)T.v[k];
    if (MODE == 0) v[kVirN3] = 0.5 * ((double)T.es - (double)T.ec);
    if (GRAD) {
#pragma unroll
      for (int k = 0; k < 9; ++k) v[kVirN3 + k] = (double)T.x[k];
    }
    if (MODE == 3) v[kVirN3 + 9] = 0.5 * ((double)T.es - (double)T.ec);
  }
  block_sum_store<NV>(v, out);
}

// Companion of the neighbourhood sweep: one thread per particle of the cells
// flagged 1 (fewer than kMinHome particles, or a stencil larger than the table).
template <int MODE>
__global__ void __launch_bounds__(256) k_hood_rest(const __grid_constant__ SweepArgs A,
                                                   const __grid_constant__ HoodArgs H, float* __restrict__ forces,
                                                   double* __restrict__ grad, const double* __restrict__ gE,
                                                   const double* __restrict__ pos, double* __restrict__ partials) {
  constexpr bool GRAD = MODE == 1 || MODE == 3;
  const float g = GRAD ? (float)*gE : 0.f;
  ThreadOut T;
  T.es = T.ec = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) T.v[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) T.x[k] = 0.f;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long ncand = 0;
  bool mine = false;
  int cx = 0, cy = 0, cz = 0;
  if (p < A.n) {
    const unsigned cc = A.cellc[p];
    cx = (int)(cc & 1023u);
    cy = (int)((cc >> 10) & 1023u);
    cz = (int)(cc >> 20);
    mine = H.flag[cx + A.nx * (cy + A.ny * cz)] == 1;
  }
  if (!__syncthreads_or(mine)) {  // nothing left here: zero partials, no reduction
    if (threadIdx.x < hood_nv(MODE)) partials[(size_t)blockIdx.x * hood_nv(MODE) + threadIdx.x] = 0.0;
    return;
  }
  if (mine) ncand = particle_sweep<MODE>(A, H, p, cx, cy, cz, T, forces, grad, g, pos);
#pragma unroll
  for (int o = 16; o; o >>= 1) ncand += __shfl_xor_sync(0xffffffffu, ncand, o);
  if ((threadIdx.x & 31) == 0 && ncand) atomicAdd(H.cand, ncand);
  store_partials<MODE>(T, partials + (size_t)blockIdx.x * hood_nv(MODE));
}

// ------------------------------------------------------------ dense cells
// Cells the neighbourhood sweep cannot stage (more than kHome particles, or a
// staged ball over kCap entries): one CTA
// per cell, one thread per home particle (groups of kDenseThreads). The
// stencil's particles are taken in windows of kWin - 2: each thread loads
// candidates of the flattened neighbour ranges (a binary search over the
// entries' offsets), shifts them into the home frame, keeps those within
// rc + d_max of the centre, and compacts them into shared memory, T = 0
// from the front and T != 0 from the back, pairs interleaved as in the
// neighbourhood sweep; then every thread sweeps the window for its own
// particle, two candidates per step in packed f32x2 (the loads are
// broadcasts), with the per-particle virial share of RedFallback. Warps
// without a home particle only load.
// The particle itself is masked by its index; with the half stencil (energy
// only) an own-cell pair counts when the neighbour's index is the larger.
constexpr int kDenseThreads = 256;
constexpr int kWin = 2048;  // window entries in shared memory (even)

__host__ __device__ constexpr size_t dense_smem_bytes(int noff) {
  return (size_t)(kWin / 2) * (sizeof(float4) + sizeof(float2)) + (size_t)kWin * sizeof(int) +
         (size_t)noff * sizeof(float4) + (size_t)(2 * noff) * sizeof(int);
}

template <int MODE>
__global__ void __launch_bounds__(kDenseThreads, 3) k_hood_dense(const __grid_constant__ SweepArgs A,
                                                                const __grid_constant__ HoodArgs H,
                                                                float* __restrict__ forces, double* __restrict__ grad,
                                                                const double* __restrict__ gE,
                                                                const double* __restrict__ pos,
                                                                double* __restrict__ partials) {
  constexpr bool FORCE = MODE != 2, ENERGY = MODE != 1, HALF = MODE == 2;
  constexpr bool GRAD = MODE == 1 || MODE == 3;
  extern __shared__ __align__(16) unsigned char dsm[];
  float4* txy = reinterpret_cast<float4*>(dsm);             // window pairs (x_2k, x_2k+1, y_2k, y_2k+1)
  float2* tzz = reinterpret_cast<float2*>(txy + kWin / 2);  // (z_2k, z_2k+1)
  int* tix = reinterpret_cast<int*>(tzz + kWin / 2);        // original index (complemented: own cell, half stencil)
  float* txyf = reinterpret_cast<float*>(txy);
  float* tzzf = reinterpret_cast<float*>(tzz);
  float4* stab = reinterpret_cast<float4*>(tix + kWin);     // stencil: (shift, unwrapped offset bits)
  int* e_start = reinterpret_cast<int*>(stab + A.noff);  // flattened offset of each entry
  int* e_j0 = e_start + A.noff;                           // first sorted particle of each entry
  __shared__ int s_nf, s_nb, s_item, s_run;
  __shared__ int s_wsum[kDenseThreads / 32];
  __shared__ float s_wmax[kDenseThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int nd = *H.ndense;
  if ((int)blockIdx.x >= nd) {  // the first nd CTAs take every dense cell through the counter
    if (tid < hood_nv(MODE)) partials[(size_t)blockIdx.x * hood_nv(MODE) + tid] = 0.0;
    return;
  }
  const float g = GRAD ? (float)*gE : 0.f;
  for (int k = tid; k < A.noff; k += kDenseThreads) {
    const Off& o = A.off[k];
    stab[k] = make_float4(o.sx, o.sy, o.sz, __int_as_float(H.opk[HALF ? 1 : 0][k]));
  }
  ThreadOut T;
  T.es = T.ec = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) T.v[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) T.x[k] = 0.f;
  unsigned long long ncand = 0;
  RedFallback<ENERGY, FORCE> red;
  red.irc = A.irc;
  red.irc2 = A.irc2;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(H.work + 5, 1);
    __syncthreads();
    const int q = s_item;
    if (q >= nd) break;
    const int h = H.dense[q];
    const int hs = A.cell_start[h], nh = A.cell_start[h + 1] - hs;
    const int cx = h % A.nx, cy = (h / A.nx) % A.ny, cz = h / (A.nx * A.ny);
    float cc[3];  // centre of the home cell (wrapped absolute frame), FP32
#pragma unroll
    for (int a = 0; a < 3; ++a)
      cc[a] = fmaf((float)cx + 0.5f, H.gf[a], fmaf((float)cy + 0.5f, H.gf[3 + a], ((float)cz + 0.5f) * H.gf[6 + a]));
    // entries: sorted ranges laid end to end
    if (tid == 0) s_run = 0;
    __syncthreads();
    for (int k0 = 0; k0 < A.noff; k0 += kDenseThreads) {
      const int k = k0 + tid;
      int len = 0;
      if (k < A.noff) {
        int ox, oy, oz;
        unpack_off(__float_as_int(stab[k].w), ox, oy, oz);
        int x2 = (cx + ox) % A.nx, y2 = (cy + oy) % A.ny, z2 = (cz + oz) % A.nz;
        x2 += x2 < 0 ? A.nx : 0;
        y2 += y2 < 0 ? A.ny : 0;
        z2 += z2 < 0 ? A.nz : 0;
        const int c = x2 + A.nx * (y2 + A.ny * z2);
        e_j0[k] = A.cell_start[c];
        len = A.cell_start[c + 1] - e_j0[k];
      }
      int inc = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        inc += lane >= o ? u : 0;
      }
      if (lane == 31) s_wsum[warp] = inc;
      __syncthreads();
      int off = s_run;
      for (int w = 0; w < warp; ++w) off += s_wsum[w];
      if (k < A.noff) e_start[k] = off + inc - len;
      __syncthreads();
      if (tid == kDenseThreads - 1) s_run = off + inc;
      __syncthreads();
    }
    const int C = s_run;
    for (int g0 = 0; g0 < nh; g0 += kDenseThreads) {
      const bool own = g0 + tid < nh;
      const int p = hs + g0 + tid;
      const float4 pi = own ? A.xs[p] : make_float4(-kFar, -kFar, -kFar, __int_as_float(-1));
      const int i = __float_as_int(pi.w);
      const bool busy = __any_sync(0xffffffffu, own);  // warps without a home particle only load
      float d = own ? fminf(sqrtf(fmaf(pi.x, pi.x, fmaf(pi.y, pi.y, pi.z * pi.z))), H.hd) : 0.f;
#pragma unroll
      for (int o = 16; o; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
      if (lane == 0) s_wmax[warp] = d;
      __syncthreads();
      float dmax = s_wmax[0];
#pragma unroll
      for (int w = 1; w < kDenseThreads / 32; ++w) dmax = fmaxf(dmax, s_wmax[w]);
      const float top = H.rc + dmax + H.eps, top2 = top * top;
      typename RedFallback<ENERGY, FORCE>::Acc acc;
      red.init(acc);
      for (int w0 = 0; w0 < C; w0 += kWin - 2) {
        const int w1 = min(C, w0 + kWin - 2);
        if (tid == 0) {
          s_nf = 0;
          s_nb = 0;
        }
        __syncthreads();
        for (int r0 = w0; r0 < w1; r0 += kDenseThreads) {
          const int t = r0 + tid;
          bool kf = false, kb = false;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (t < w1) {
            int lo = 0, hi = A.noff;  // last entry whose range starts at or before t
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (e_start[mid] <= t) lo = mid;
              else hi = mid;
            }
            const float4 e = stab[lo];
            const float4 qj = __ldg(&A.xs[e_j0[lo] + (t - e_start[lo])]);
            v.x = qj.x + e.x;
            v.y = qj.y + e.y;
            v.z = qj.z + e.z;
            const int jo = __float_as_int(qj.w);
            v.w = __int_as_float(HALF && lo == 0 ? ~jo : jo);  // own cell marked by the complement
            bool wrap = false;
            if (FORCE) {
              int ox, oy, oz;
              unpack_off(__float_as_int(e.w), ox, oy, oz);
              wrap = (cx + ox < 0) || (cx + ox >= A.nx) || (cy + oy < 0) || (cy + oy >= A.ny) || (cz + oz < 0) ||
                     (cz + oz >= A.nz);
            }
            const bool keep = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z)) < top2;
            kf = keep && !wrap;
            kb = keep && wrap;
          }
          const unsigned mf = __ballot_sync(0xffffffffu, kf), mb = __ballot_sync(0xffffffffu, kb);
          int bf = 0, bb = 0;
          if (lane == 0) {
            if (mf) bf = atomicAdd(&s_nf, __popc(mf));
            if (mb) bb = atomicAdd(&s_nb, __popc(mb));
          }
          bf = __shfl_sync(0xffffffffu, bf, 0);
          bb = __shfl_sync(0xffffffffu, bb, 0);
          if (kf || kb) {
            const int e = kf ? bf + __popc(mf & lt) : kWin - 1 - (bb + __popc(mb & lt));
            txyf[(e >> 1) * 4 + (e & 1)] = v.x;
            txyf[(e >> 1) * 4 + 2 + (e & 1)] = v.y;
            tzzf[(e >> 1) * 2 + (e & 1)] = v.z;
            tix[e] = __float_as_int(v.w);
          }
        }
        __syncthreads();
        const int nf = s_nf, nb = s_nb;
        if (tid < 2 && ((tid == 0 ? nf : nb) & 1)) {  // padding after an odd segment
          const int e = tid == 0 ? nf : kWin - 1 - nb;
          txyf[(e >> 1) * 4 + (e & 1)] = kFar;
          txyf[(e >> 1) * 4 + 2 + (e & 1)] = kFar;
          tzzf[(e >> 1) * 2 + (e & 1)] = kFar;
          tix[e] = -1;
        }
        __syncthreads();
        if (own) ncand += (unsigned long long)(nf + nb);
        if (busy) {
          const float2 nx = f2(-pi.x), ny = f2(-pi.y), nz = f2(-pi.z);
#pragma unroll
          for (int seg = 0; seg < 2; ++seg) {
            acc.wrap = seg == 1;
            const int t0 = seg == 0 ? 0 : kWin - ((nb + 1) & ~1);
            const int t1 = seg == 0 ? ((nf + 1) & ~1) : kWin;
            for (int t = t0; t < t1; t += 2) {
              const float4 xy = txy[t >> 1];
              const float2 zz = tzz[t >> 1];
              const int2 jj = *reinterpret_cast<const int2*>(tix + t);
              const float2 dx = __fadd2_rn(make_float2(xy.x, xy.y), nx);
              const float2 dy = __fadd2_rn(make_float2(xy.z, xy.w), ny);
              const float2 dz = __fadd2_rn(zz, nz);
              const float2 d2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
              bool h0, h1;
              if (HALF) {
                h0 = jj.x >= 0 || ~jj.x > i;
                h1 = jj.y >= 0 || ~jj.y > i;
              } else {
                h0 = jj.x != i;
                h1 = jj.y != i;
              }
              h0 = h0 && d2.x < A.rc2;
              h1 = h1 && d2.y < A.rc2;
              red.hit2(acc, dx, dy, dz, d2, h0, h1);
            }
            red.cell_done(acc);
          }
        }
        __syncthreads();
      }
      if (own) {
        if (ENERGY) T.add_energy(acc.e.x + acc.e.y);
        if (FORCE) {
#pragma unroll
          for (int k = 0; k < 6; ++k) T.v[k] += acc.w[k].x + acc.w[k].y;
          hood_particle_out<MODE>(T, i, pi.x, pi.y, pi.z, cc, acc.tx, acc.ty, acc.tz, acc.ax, acc.ay, acc.az, forces,
                                  grad, g, pos);
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) ncand += __shfl_xor_sync(0xffffffffu, ncand, o);
  if (lane == 0 && ncand) atomicAdd(H.cand, ncand);
  store_partials<MODE>(T, partials + (size_t)blockIdx.x * hood_nv(MODE));
}

// MODE 0: energy, forces, virial (full shell). MODE 1: backward: grad_pos, X,
// virial (full shell). MODE 2: energy (half shell). MODE 3: energy and the
// backward outputs in one full-shell sweep. MODES 4, 5, 6: pair count, sum
// 1/r, distance histogram (half shell; the histogram in dynamic shared memory
// after Smem).
template <int MODE>
__global__ void __launch_bounds__(kThreads, 5) k_hood(const __grid_constant__ SweepArgs A, const __grid_constant__ HoodArgs H,
                                                      float* __restrict__ forces, double* __restrict__ grad,
                                                      const double* __restrict__ gE, const double* __restrict__ pos,
                                                      double* __restrict__ partials) {
  constexpr bool SCALAR = MODE >= 4;
  constexpr bool FORCE = MODE != 2 && !SCALAR, ENERGY = MODE != 1 && !SCALAR, HALF = MODE == 2 || SCALAR;
  constexpr bool GRAD = MODE == 1 || MODE == 3;
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem& S = *reinterpret_cast<Smem*>(smraw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float g = GRAD ? (float)*gE : 0.f;
  for (int k = tid; k < kWarps * 16; k += kThreads) (&S.out[0][0])[k] = 0.0;
  float* const xyf = reinterpret_cast<float*>(S.xy);
  float* const zzf = reinterpret_cast<float*>(S.zz);
  float* const oxyf = reinterpret_cast<float*>(S.oxy);
  float* const ozzf = reinterpret_cast<float*>(S.ozz);
  for (int k = tid; k < A.noff && k < kTab; k += kThreads) {
    const Off& o = A.off[k];
    S.otab[k] = make_float4(o.sx, o.sy, o.sz, __int_as_float(H.opk[HALF ? 1 : 0][k]));
  }
  ScalarRed R;
  R.rc2 = A.rc2;
  R.scale2 = H.hscale * H.hscale;
  R.xlim = H.hxlim;
  unsigned* const hist_all = reinterpret_cast<unsigned*>(smraw + sizeof(Smem));
  R.hist = hist_all + (lane & (H.hcopies - 1)) * H.hstride;
  if (MODE == 6)
    for (int b = tid; b < H.hcopies * H.hstride; b += kThreads) hist_all[b] = 0u;
  unsigned cnt = 0;  // MODE 4: this lane's pairs
  __syncthreads();
  if (tid == 0) build_rows(A, S);
  // Work items (cells of the list made by k_hood_list) come from an atomic
  // counter two ahead: thread 0 keeps the list positions in registers, so the
  // atomic's latency overlaps whole cells, and every thread prefetches into L1
  // the cell ranges it will read for the next cell while this one is swept.
  if (tid == 0) S.ncand = 0;
  const int nlist = H.work[6];
  int next1 = 0, next2 = 0;
  if (tid == 0) {
    next1 = atomicAdd(H.work, 1);
    next2 = atomicAdd(H.work, 1);
  }

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      S.item = next1 < nlist ? H.list[next1] : -1;
      S.nf = 0;
      S.nb = 0;
    }
    __syncthreads();
    const int h = S.item;
    if (h < 0) break;
    if (tid == 0) {
      next1 = next2;
      next2 = atomicAdd(H.work, 1);
    }
    const int hs = A.cell_start[h];
    const int nh = A.cell_start[h + 1] - hs;
    const int cx = h % A.nx, cy = (h / A.nx) % A.ny, cz = h / (A.nx * A.ny);
    float cc[3];  // centre of the home cell (wrapped absolute frame), FP32
#pragma unroll
    for (int a = 0; a < 3; ++a)
      cc[a] = fmaf((float)cx + 0.5f, H.gf[a], fmaf((float)cy + 0.5f, H.gf[3 + a], ((float)cz + 0.5f) * H.gf[6 + a]));

    // ---- home particles (sorted order) and their largest distance from the centre
    float d = 0.f;
    if (tid < nh) {
      const float4 hq = A.xs[hs + tid];
      d = fminf(sqrtf(fmaf(hq.x, hq.x, fmaf(hq.y, hq.y, hq.z * hq.z))), H.hd);
      S.hid[tid] = __float_as_int(hq.w);
      if (GRAD) prefetch_l1(pos + (size_t)__float_as_int(hq.w) * 3);
      oxyf[(tid >> 1) * 4 + (tid & 1)] = hq.x;
      oxyf[(tid >> 1) * 4 + 2 + (tid & 1)] = hq.y;
      ozzf[(tid >> 1) * 2 + (tid & 1)] = hq.z;
    }
    if (tid == 0 && (nh & 1)) {
      oxyf[(nh >> 1) * 4 + 1] = kFar;
      oxyf[(nh >> 1) * 4 + 3] = kFar;
      ozzf[(nh >> 1) * 2 + 1] = kFar;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    if (lane == 0) S.wmax[warp] = d;
    __syncthreads();
    float dmax = S.wmax[0];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) dmax = fmaxf(dmax, S.wmax[w]);
    const float top = H.rc + dmax + H.eps;

    // ---- staging
    stage_rows<FORCE>(A, S, cx, cy, cz, top * top);
    __syncthreads();
    const int nf = S.nf, nb = S.nb;
    if (nf + nb + 2 > kCap) {  // left to the dense-cell sweep
      if (tid == 0) {
        H.flag[h] = 2;
        H.dense[atomicAdd(H.ndense, 1)] = h;
      }
      continue;
    }
    if (tid == 0) H.flag[h] = 0;
    if (tid == 0)
      S.ncand += (unsigned long long)nh * (unsigned long long)(nf + nb) +
                 (unsigned long long)(HALF ? nh * (nh - 1) / 2 : nh * (nh - 1));
    if (tid == 0 && (nf & 1)) {  // padding after an odd segment
      xyf[(nf >> 1) * 4 + 1] = kFar;
      xyf[(nf >> 1) * 4 + 3] = kFar;
      zzf[(nf >> 1) * 2 + 1] = kFar;
    }
    if (tid == 1 && (nb & 1)) {
      const int e = kCap - nb - 1;
      xyf[(e >> 1) * 4 + 0] = kFar;
      xyf[(e >> 1) * 4 + 2] = kFar;
      zzf[(e >> 1) * 2 + 0] = kFar;
    }
    __syncthreads();

    // ---- sweep: groups of two home particles per warp
    const int ngroups = (nh + 1) >> 1;
    const int k0a = 0, k1a = (nf + 1) >> 1;
    const int k0b = (kCap - nb) >> 1, k1b = kCap >> 1;
    for (int gi = warp; gi < ngroups; gi += kWarps) {
      const int t0 = 2 * gi, t1 = 2 * gi + 1;
      const bool has1 = t1 < nh;
      float2 I[6];
      I[0] = f2(-own_x(S, t0));
      I[1] = f2(-own_y(S, t0));
      I[2] = f2(-own_z(S, t0));
      I[3] = f2(has1 ? -own_x(S, t1) : kFar);
      I[4] = f2(has1 ? -own_y(S, t1) : kFar);
      I[5] = f2(has1 ? -own_z(S, t1) : kFar);
      if (SCALAR) {
        float2 sacc = f2(0.f);
        scalar_scan<MODE>(S.xy, S.zz, k0a, k1a, I, R, cnt, sacc);
        scalar_own<MODE>(S.oxy, S.ozz, ngroups, t0, t1, I, R, cnt, sacc);
        if (k1b > k0b) scalar_scan<MODE>(S.xy, S.zz, k0b, k1b, I, R, cnt, sacc);
        if (MODE == 5) {
          const float t = warp_sum(sacc.x + sacc.y);
          if (lane == 0) S.out[warp][15] += (double)t;
        }
        continue;
      }
      HAcc a0, a1;
      a0.gx = a0.gy = a0.gz = a1.gx = a1.gy = a1.gz = f2(0.f);
      float2 e = f2(0.f);
      hood_scan<ENERGY, FORCE, false>(S.xy, S.zz, k0a, k1a, I, A.rc2, A.irc, A.irc2, a0, a1, e, nullptr);
      hood_own<ENERGY, FORCE, HALF>(S.oxy, S.ozz, ngroups, t0, t1, I, A.rc2, A.irc, A.irc2, a0, a1, e);
      if (FORCE) {
        // per-lane partial Gn: the T = 0 part from the first scan, then the
        // part of the neighbours across the boundary; all warp-summed at once
        float v[16];
        v[0] = a0.gx.x + a0.gx.y;
        v[1] = a0.gy.x + a0.gy.y;
        v[2] = a0.gz.x + a0.gz.y;
        v[3] = a1.gx.x + a1.gx.y;
        v[4] = a1.gy.x + a1.gy.y;
        v[5] = a1.gz.x + a1.gz.y;
#pragma unroll
        for (int q = 6; q < 16; ++q) v[q] = 0.f;
        if (k1b > k0b) {
          a0.gx = a0.gy = a0.gz = a1.gx = a1.gy = a1.gz = f2(0.f);
          float2 w[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) w[q] = f2(0.f);
          hood_scan<ENERGY, FORCE, true>(S.xy, S.zz, k0b, k1b, I, A.rc2, A.irc, A.irc2, a0, a1, e, w);
          float wv[8];
#pragma unroll
          for (int q = 0; q < 6; ++q) wv[q] = w[q].x + w[q].y;
          wv[6] = wv[7] = 0.f;
          warp_reduce_multi<8>(wv);  // lane l: value l >> 2
          if ((lane & 3) == 0 && (lane >> 2) < 6) S.out[warp][lane >> 2] += (double)wv[0];
          v[6] = a0.gx.x + a0.gx.y;
          v[7] = a0.gy.x + a0.gy.y;
          v[8] = a0.gz.x + a0.gz.y;
          v[9] = a1.gx.x + a1.gx.y;
          v[10] = a1.gy.x + a1.gy.y;
          v[11] = a1.gz.x + a1.gz.y;
        }
        if (ENERGY) v[12] = e.x + e.y;
        warp_reduce_multi<16>(v);  // lane l: value l >> 1
        // acc[t][0..2]: T != 0 part of Gn, acc[t][3..5]: its T = 0 part
        const int k = lane >> 1;
        if ((lane & 1) == 0) {
          if (k < 12) {
            const int kk = k < 6 ? k : k - 6;  // component of the pair (t0: 0..2, t1: 3..5)
            const int t = kk < 3 ? t0 : t1;
            if (kk < 3 || has1) S.acc[t][(k < 6 ? 3 : 0) + kk % 3] = v[0];
          } else if (ENERGY && k == 12) {
            S.out[warp][15] += (double)v[0];
          }
        }
      } else {
        if (k1b > k0b)
          hood_scan<ENERGY, FORCE, false>(S.xy, S.zz, k0b, k1b, I, A.rc2, A.irc, A.irc2, a0, a1, e, nullptr);
        if (ENERGY) {
          const float t = warp_sum(e.x + e.y);
          if (lane == 0) S.out[warp][15] += (double)t;
        }
      }
    }
    __syncthreads();
    if (FORCE && warp * 32 < nh) {  // warp-uniform: every lane joins the reductions
      float o[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = 0.f;
      if (tid < nh) {
        const int t = tid;
        particle_terms<MODE>(o, S.hid[t], own_x(S, t), own_y(S, t), own_z(S, t), cc, S.acc[t][0] + S.acc[t][3],
                             S.acc[t][1] + S.acc[t][4], S.acc[t][2] + S.acc[t][5], S.acc[t][3], S.acc[t][4],
                             S.acc[t][5], forces, grad, g, pos);
      }
      constexpr int NO = GRAD ? 15 : 6;
      warp_reduce_multi<16>(o);  // lane l: value l >> 1
      if ((lane & 1) == 0 && (lane >> 1) < NO) S.out[warp][lane >> 1] += (double)o[0];
    }
  }

  // candidate count: one atomic per CTA
  __syncthreads();
  if (tid == 0 && S.ncand) atomicAdd(H.cand, S.ncand);
  if (MODE == 4) {
    unsigned long long c = cnt;
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0 && c) atomicAdd(H.count, c);
  }
  if (MODE == 6)
    for (int b = tid; b < H.nbins; b += kThreads)
    {
      unsigned c = 0;
      for (int q = 0; q < H.hcopies; ++q) c += hist_all[q * H.hstride + b];
      if (c) atomicAdd(&H.hist[b], (unsigned long long)c);
    }
  // per-CTA partials (layout of the other sweeps) from the per-warp sums, fixed order
  constexpr int NV = hood_nv(MODE);
  if (tid < NV) {
    int src;  // S.out column of partial tid
    double sign = 1.0;
    if (HALF) {
      src = 15;
    } else if (tid < kVirN3) {
      src = tid;
      sign = -1.0;  // the accumulator of the other sweeps is sum fs r (x) r = -(sum fsn r (x) r)
    } else if (MODE == 0) {
      src = 15;
      sign = 0.5;  // full shell: each pair-image twice
    } else if (tid < kVirN3 + 9) {
      src = tid;
    } else {
      src = 15;
      sign = 0.5;
    }
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) v += S.out[w][src];
    partials[(size_t)blockIdx.x * NV + tid] = sign * v;
  }
}

// ------------------------------------------------------------ half shell
// Each pair-image once (Sec. 2.8: "only half of the neighboring cells are
// evaluated"): one CTA per home cell stages the particles of the half
// stencil's cells within rc + d_max of the centre, and sweeps them
// entry-major: a warp holds 64 staged entries (two per lane) and runs over
// the home particles four at a time, so the force on each entry accumulates
// in the lane's registers and leaves the CTA as one vector atomic per entry,
// while the forces on the four home particles are warp-summed per step into
// shared memory and leave as one vector atomic per home particle. Forces thus
// land in a per-sorted-particle FP32 buffer, from which k_half_finish writes
// the outputs and the per-particle virial and box-gradient shares.
//
// Virial. With X the wrapped absolute positions, a pair-image (h, e) with
// lattice image T of the entry has r = X_e + T.H - X_h, so over all pairs
//   sum fsn r (x) r = sum_p X_p (x) F_p + sum_pairs (T.H) (x) f_e,
// f_e = fsn r the force on the entry: the first sum is per particle
// (k_half_finish), the second is added here for the entries across the
// boundary (T != 0) from their accumulated forces. In the partials layout of
// the other sweeps (minus the sum over ordered pairs) this is -2 times it.
//
// Cells whose particles or half neighbourhood exceed the buffers (more than
// kHome particles, more than kHCap particles in the half stencil's cells)
// take the windowed form of the same sweep: the half neighbourhood's row
// segments are laid end to end and staged in windows of kHCap particles, each
// window swept against the home particles in batches of kHome, and the pairs
// within the cell are swept as a last window per batch (the cell's particles
// from the batch's first on, ordered by index). Every non-empty cell is
// swept, so the path covers the whole grid whenever both stencils fit the
// table.

struct HalfSmem {
  float4 ent[kHCap + 32];  // (x, y, z in the home frame, sorted position as int bits); 32 trash entries
  unsigned short img[kHCap];  // lattice image of the T != 0 entries, (tx, ty, tz) as 5-bit signed fields
  unsigned short ilist[kHCap];  // windowed cells: the staged entries within a batch's ball
  float4 home[kHome + 4];  // home particles (-x, -y, -z, sorted position), padded by far entries
  float4 own[kHome];       // the same with (x, y, z): the own cell's entries
  float hg[kHome][3];      // per home particle: sum of fsn r over its entries
  float4 otab[kTab];       // half stencil: (shift x, y, z, unwrapped offset as int bits)
  int4 seg[kTab];          // windowed cells: row segments (first particle, flattened start, ebase, back | image << 1)
  unsigned short rowk[kTab + 1];
  int nrows, nseg, ctot;
  int oct[9];              // windowed cells: octant ranges of the cell's particles
  float bmin[kWarps][6];   // batch_ball: per-warp minima
  float wmax[kWarps];
  int nf, nb, item, next, nl;
  unsigned long long ncand;
  double out[kWarps][16];
};

// Row segment of the half stencil (the same walk as row_segment) with the
// segment's lattice image packed as bytes.
template <int DUMMY>
__device__ __forceinline__ RowSeg half_segment(const SweepArgs& A, const HalfSmem& S, int r, int which, int cx, int cy,
                                               int cz, int& image) {
  RowSeg g;
  g.p0 = g.p1 = g.ebase = g.back = 0;
  g.valid = false;
  image = 0;
  const int e0 = S.rowk[r], e1 = S.rowk[r + 1];
  int ox0, oy, oz, ox1, t1, t2;
  unpack_off(__float_as_int(S.otab[e0].w), ox0, oy, oz);
  unpack_off(__float_as_int(S.otab[e1 - 1].w), ox1, t1, t2);
  int y2 = cy + oy, z2 = cz + oz;
  const int ty = floordiv_i(y2, A.ny), tz = floordiv_i(z2, A.nz);
  y2 -= ty * A.ny;
  z2 -= tz * A.nz;
  int ox = ox0;
  for (int k = 0; ox <= ox1; ++k) {
    const int x = cx + ox;
    const int tx = floordiv_i(x, A.nx);
    const int xw = x - tx * A.nx;
    const int len = min(ox1 - ox + 1, A.nx - xw);
    if (k == which) {
      const int ca = xw + A.nx * (y2 + A.ny * z2);
      g.p0 = A.cell_start[ca];
      g.p1 = A.cell_start[ca + len];
      g.ebase = e0 - ox0 + tx * A.nx - cx;
      g.back = (tx | ty | tz) != 0 ? 1 : 0;
      g.valid = true;
      image = (tx & 31) | ((ty & 31) << 5) | ((tz & 31) << 10);  // |t| <= 4: stencil reach <= 4
      break;
    }
    ox += len;
  }
  return g;
}

__device__ __forceinline__ int half_slot(bool keep, bool back, int r, int lane) {
  const int e = back ? kHCap - 1 - r : r;
  return (keep && e >= 0 && e < kHCap) ? e : kHCap + lane;
}

// Staging of the half neighbourhood: the row walk of stage_rows, writing
// (x', sorted position) entries and the image of the T != 0 ones.
__device__ __forceinline__ void half_stage(const SweepArgs& A, HalfSmem& S, int cx, int cy, int cz, float top2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int nrows = S.nrows;
  const int nmine = nrows > warp ? (nrows - 1 - warp) / kWarps + 1 : 0;
  for (int m0 = 0; m0 < nmine; m0 += 16) {
    const int m = m0 + (lane >> 1);
    RowSeg sg;
    sg.p0 = sg.p1 = sg.ebase = sg.back = 0;
    int img = 0;
    bool more = false;
    if (m < nmine) {
      const int r = warp + kWarps * m;
      sg = half_segment<0>(A, S, r, lane & 1, cx, cy, cz, img);
      if (!sg.valid) sg.p0 = sg.p1 = 0;
      int dummy;
      if (lane & 1) more = half_segment<0>(A, S, r, 2, cx, cy, cz, dummy).valid;
    }
    unsigned live = __ballot_sync(0xffffffffu, sg.p1 > sg.p0);
    unsigned mm = __ballot_sync(0xffffffffu, more);
    for (int which = 2;; ++which) {
      while (live) {
        const int src = __ffs(live) - 1;
        live &= live - 1;
        const int p0 = __shfl_sync(0xffffffffu, sg.p0, src);
        const int p1 = __shfl_sync(0xffffffffu, sg.p1, src);
        const int eb = __shfl_sync(0xffffffffu, sg.ebase, src);
        const bool back = __shfl_sync(0xffffffffu, sg.back, src) != 0;
        const int im = __shfl_sync(0xffffffffu, img, src);
        for (int pb = p0; pb < p1; pb += 32 * kStageBatch) {
          float4 v[kStageBatch];
          unsigned c[kStageBatch];
#pragma unroll
          for (int u = 0; u < kStageBatch; ++u) {
            const int p = min(pb + 32 * u + lane, p1 - 1);
            v[u] = A.xs[p];
            c[u] = A.cellc[p];
          }
          unsigned mk[kStageBatch];
          int n = 0;
#pragma unroll
          for (int u = 0; u < kStageBatch; ++u) {
            const float4 sh = S.otab[eb + (int)(c[u] & 1023u)];
            v[u].x += sh.x;
            v[u].y += sh.y;
            v[u].z += sh.z;
            v[u].w = __int_as_float(min(pb + 32 * u + lane, p1 - 1));
            const bool keep = pb + 32 * u + lane < p1 &&
                              fmaf(v[u].x, v[u].x, fmaf(v[u].y, v[u].y, v[u].z * v[u].z)) < top2;
            mk[u] = __ballot_sync(0xffffffffu, keep);
            n += __popc(mk[u]);
          }
          int base = 0;
          if (lane == 0 && n) base = atomicAdd(back ? &S.nb : &S.nf, n);
          base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
          for (int u = 0; u < kStageBatch; ++u) {
            const bool keep = (mk[u] >> lane) & 1u;
            const int e = half_slot(keep, back, base + __popc(mk[u] & lt), lane);
            S.ent[e] = v[u];
            if (back && e < kHCap) S.img[e] = (unsigned short)im;
            base += __popc(mk[u]);
          }
        }
      }
      // rows of more than two segments (grids narrower than the row): segment `which` of each
      if (!mm) break;
      live = 0;
      unsigned still = 0;
      if (m < nmine && ((mm >> lane) & 1u)) {
        const int r = warp + kWarps * m;
        sg = half_segment<0>(A, S, r, which, cx, cy, cz, img);
        if (!sg.valid) sg.p0 = sg.p1 = 0;
        int dummy;
        still = half_segment<0>(A, S, r, which + 1, cx, cy, cz, dummy).valid ? 1u : 0u;
      } else {
        sg.p0 = sg.p1 = 0;
      }
      live = __ballot_sync(0xffffffffu, sg.p1 > sg.p0);
      mm = __ballot_sync(0xffffffffu, still != 0);
      if (!live && !mm) break;
    }
  }
}

constexpr int kEnt = 4;             // staged entries per lane in a chunk of the half-shell sweep
constexpr int kChunk = 32 * kEnt;   // entries per chunk

// The staged entries of a cell taken as one sequence: the T = 0 entries
// [0, nf), then the T != 0 entries (stored at the back of the buffer), then
// the home particles themselves (own cell). Position j of the sequence: its
// entry, and (own cell) its home index, else a large value.
struct SeqInfo {
  int nf, nb, nh;
  int obase;  // own pass of a windowed cell: position j is own particle j + obase of the batch
  int wf;     // list pass of a windowed cell: the window's T = 0 entries (the others are T != 0)
};
// Kinds of sequence: the staged entries then the home particles (fast path),
// a windowed cell's own particles (own pass), the entries of S.ilist (list
// pass: a window's entries within a batch's ball; nf = list length).
constexpr int kSeqPlain = 0, kSeqOwn = 1, kSeqList = 2;

template <int SEQ>
__device__ __forceinline__ float4 seq_entry(const HalfSmem& S, const SeqInfo& q, int j, int& own, bool far_up) {
  own = 0x7fffffff;
  if (SEQ == kSeqList) {
    if (j < q.nf) return S.ent[S.ilist[j]];
    return far_up ? make_float4(kFar, kFar, kFar, 0.f) : make_float4(-kFar, -kFar, -kFar, 0.f);
  }
  if (j < q.nf) {
    if (SEQ == kSeqOwn) own = j + q.obase;
    return S.ent[j];
  }
  if (j < q.nf + q.nb) return S.ent[kHCap - q.nb + (j - q.nf)];
  if (j < q.nf + q.nb + q.nh) {
    own = j - q.nf - q.nb;
    return S.own[own];
  }
  return far_up ? make_float4(kFar, kFar, kFar, 0.f) : make_float4(-kFar, -kFar, -kFar, 0.f);
}

// One chunk of kChunk positions of the sequence (kEnt per lane: base + lane
// + 32 u) against every home particle, four home particles per step. MASK
// (the chunk holds own-cell positions): a pair with an own-cell entry counts
// when the entry comes after the home particle. The lane's entries' forces
// (sum of fsn r, r = entry - home) accumulate in jx, jy, jz (pair k: positions
// u = 2k, 2k + 1); each home particle's sum of fsn r over the chunk is
// warp-summed per step into S.hg. SEQ: the kind of sequence (seq_entry); in
// the own pass of a windowed cell every entry is an own-cell particle (index
// j + obase within the batch).
// Scalar modes (MODE 2 energy, 4 count, 5 sum 1/r, 6 histogram) evaluate the
// same candidates with the reduction of scalar_pair and no forces: the count
// in cnt, the energy or sum 1/r in e, the bins in R.hist.
// KB: the chunk's blocks of 64 positions that hold sequence positions (a last
// chunk of at most 64 skips the second block's arithmetic).
template <bool MASK, int SEQ = kSeqPlain, int MODE = 3, int KB = kEnt / 2>
__device__ __forceinline__ void half_chunk(HalfSmem& S, const SeqInfo& sq, int base, int nh, float rc2, float irc,
                                           float irc2, float2 (&jx)[kEnt / 2], float2 (&jy)[kEnt / 2],
                                           float2 (&jz)[kEnt / 2], float2& e, unsigned& cnt, const ScalarRed& R) {
  constexpr bool SCALAR = MODE == 2 || MODE >= 4;
  const int lane = threadIdx.x & 31;
  float2 qx[kEnt / 2], qy[kEnt / 2], qz[kEnt / 2];
  int own[kEnt];
#pragma unroll
  for (int k = 0; k < kEnt / 2; ++k) {
    jx[k] = jy[k] = jz[k] = f2(0.f);
    if (k >= KB) continue;
    const float4 a = seq_entry<SEQ>(S, sq, base + lane + 64 * k, own[2 * k], true);
    const float4 b = seq_entry<SEQ>(S, sq, base + lane + 64 * k + 32, own[2 * k + 1], false);
    qx[k] = make_float2(a.x, b.x);
    qy[k] = make_float2(a.y, b.y);
    qz[k] = make_float2(a.z, b.z);
  }
  if (SCALAR) {
    for (int h = 0; h < nh; ++h) {
      const float4 hp = S.home[h];  // broadcast; negated coordinates
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const bool m0 = !MASK || own[2 * k] > h, m1 = !MASK || own[2 * k + 1] > h;
        scalar_pair<MODE, MASK>(qx[k], qy[k], qz[k], f2(hp.x), f2(hp.y), f2(hp.z), m0, m1, R, cnt, e);
      }
    }
    return;
  }
  for (int h0 = 0; h0 < nh; h0 += 4) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 hp = S.home[h0 + u];  // broadcast; negated coordinates, padded past nh by far entries
      float2 gx = f2(0.f), gy = f2(0.f), gz = f2(0.f);
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const float2 dx = __fadd2_rn(qx[k], f2(hp.x)), dy = __fadd2_rn(qy[k], f2(hp.y)),
                     dz = __fadd2_rn(qz[k], f2(hp.z));
        float2 d2 = __fmul2_rn(dz, dz);
        d2 = __ffma2_rn(dy, dy, d2);
        d2 = __ffma2_rn(dx, dx, d2);
        float2 y = make_float2(rsqrtf(d2.x), rsqrtf(d2.y));
        if (MASK) {
          y.x = (own[2 * k] > h0 + u && d2.x < rc2) ? y.x : 0.f;
          y.y = (own[2 * k + 1] > h0 + u && d2.y < rc2) ? y.y : 0.f;
        }
        float2 fsn = __fmul2_rn(__ffma2_rn(y, y, f2(-irc2)), y);
        fsn.x = fmaxf(fsn.x, 0.f);
        fsn.y = fmaxf(fsn.y, 0.f);
        jx[k] = __ffma2_rn(fsn, dx, jx[k]);
        jy[k] = __ffma2_rn(fsn, dy, jy[k]);
        jz[k] = __ffma2_rn(fsn, dz, jz[k]);
        gx = __ffma2_rn(fsn, dx, gx);
        gy = __ffma2_rn(fsn, dy, gy);
        gz = __ffma2_rn(fsn, dz, gz);
        float2 t = __ffma2_rn(__fmul2_rn(d2, y), f2(-irc), f2(1.0f));
        t.x = fmaxf(t.x, 0.f);
        t.y = fmaxf(t.y, 0.f);
        e = __ffma2_rn(__fmul2_rn(t, t), y, e);
      }
      v[3 * u + 0] = gx.x + gx.y;
      v[3 * u + 1] = gy.x + gy.y;
      v[3 * u + 2] = gz.x + gz.y;
    }
    v[12] = v[13] = v[14] = v[15] = 0.f;
    warp_reduce_multi<16>(v);  // lane l: value l >> 1
    const int k = lane >> 1;
    if ((lane & 1) == 0 && k < 12 && h0 + k / 3 < nh) atomicAdd(&S.hg[h0 + k / 3][k % 3], v[0]);
  }
}

// Adds the accumulated force of sequence position j to its particle (vector
// atomic) and, for an entry across the boundary, the symmetric part of
// (T.H) (x) f to the lane's virial sums.
template <int SEQ = kSeqPlain>
__device__ __forceinline__ void half_flush(const HoodArgs& H, const HalfSmem& S, const SeqInfo& q, int j, float fx,
                                           float fy, float fz, float* wv) {
  if (j >= q.nf + q.nb + q.nh || (fx == 0.f && fy == 0.f && fz == 0.f)) return;
  bool back;
  int idx;
  if (SEQ == kSeqList) {
    idx = S.ilist[j];
    back = idx >= q.wf;
  } else {
    back = j >= q.nf && j < q.nf + q.nb;
    idx = j < q.nf ? j : (back ? kHCap - q.nb + (j - q.nf) : -1);
  }
  const int p = __float_as_int(idx >= 0 ? S.ent[idx].w : S.own[j - q.nf - q.nb].w);
  atomicAdd(&H.hforce[p], make_float4(fx, fy, fz, 0.f));
  if (back) {
    const int im = S.img[idx];
    const float tx = (float)((im << 27) >> 27), ty = (float)((im << 22) >> 27), tz = (float)((im << 17) >> 27);
    float t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) t[a] = tx * H.hrow[a] + ty * H.hrow[3 + a] + tz * H.hrow[6 + a];
    const float f[3] = {fx, fy, fz};
    wv[0] += t[0] * f[0];
    wv[1] += 0.5f * (t[0] * f[1] + t[1] * f[0]);
    wv[2] += 0.5f * (t[0] * f[2] + t[2] * f[0]);
    wv[3] += t[1] * f[1];
    wv[4] += 0.5f * (t[1] * f[2] + t[2] * f[1]);
    wv[5] += t[2] * f[2];
  }
}

// ------------------------------------------------ windowed half-shell cells

// Row segments of the half stencil at cell (cx, cy, cz) laid end to end, by
// warp 0: S.seg[k] = (first particle, flattened start, ebase, back | image
// << 1), S.nseg of them, S.ctot particles in all. A segment covers at least
// one stencil entry, so there are at most kTab - 1.
__device__ void half_segments(const SweepArgs& A, HalfSmem& S, int cx, int cy, int cz) {
  const int lane = threadIdx.x & 31;
  int nseg = 0;
  for (int r0 = 0; r0 < S.nrows; r0 += 32) {
    const int r = r0 + lane;
    int ns = 0, img = 0;
    if (r < S.nrows)
      while (half_segment<0>(A, S, r, ns, cx, cy, cz, img).valid) ++ns;
    int inc = ns;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      inc += lane >= o ? t : 0;
    }
    const int first = nseg + inc - ns;
    for (int k = 0; k < ns; ++k) {
      const RowSeg g = half_segment<0>(A, S, r, k, cx, cy, cz, img);
      S.seg[first + k] = make_int4(g.p0, g.p1 - g.p0, g.ebase, g.back | (img << 1));  // .y: length for now
    }
    nseg += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();
  int total = 0;
  for (int k0 = 0; k0 < nseg; k0 += 32) {
    const int k = k0 + lane;
    const int len = k < nseg ? S.seg[k].y : 0;
    int inc = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      inc += lane >= o ? t : 0;
    }
    if (k < nseg) S.seg[k].y = total + inc - len;
    total += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane == 0) {
    S.nseg = nseg;
    S.ctot = total;
  }
}

// Staging of the flattened half-neighbourhood positions [w0, w1) (at most
// kHCap): each position's segment by binary search over the starts, then the
// shift, the test against the ball of centre b (home frame) and squared
// radius top2, and the compaction of half_stage (T = 0 entries from the
// front, T != 0 from the back).
__device__ void half_stage_window(const SweepArgs& A, HalfSmem& S, int w0, int w1, float bx, float by, float bz,
                                  float top2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int nseg = S.nseg;
  for (int tb = w0 + warp * 32 * kStageBatch; tb < w1; tb += kWarps * 32 * kStageBatch) {
    float4 v[kStageBatch];
    unsigned c[kStageBatch];
    int meta[kStageBatch], eb[kStageBatch];
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const int t = min(tb + 32 * u + lane, w1 - 1);
      int lo = 0, hi = nseg;  // the last segment starting at or before t
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (S.seg[mid].y <= t) lo = mid;
        else hi = mid;
      }
      const int4 sg = S.seg[lo];
      const int p = sg.x + (t - sg.y);
      v[u] = A.xs[p];
      v[u].w = __int_as_float(p);
      c[u] = A.cellc[p];
      eb[u] = sg.z;
      meta[u] = sg.w;
    }
    unsigned mf[kStageBatch], mb[kStageBatch];
    int nfn = 0, nbn = 0;
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const float4 sh = S.otab[eb[u] + (int)(c[u] & 1023u)];
      v[u].x += sh.x;
      v[u].y += sh.y;
      v[u].z += sh.z;
      const float ex = v[u].x - bx, ey = v[u].y - by, ez = v[u].z - bz;
      const bool keep = tb + 32 * u + lane < w1 && fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < top2;
      const bool back = (meta[u] & 1) != 0;
      mf[u] = __ballot_sync(0xffffffffu, keep && !back);
      mb[u] = __ballot_sync(0xffffffffu, keep && back);
      nfn += __popc(mf[u]);
      nbn += __popc(mb[u]);
    }
    int bf = 0, bb = 0;
    if (lane == 0) {
      if (nfn) bf = atomicAdd(&S.nf, nfn);
      if (nbn) bb = atomicAdd(&S.nb, nbn);
    }
    bf = __shfl_sync(0xffffffffu, bf, 0);
    bb = __shfl_sync(0xffffffffu, bb, 0);
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const bool back = (meta[u] & 1) != 0;
      const bool keep = ((back ? mb[u] : mf[u]) >> lane) & 1u;
      const int e = half_slot(keep, back, back ? bb + __popc(mb[u] & lt) : bf + __popc(mf[u] & lt), lane);
      S.ent[e] = v[u];
      if (back && e < kHCap) S.img[e] = (unsigned short)(meta[u] >> 1);
      bf += __popc(mf[u]);
      bb += __popc(mb[u]);
    }
  }
}

// One batch of at most kHome home particles (sorted positions hp ..) against
// the staged sequence sq: the chunks of the sequence from a counter, the
// entries' forces flushed per chunk, the home particles' forces at the end.
// SEQ: the kind of sequence (own pass: every entry an own-cell particle,
// masked by index).
template <int SEQ, int MODE>
__device__ void half_batch(const SweepArgs& A, const HoodArgs& H, HalfSmem& S, const SeqInfo& sq, int hp, int nbh,
                           float2& e, float* wv, unsigned& cnt, const ScalarRed& R) {
  constexpr bool SCALAR = MODE == 2 || MODE >= 4;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int t = tid; t < kHome + 4; t += kThreads) {
    if (t < nbh) {
      const float4 hq = A.xs[hp + t];
      S.home[t] = make_float4(-hq.x, -hq.y, -hq.z, __int_as_float(hp + t));
    } else {
      S.home[t] = make_float4(kFar, -kFar, kFar, __int_as_float(0));
    }
  }
  if (tid == 0) S.next = 0;
  __syncthreads();
  const int nch = (sq.nf + sq.nb + kChunk - 1) / kChunk;
  for (;;) {
    int c = 0;
    if (lane == 0) c = atomicAdd(&S.next, 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= nch) break;
    float2 jx[kEnt / 2], jy[kEnt / 2], jz[kEnt / 2];
    const int base = c * kChunk;
    constexpr bool MASK = SEQ == kSeqOwn;
    if (sq.nf + sq.nb - base > 64)
      half_chunk<MASK, SEQ, MODE, 2>(S, sq, base, nbh, A.rc2, A.irc, A.irc2, jx, jy, jz, e, cnt, R);
    else
      half_chunk<MASK, SEQ, MODE, 1>(S, sq, base, nbh, A.rc2, A.irc, A.irc2, jx, jy, jz, e, cnt, R);
    if (!SCALAR) {
#pragma unroll
      for (int k = 0; k < kEnt / 2; ++k) {
        const int j0 = base + lane + 64 * k;
        half_flush<SEQ>(H, S, sq, j0, jx[k].x, jy[k].x, jz[k].x, wv);
        half_flush<SEQ>(H, S, sq, j0 + 32, jx[k].y, jy[k].y, jz[k].y, wv);
      }
    }
  }
  __syncthreads();
  if (!SCALAR && tid < nbh) {
    const float gx = S.hg[tid][0], gy = S.hg[tid][1], gz = S.hg[tid][2];
    if (gx != 0.f || gy != 0.f || gz != 0.f) atomicAdd(&H.hforce[hp + tid], make_float4(-gx, -gy, -gz, 0.f));
    S.hg[tid][0] = S.hg[tid][1] = S.hg[tid][2] = 0.f;
  }
  __syncthreads();
}

// Ball of a batch of home particles (sorted positions hp .. hp + nbh): the
// middle of their bounding box (home frame) and the squared staging radius
// (rc + their largest distance from it + the rounding margin)^2.
__device__ void batch_ball(const SweepArgs& A, const HoodArgs& H, HalfSmem& S, int hp, int nbh, float& bx,
                           float& by, float& bz, float& top2) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
  float v[6] = {kFar, kFar, kFar, kFar, kFar, kFar};  // min x, y, z and minus max x, y, z
  if (tid < nbh) {
    q = A.xs[hp + tid];
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = -q.x;
    v[4] = -q.y;
    v[5] = -q.z;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = fminf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
  if (lane < 6) S.bmin[warp][lane] = v[lane];
  __syncthreads();
  float m[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    m[k] = S.bmin[0][k];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) m[k] = fminf(m[k], S.bmin[w][k]);
  }
  bx = 0.5f * (m[0] - m[3]);
  by = 0.5f * (m[1] - m[4]);
  bz = 0.5f * (m[2] - m[5]);
  float d = 0.f;
  if (tid < nbh) {
    const float ex = q.x - bx, ey = q.y - by, ez = q.z - bz;
    d = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
  __syncthreads();  // every warp has read S.bmin
  if (lane == 0) S.wmax[warp] = d;
  __syncthreads();
  float dm = S.wmax[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) dm = fmaxf(dm, S.wmax[w]);
  const float top = H.rc + dm + H.eps;
  top2 = top * top;
}

// A cell that does not fit the buffers: its half neighbourhood in windows,
// each against the home particles in batches, then the pairs within the cell
// (batch b against the particles from its first on). The batches of the
// neighbourhood pass are the cell's particles in ranges of at most kHome,
// split at the octant boundaries of their order (cells of kOctMin..kOctCap
// particles are ordered by octant by the build), each with its own ball
// (batch_ball), so the particles of a dense cell see about half the
// candidates of the cell's ball. Returns the candidates.
template <int MODE>
__device__ __forceinline__ unsigned long long half_windowed(const SweepArgs& A, const HoodArgs& H, HalfSmem& S,
                                                            int hs, int nh, int cx, int cy, int cz, float2& e,
                                                            float* wv, unsigned& cnt, const ScalarRed& R) {
  const int tid = threadIdx.x;
  if (threadIdx.x < 32) half_segments(A, S, cx, cy, cz);
  // octant ranges of the cell's order: S.oct[g] .. S.oct[g + 1]
  const bool octs = nh >= kOctMin && nh <= kOctCap;
  if (tid < 9) S.oct[tid] = 0;
  __syncthreads();
  if (octs)
    for (int t = tid; t < nh; t += kThreads) {
      const float4 q = A.xs[hs + t];
      atomicAdd(&S.oct[1 + ((q.x > 0.f ? 1 : 0) | (q.y > 0.f ? 2 : 0) | (q.z > 0.f ? 4 : 0))], 1);
    }
  __syncthreads();
  if (tid == 0) {
    if (octs)
      for (int g = 0; g < 8; ++g) S.oct[g + 1] += S.oct[g];
    else
      for (int g = 1; g < 9; ++g) S.oct[g] = nh;  // one group
  }
  __syncthreads();
  // the window's staging ball: the cell's particles' largest distance from
  // the cell centre
  {
    float d = 0.f;
    for (int t = tid; t < nh; t += kThreads) {
      const float4 q = A.xs[hs + t];
      d = fmaxf(d, fminf(sqrtf(fmaf(q.x, q.x, fmaf(q.y, q.y, q.z * q.z))), H.hd));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    if ((tid & 31) == 0) S.wmax[tid >> 5] = d;
  }
  __syncthreads();
  float dcell = S.wmax[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) dcell = fmaxf(dcell, S.wmax[w]);
  const float tcell = H.rc + dcell + H.eps;
  const int C = S.ctot;
  unsigned long long cand = 0;
  for (int w0 = 0; w0 < C; w0 += kHCap) {
    if (tid == 0) {
      S.nf = 0;
      S.nb = 0;
    }
    __syncthreads();
    half_stage_window(A, S, w0, min(C, w0 + kHCap), 0.f, 0.f, 0.f, tcell * tcell);
    __syncthreads();
    const int wf = min(S.nf, kHCap), wb = min(S.nb, kHCap - wf);
    for (int g = 0; g < 8; ++g) {
      const int g0 = S.oct[g], g1 = S.oct[g + 1];
      for (int b0 = g0; b0 < g1; b0 += kHome) {
        const int nbh = min(kHome, g1 - b0);
        float bx, by, bz, top2;
        batch_ball(A, H, S, hs + b0, nbh, bx, by, bz, top2);  // ends with a barrier
        // the window's entries within the batch's ball
        if (tid == 0) S.nl = 0;
        __syncthreads();
        for (int i0 = (tid >> 5) * 32; i0 < wf + wb; i0 += kThreads) {
          const int i = i0 + (tid & 31);
          const int idx = i < wf ? i : kHCap - wb + (i - wf);
          bool keep = false;
          if (i < wf + wb) {
            const float4 q = S.ent[idx];
            const float ex = q.x - bx, ey = q.y - by, ez = q.z - bz;
            keep = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < top2;
          }
          const unsigned m = __ballot_sync(0xffffffffu, keep);
          int at = 0;
          if ((tid & 31) == 0 && m) at = atomicAdd(&S.nl, __popc(m));
          at = __shfl_sync(0xffffffffu, at, 0);
          if (keep) S.ilist[at + __popc(m & ((1u << (tid & 31)) - 1u))] = (unsigned short)idx;
        }
        __syncthreads();
        SeqInfo sq;
        sq.nf = S.nl;  // read by every thread before batch_ball's next barriers
        sq.nb = 0;
        sq.nh = 0;
        sq.obase = 0;
        sq.wf = wf;
        half_batch<kSeqList, MODE>(A, H, S, sq, hs + b0, nbh, e, wv, cnt, R);
        cand += (unsigned long long)nbh * (unsigned long long)sq.nf;
      }
    }
  }
  for (int b0 = 0; b0 < nh; b0 += kHome) {
    const int nbh = min(kHome, nh - b0);
    for (int o0 = b0; o0 < nh; o0 += kHCap) {
      const int no = min(kHCap, nh - o0);
      for (int j = tid; j < no; j += kThreads) {
        const float4 q = A.xs[hs + o0 + j];
        S.ent[j] = make_float4(q.x, q.y, q.z, __int_as_float(hs + o0 + j));
      }
      SeqInfo sq;
      sq.nf = no;
      sq.nb = 0;
      sq.nh = 0;
      sq.obase = o0 - b0;
      sq.wf = 0;
      half_batch<kSeqOwn, MODE>(A, H, S, sq, hs + b0, nbh, e, wv, cnt, R);  // its first barrier also covers the entries
      cand += (unsigned long long)nbh * (unsigned long long)no -
              (o0 == b0 ? (unsigned long long)nbh * (unsigned long long)(nbh + 1) / 2 : 0ull);
    }
  }
  return cand;
}

// WIN = false: the fast-path cells (list); true: the windowed cells (dense),
// from a counter of their own.
template <int MODE, bool WIN>
__global__ void __launch_bounds__(kThreads, 5) k_hood_half(const __grid_constant__ SweepArgs A,
                                                           const __grid_constant__ HoodArgs H,
                                                           double* __restrict__ partials) {
  constexpr bool ENERGY = MODE != 1 && MODE != 4 && MODE != 6;  // MODE 5 sums 1/r where the energy goes
  constexpr bool SCALAR = MODE == 2 || MODE >= 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  HalfSmem& S = *reinterpret_cast<HalfSmem*>(smraw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NV = hood_nv(MODE);
  const int ntot = WIN ? *H.ndense : H.work[6];
  if (ntot == 0) {  // no cell of this kind
    if (tid < NV) partials[(size_t)blockIdx.x * NV + tid] = 0.0;
    return;
  }
  for (int k = tid; k < kWarps * 16; k += kThreads) (&S.out[0][0])[k] = 0.0;
  for (int k = tid; k < A.noff && k < kTab; k += kThreads) {
    const Off& o = A.off[k];
    S.otab[k] = make_float4(o.sx, o.sy, o.sz, __int_as_float(H.opk[1][k]));
  }
  for (int k = tid; k < kHome * 3; k += kThreads) (&S.hg[0][0])[k] = 0.f;
  if (tid == 0) S.ncand = 0;
  __syncthreads();
  if (tid == 0) {
    const int ne = A.noff < kTab ? A.noff : kTab;
    int nr = 0, pox = 0, poy = 0, poz = 0;
    for (int k = 1; k < ne; ++k) {
      int ox, oy, oz;
      unpack_off(__float_as_int(S.otab[k].w), ox, oy, oz);
      if (k == 1 || oy != poy || oz != poz || ox != pox + 1) S.rowk[nr++] = (unsigned short)k;
      pox = ox;
      poy = oy;
      poz = oz;
    }
    S.rowk[nr] = (unsigned short)(ne > 1 ? ne : 1);
    S.nrows = nr;
  }
  // scalar modes (energy, count, sum 1/r, histogram): the cutoff, the
  // histogram's copies after HalfSmem (as in k_hood), the lane's count
  ScalarRed R;
  R.rc2 = A.rc2;
  R.irc = A.irc;
  R.scale2 = H.hscale * H.hscale;
  R.xlim = H.hxlim;
  unsigned* const hist_all = reinterpret_cast<unsigned*>(smraw + sizeof(HalfSmem));
  R.hist = hist_all + (lane & (H.hcopies - 1)) * H.hstride;
  if (MODE == 6)
    for (int b = tid; b < H.hcopies * H.hstride; b += kThreads) hist_all[b] = 0u;
  unsigned cnt = 0;
  float wv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // lane's sum of (T.H) (x) f over its entries across the boundary
  float2 e = f2(0.f);
  const int* items = WIN ? H.dense : H.list;
  int* counter = WIN ? H.work + 5 : H.work;
  int next1 = 0;
  if (tid == 0) next1 = atomicAdd(counter, 1);
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      S.item = next1 < ntot ? items[next1] : -1;
      if (next1 < ntot) next1 = atomicAdd(counter, 1);
      S.nf = 0;
      S.nb = 0;
      S.next = 0;
    }
    __syncthreads();
    const int h = S.item;
    if (h < 0) break;
    const int hs = A.cell_start[h];
    const int nh = A.cell_start[h + 1] - hs;
    const int cx = h % A.nx, cy = (h / A.nx) % A.ny, cz = h / (A.nx * A.ny);
    constexpr bool win = WIN;
    if (WIN) {
      const unsigned long long cand = half_windowed<MODE>(A, H, S, hs, nh, cx, cy, cz, e, wv, cnt, R);
      if (tid == 0) S.ncand += cand;
    } else {
    float d = 0.f;
    for (int t = tid; t < kHome + 4; t += kThreads) {
      if (t < nh) {
        const float4 hq = A.xs[hs + t];
        d = fmaxf(d, fminf(sqrtf(fmaf(hq.x, hq.x, fmaf(hq.y, hq.y, hq.z * hq.z))), H.hd));
        S.home[t] = make_float4(-hq.x, -hq.y, -hq.z, __int_as_float(hs + t));  // negated: d = x_e + home
        S.own[t] = make_float4(hq.x, hq.y, hq.z, __int_as_float(hs + t));
      } else {
        S.home[t] = make_float4(kFar, -kFar, kFar, __int_as_float(0));  // padding: far from every entry
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    if (lane == 0) S.wmax[warp] = d;
    __syncthreads();
    float dmax = S.wmax[0];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) dmax = fmaxf(dmax, S.wmax[w]);
    const float top = H.rc + dmax + H.eps;
    half_stage(A, S, cx, cy, cz, top * top);
    __syncthreads();
    const int nf = min(S.nf, kHCap), nb = min(S.nb, kHCap - nf);  // k_hood_list guarantees nf + nb <= kHCap
    SeqInfo sq;
    sq.nf = nf;
    sq.nb = nb;
    sq.nh = nh;
    sq.obase = 0;
    sq.wf = 0;
    const int nseq = nf + nb + nh;
    const int nch = (nseq + kChunk - 1) / kChunk;
    const int cmask = (nf + nb) / kChunk;  // the first chunk holding own-cell positions
    if (tid == 0) S.ncand += (unsigned long long)nh * (unsigned long long)(nf + nb) + (unsigned long long)(nh * (nh - 1) / 2);
    // chunks of the sequence, taken from a counter; only the chunks holding
    // own-cell positions apply the order mask
    for (;;) {
      int c = 0;
      if (lane == 0) c = atomicAdd(&S.next, 1);
      c = __shfl_sync(0xffffffffu, c, 0);
      if (c >= nch) break;
      float2 jx[kEnt / 2], jy[kEnt / 2], jz[kEnt / 2];
      const int base = c * kChunk;
      const bool full = nseq - base > 64;  // else the chunk's second half is padding
      if (c < cmask) {
        if (full) half_chunk<false, false, MODE, 2>(S, sq, base, nh, A.rc2, A.irc, A.irc2, jx, jy, jz, e, cnt, R);
        else half_chunk<false, false, MODE, 1>(S, sq, base, nh, A.rc2, A.irc, A.irc2, jx, jy, jz, e, cnt, R);
      } else {
        if (full) half_chunk<true, false, MODE, 2>(S, sq, base, nh, A.rc2, A.irc, A.irc2, jx, jy, jz, e, cnt, R);
        else half_chunk<true, false, MODE, 1>(S, sq, base, nh, A.rc2, A.irc, A.irc2, jx, jy, jz, e, cnt, R);
      }
      if (!SCALAR) {
#pragma unroll
        for (int k = 0; k < kEnt / 2; ++k) {
          const int j0 = base + lane + 64 * k;
          half_flush(H, S, sq, j0, jx[k].x, jy[k].x, jz[k].x, wv);
          half_flush(H, S, sq, j0 + 32, jx[k].y, jy[k].y, jz[k].y, wv);
        }
      }
    }
    }  // fast path
    // this cell's energy and boundary terms into the warp's FP64 sums
    {
      float v[8] = {wv[0], wv[1], wv[2], wv[3], wv[4], wv[5], ENERGY ? e.x + e.y : 0.f, 0.f};
      warp_reduce_multi<8>(v);  // lane l: value l >> 2
      if ((lane & 3) == 0 && (lane >> 2) < 6) S.out[warp][lane >> 2] += -2.0 * (double)v[0];
      if (ENERGY && lane == 24) S.out[warp][15] += (double)v[0];
#pragma unroll
      for (int q = 0; q < 6; ++q) wv[q] = 0.f;
      e = f2(0.f);
    }
    __syncthreads();
    // the home particles' forces: minus their sums of fsn r (the windowed
    // path has added them per batch)
    if (!win && !SCALAR && tid < nh) {
      const float gx = S.hg[tid][0], gy = S.hg[tid][1], gz = S.hg[tid][2];
      if (gx != 0.f || gy != 0.f || gz != 0.f) atomicAdd(&H.hforce[hs + tid], make_float4(-gx, -gy, -gz, 0.f));
      S.hg[tid][0] = S.hg[tid][1] = S.hg[tid][2] = 0.f;
    }
  }
  // per-CTA partials: -2 (T.H) (x) f sums, energy (each pair-image once)
  __syncthreads();
  if (tid == 0 && S.ncand) atomicAdd(H.cand, S.ncand);
  if (MODE == 4) {
    unsigned long long c = cnt;
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0 && c) atomicAdd(H.count, c);
  }
  if (MODE == 6)
    for (int b = tid; b < H.nbins; b += kThreads) {
      unsigned c = 0;
      for (int q = 0; q < H.hcopies; ++q) c += hist_all[q * H.hstride + b];
      if (c) atomicAdd(&H.hist[b], (unsigned long long)c);
    }
  if (tid < NV) {
    int src;
    if (SCALAR) src = 15;
    else if (tid < kVirN3) src = tid;
    else if (MODE == 0) src = 15;
    else if (tid < kVirN3 + 9) src = -1;  // X: from k_half_finish
    else src = 15;
    double acc = 0.0;
    if (src >= 0)
      for (int w = 0; w < kWarps; ++w) acc += S.out[w][src];
    partials[(size_t)blockIdx.x * NV + tid] = acc;
  }
}

// Per particle i after the half-shell sweep: its force F (from the
// accumulated buffer, which it clears for the next launch), the outputs
// (MODE 0: forces; 1, 3: grad = -g F) and the per-CTA sums of -2 X (x) F
// (symmetric part) and, for the gradient modes, x_raw (x) F.
// FP32 <-> FP64 conversions from the IEEE bit layouts, on the integer pipes
// (this GPU issues FP64 conversions at a small fraction of the FP32 rate):
// f2d_bits is exact for finite values (FP32 subnormals, which the FTZ
// arithmetic producing them never yields, go to zero); d2f_bits rounds to
// nearest even, out of range to zero or infinity.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0) return (u >> 31) ? -0.0 : 0.0;
  const unsigned long long d = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(e == 255 ? 2047 : e + 896) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned s = (unsigned)(b >> 63) << 31;
  int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e <= 0) return __uint_as_float(s);
  unsigned m = (unsigned)((b >> 29) & 0x7fffffu);
  const unsigned long long rem = b & ((1ull << 29) - 1), half = 1ull << 28;
  if (rem > half || (rem == half && (m & 1u))) {
    if (++m == 0x800000u) {
      m = 0;
      ++e;
    }
  }
  if (e >= 255) return __uint_as_float(s | 0x7f800000u);
  return __uint_as_float(s | ((unsigned)e << 23) | m);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_half_finish(const __grid_constant__ SweepArgs A,
                                                     const __grid_constant__ HoodArgs H, float* __restrict__ forces,
                                                     double* __restrict__ grad, const double* __restrict__ gE,
                                                     const double* __restrict__ pos, double* __restrict__ partials) {
  constexpr bool GRAD = MODE == 1 || MODE == 3;
  constexpr int NV = hood_nv(MODE);
  const float g = GRAD ? (float)*gE : 0.f;
  float o[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) o[q] = 0.f;
  // original order: FP64 positions and gradients coalesced. Four particles per
  // thread and step, each load stage issued for all four before the next, so
  // that the dependent loads (cell start, then the accumulated force) overlap.
  constexpr int U = 4;
  const int stride = gridDim.x * blockDim.x;
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < A.n; i0 += U * stride) {
    float4 q[U];
    int p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * stride;
      q[u] = i < A.n ? H.xl[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      p[u] = i < A.n ? H.slot[i] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned cc = __float_as_uint(q[u].w);
      const int i = i0 + u * stride;
      if (i < A.n)
        p[u] += A.cell_start[(int)(cc & 1023u) + A.nx * ((int)((cc >> 10) & 1023u) + A.ny * (int)(cc >> 20))];
    }
    float4 f4[U];
#pragma unroll
    for (int u = 0; u < U; ++u) f4[u] = i0 + u * stride < A.n ? H.hforce[p[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * stride;
      if (i >= A.n) break;
      H.hforce[p[u]] = make_float4(0.f, 0.f, 0.f, 0.f);
      const unsigned cc = __float_as_uint(q[u].w);
      const float cx = (float)(cc & 1023u) + 0.5f, cy = (float)((cc >> 10) & 1023u) + 0.5f, cz = (float)(cc >> 20) + 0.5f;
      float X[3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
        X[a] = fmaf(cx, H.gf[a], fmaf(cy, H.gf[3 + a], cz * H.gf[6 + a])) + (a == 0 ? q[u].x : a == 1 ? q[u].y : q[u].z);
      const float F[3] = {f4[u].x, f4[u].y, f4[u].z};
      o[0] -= 2.f * X[0] * F[0];
      o[1] -= X[0] * F[1] + X[1] * F[0];
      o[2] -= X[0] * F[2] + X[2] * F[0];
      o[3] -= 2.f * X[1] * F[1];
      o[4] -= X[1] * F[2] + X[2] * F[1];
      o[5] -= 2.f * X[2] * F[2];
      if (MODE == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) forces[(size_t)i * 3 + a] = F[a];
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) grad[(size_t)i * 3 + a] = f2d_bits(-g * F[a]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float xa = d2f_bits(pos[(size_t)i * 3 + a]);
#pragma unroll
          for (int b = 0; b < 3; ++b) o[6 + a * 3 + b] = fmaf(xa, F[b], o[6 + a * 3 + b]);
        }
      }
    }
  }
  // -2 X (x) F sums already carry the sign of the partials; X (x) F as is
  warp_reduce_multi<16>(o);  // lane l: value l >> 1
  __shared__ double sm[8][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if ((lane & 1) == 0) sm[warp][lane >> 1] = (double)o[0];
  __syncthreads();
  if (threadIdx.x < NV) {
    int src;  // column of o for partial threadIdx.x
    if (threadIdx.x < kVirN3) src = threadIdx.x;
    else if (MODE == 0) src = -1;  // energy: from the sweep
    else if (threadIdx.x < kVirN3 + 9) src = threadIdx.x;
    else src = -1;
    double acc = 0.0;
    if (src >= 0)
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += sm[w][src];
    partials[(size_t)blockIdx.x * NV + threadIdx.x] = acc;
  }
}

}  // namespace

// Shared memory of k_hood<mode>: Smem, and for the histogram its copies (the
// most of the size the grid is sized for; at least one copy).
constexpr int kHistWords = 1408;  // histogram copies fitting five CTAs per SM
static_assert(hist_stride(kMaxBins) >= kHistWords, "the largest histogram bounds every copy set");
size_t hood_mode_smem(int mode) {
  return sizeof(Smem) + (mode == 6 ? sizeof(unsigned) * (size_t)hist_stride(kMaxBins) : 0);
}
int hist_copies(int nbins) {
  int c = 8;
  while (c > 1 && c * hist_stride(nbins) > kHistWords) c >>= 1;
  return c;
}

int hood_grid(int mode) {
  static DevCache cached[7];
  if (mode < 0 || mode > 6) return 0;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (const int c = cached[mode].get(dev)) return c;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cudaError_t e;
  const size_t sm = hood_mode_smem(mode);
  if (mode == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood<0>, kThreads, sm);
  else if (mode == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood<1>, kThreads, sm);
  else if (mode == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood<2>, kThreads, sm);
  else if (mode == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood<3>, kThreads, sm);
  else if (mode == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood<4>, kThreads, sm);
  else if (mode == 5) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood<5>, kThreads, sm);
  else {
    e = cudaFuncSetAttribute(k_hood<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood<6>, kThreads, sm);
  }
  if (e != cudaSuccess || per < 1) return 0;
  cached[mode].put(dev, sms * per);
  return sms * per;
}

size_t hood_smem_bytes() { return sizeof(Smem); }

// Persistent CTAs of the half-shell sweep, per mode (0, 1, 3).
// Shared memory of k_hood_half<mode>: HalfSmem, and for the histogram its
// largest set of copies.
size_t half_mode_smem(int mode) {
  return sizeof(HalfSmem) + (mode == 6 ? sizeof(unsigned) * (size_t)hist_stride(kMaxBins) : 0);
}

template <int M>
cudaError_t half_setup(int bytes, int* per) {
  cudaError_t e = cudaFuncSetAttribute(k_hood_half<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hood_half<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_hood_half<M, false>, kThreads, bytes);
  return e;
}

// Persistent CTAs of the half-shell sweep, per mode (0, 1, 3; scalar 2, 4,
// 5, 6); also raises the kernels' shared-memory limit on the current device.
int half_grid(int mode) {
  static DevCache cached[7];
  if (mode < 0 || mode > 6) return 0;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (const int c = cached[mode].get(dev)) return c;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int bytes = (int)half_mode_smem(mode);
  cudaError_t e;
  switch (mode) {
    case 0: e = half_setup<0>(bytes, &per); break;
    case 1: e = half_setup<1>(bytes, &per); break;
    case 3: e = half_setup<3>(bytes, &per); break;
    case 2: e = half_setup<2>(bytes, &per); break;
    case 4: e = half_setup<4>(bytes, &per); break;
    case 5: e = half_setup<5>(bytes, &per); break;
    default: e = half_setup<6>(bytes, &per); break;
  }
  if (e != cudaSuccess || per < 1) return 0;
  cached[mode].put(dev, sms * per);
  return sms * per;
}

// Persistent CTAs of the dense-cell sweep (all resident), per mode; also
// raises the kernels' shared-memory limit on the current device.
int dense_grid(int mode) {
  static DevCache cached[4];
  if (mode < 0 || mode > 3) return 0;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (const int c = cached[mode].get(dev)) return c;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int most = (int)dense_smem_bytes(kMaxOff);
  cudaError_t e;
  if (mode == 0) {
    e = cudaFuncSetAttribute(k_hood_dense<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood_dense<0>, kDenseThreads, most);
  } else if (mode == 1) {
    e = cudaFuncSetAttribute(k_hood_dense<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood_dense<1>, kDenseThreads, most);
  } else if (mode == 2) {
    e = cudaFuncSetAttribute(k_hood_dense<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood_dense<2>, kDenseThreads, most);
  } else {
    e = cudaFuncSetAttribute(k_hood_dense<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hood_dense<3>, kDenseThreads, most);
  }
  if (e != cudaSuccess || per < 1) return 0;
  cached[mode].put(dev, sms * per);
  return sms * per;
}

// Occupancy grid of a kernel with `smem` bytes of dynamic shared memory.
template <class K>
int grid_for(K kernel, size_t smem) {
  int per = 0, sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, smem) != cudaSuccess || per < 1)
    return 0;
  return sms * per;
}

bool hood_half_fits(const SweepArgs& A) { return A.noff <= kTab; }

// Scalar reductions over the half stencil. When the stencil fits the table,
// the work lists of the half-shell sweep split the cells: the fast-path cells
// (at most kHome particles, at most kHCap in the half neighbourhood) go to the
// home-major k_hood<mode>, the others to the windowed k_hood_half<mode, true>
// (octant batches, index lists); otherwise k_hood<mode> takes the cells it can
// and the per-particle sweep the rest. Measured with the half-shell kernel
// alone for every cell: 1M lattice count 0.60 against 0.57 ms, histogram 1.05
// against 0.93 ms (the home-major kernel is faster on small cells).
int launch_hood_scalar(const SweepArgs& A, const HoodArgs& Hin, int* work, int kind, unsigned long long* count,
                       double* partials, long long partials_cap, double* sums, double* scalar_out, int nbins,
                       float rmax, unsigned long long* hist, cudaStream_t s, int* lists_half) {
  if (kind < 0 || kind > 3) return CL_ERR_INVALID_ARG;
  const int mode = kind == 3 ? 2 : 4 + kind;
  const bool scalar = kind == 1 || kind == 3;  // FP64 partials and a final reduction
  const int final_mode = kind == 3 ? 1 : 0;
  if (kind == 2 && (nbins < 1 || nbins > kMaxBins || !(rmax > 0.f))) return CL_ERR_INVALID_ARG;
  const bool half = hood_half_fits(A);
  if (kind == 3 && !half) return CL_ERR_UNSUPPORTED;  // the caller takes launch_hood's mode 2
  HoodArgs H = Hin;
  H.work = work;
  H.cand = reinterpret_cast<unsigned long long*>(work + 2);
  H.ndense = work + 7;
  H.half = half ? 1 : 0;
  H.count = count;
  H.hist = hist;
  H.nbins = kind == 2 ? nbins : 0;
  H.rmax = kind == 2 ? rmax : 0.f;
  H.hscale = kind == 2 ? (float)nbins / rmax : 0.f;
  H.hxlim = kind == 2 ? (float)std::min((double)nbins, (double)Hin.rc * ((double)nbins / rmax)) : 0.f;
  H.hcopies = kind == 2 ? hist_copies(nbins) : 1;
  H.hstride = kind == 2 ? hist_stride(nbins) : 0;
  const bool reuse = half && lists_half && *lists_half;  // the half-shell work lists of this cell list are built
  if (cudaMemsetAsync(work, 0, (reuse ? 6 : 8) * sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  if (kind == 0 && cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess) return CL_ERR_CUDA;
  if (kind == 2 && cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * nbins, s) != cudaSuccess) return CL_ERR_CUDA;
  if (A.n <= 0) {
    if (!scalar) return CL_OK;
    if (cudaMemsetAsync(partials, 0, sizeof(double), s) != cudaSuccess) return CL_ERR_CUDA;
    return finish_reduction(final_mode, 3, nullptr, 1, 1, partials, sums, scalar_out, nullptr, nullptr, nullptr, s);
  }
  if (lists_half) *lists_half = half ? 1 : 0;
  // grids: the home-major kernel, and (half) the windowed kernel
  const size_t hist_bytes = kind == 2 ? sizeof(unsigned) * (size_t)H.hcopies * H.hstride : 0;
  const size_t smem = sizeof(Smem) + hist_bytes, hsmem = sizeof(HalfSmem) + hist_bytes;
  if (hood_grid(mode) <= 0 || (half && half_grid(mode) <= 0)) return CL_ERR_CUDA;  // also raise the smem limits
  int nb = 0, nhb = 0;
  switch (mode) {
    case 2: nb = grid_for(k_hood<2>, smem); nhb = grid_for(k_hood_half<2, true>, hsmem); break;
    case 4: nb = grid_for(k_hood<4>, smem); nhb = grid_for(k_hood_half<4, true>, hsmem); break;
    case 5: nb = grid_for(k_hood<5>, smem); nhb = grid_for(k_hood_half<5, true>, hsmem); break;
    default: nb = grid_for(k_hood<6>, smem); nhb = grid_for(k_hood_half<6, true>, hsmem); break;
  }
  if (nb <= 0 || nhb <= 0) return CL_ERR_CUDA;
  nb = std::min(nb, Hin.ncells);
  nhb = half ? std::min(nhb, Hin.ncells) : 0;
  const int nrest = half ? 0 : flagged_blocks(A.n);
  if (scalar && nb + nhb + nrest > partials_cap) return CL_ERR_INVALID_ARG;
  if (!reuse) {
    k_hood_list<<<(H.ncells + 255) / 256, 256, 0, s>>>(A.cell_start, H.ncells, A.noff, work, H.list, H.flag, H.dense,
                                                       H.ndense, H, half ? A.noff : 0, A.nx, A.ny, A.nz);
    if (half && launch_octsort(H.dense, H.ndense, A.cell_start, const_cast<float4*>(A.xs), const_cast<int*>(H.slot),
                               s) != CL_OK)
      return CL_ERR_CUDA;
  }
  double* p2 = partials + nb;
  switch (mode) {
    case 2:
      k_hood<2><<<nb, kThreads, smem, s>>>(A, H, nullptr, nullptr, nullptr, nullptr, partials);
      k_hood_half<2, true><<<nhb, kThreads, hsmem, s>>>(A, H, p2);
      break;
    case 4:
      k_hood<4><<<nb, kThreads, smem, s>>>(A, H, nullptr, nullptr, nullptr, nullptr, partials);
      if (half) k_hood_half<4, true><<<nhb, kThreads, hsmem, s>>>(A, H, p2);
      break;
    case 5:
      k_hood<5><<<nb, kThreads, smem, s>>>(A, H, nullptr, nullptr, nullptr, nullptr, partials);
      if (half) k_hood_half<5, true><<<nhb, kThreads, hsmem, s>>>(A, H, p2);
      break;
    default:
      k_hood<6><<<nb, kThreads, smem, s>>>(A, H, nullptr, nullptr, nullptr, nullptr, partials);
      if (half) k_hood_half<6, true><<<nhb, kThreads, hsmem, s>>>(A, H, p2);
      break;
  }
  if (cudaGetLastError() != cudaSuccess) return CL_ERR_CUDA;
  if (!half) {  // one thread per particle for the cells the staged sweep left (flag != 0)
    int e = CL_OK;
    if (kind == 0) e = launch_count_flagged(A, H.flag, count, s);
    else if (kind == 2) e = launch_hist_flagged(A, H.flag, nbins, rmax, hist, s);
    else e = launch_suminvr_flagged(A, H.flag, partials + nb, s);
    if (e != CL_OK) return e;
  }
  if (!scalar) return CL_OK;
  return finish_reduction(final_mode, 3, nullptr, nb + nhb + nrest, 1, partials, sums, scalar_out, nullptr, nullptr,
                          nullptr, s);
}

int fill_hood_args(const Geo& geo, const int* opk_full, int noff_full, const int* opk_half, int noff_half,
                   HoodArgs* H) {
  std::memset(H, 0, sizeof(*H));
  for (int k = 0; k < noff_full && k < kMaxOff; ++k) H->opk[0][k] = opk_full[k];
  for (int k = 0; k < noff_half && k < kMaxOff; ++k) H->opk[1][k] = opk_half[k];
  {  // rows of the half stencil, for the work lists' neighbourhood counts
    int nr = 0;
    bool fits = true;
    for (int k = 1; k < noff_half && k < kMaxOff; ++k) {
      const int v = opk_half[k];
      const int ox = (signed char)(v & 0xff), oy = (signed char)((v >> 8) & 0xff), oz = (signed char)((v >> 16) & 0xff);
      if (nr > 0 && H->rows_half[nr - 1][2] == oy && H->rows_half[nr - 1][3] == oz && H->rows_half[nr - 1][1] + 1 == ox) {
        H->rows_half[nr - 1][1] = (signed char)ox;
        continue;
      }
      if (nr == 128) {
        fits = false;
        break;
      }
      H->rows_half[nr][0] = H->rows_half[nr][1] = (signed char)ox;
      H->rows_half[nr][2] = (signed char)oy;
      H->rows_half[nr][3] = (signed char)oz;
      ++nr;
    }
    H->nrows_half = fits ? nr : 0;
  }
  double hd = 0.0;
  for (int s = 0; s < 8; ++s) {
    double v[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
      const double sg = ((s >> k) & 1) ? 0.5 : -0.5;
      for (int a = 0; a < 3; ++a) v[a] += sg * geo.h[k * 3 + a] / geo.n[k];
    }
    const double d = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (d > hd) hd = d;
  }
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) {
      H->g[k * 3 + a] = geo.h[k * 3 + a] / geo.n[k];
      H->gf[k * 3 + a] = (float)H->g[k * 3 + a];
      H->hrow[k * 3 + a] = (float)geo.h[k * 3 + a];
    }
  const double eps = 1e-4 * (geo.rc + hd);
  H->rc = (float)geo.rc;
  H->hd = (float)(hd * (1.0 + 1e-6));
  H->eps = (float)eps;
  H->ncells = (int)geo.ncells;
  return CL_OK;
}

bool half_path_applies(const SweepArgs& A, const SweepArgs* Ahalf, const HoodArgs& H, int mode) {
  return Ahalf && mode != 2 && H.hforce && A.noff <= kTab && Ahalf->noff <= kTab && A.n > 0;
}

int launch_hood(const SweepArgs& A, const SweepArgs* Ahalf, const HoodArgs& Hin, int* work, int mode,
                const double* hinv, float* forces, double* grad, const double* gE, const double* pos,
                double* partials, long long partials_cap, double* sums, double* energy, double* virial,
                double* gradbox, cudaStream_t s, int* lists_half) {
  const int NV = hood_nv(mode);
  const bool half = half_path_applies(A, Ahalf, Hin, mode);
  const int nrest = (A.n + 255) / 256;  // CTAs of the companion sweep (and bound of the finish grid)
  const int final_mode = mode == 2 ? 1 : (mode == 0 ? 2 : (mode == 1 ? 3 : 4));
  HoodArgs H = Hin;
  H.work = work;
  H.cand = reinterpret_cast<unsigned long long*>(work + 2);
  H.ndense = work + 7;
  H.half = half ? 1 : 0;
  // the half-shell work lists depend on the cell list only: built once per
  // list (lists_half says whether the buffers hold them) and reused
  const bool reuse = half && lists_half && *lists_half;
  if (cudaMemsetAsync(work, 0, (reuse ? 6 : 8) * sizeof(int), s) != cudaSuccess) return CL_ERR_CUDA;
  if (!reuse) {
    k_hood_list<<<(H.ncells + 255) / 256, 256, 0, s>>>(A.cell_start, H.ncells, A.noff, work, H.list, H.flag,
                                                       H.dense, H.ndense, H, half ? Ahalf->noff : 0, A.nx, A.ny, A.nz);
    // the windowed cells' particles in octant order (half_windowed's batches)
    if (half && launch_octsort(H.dense, H.ndense, A.cell_start, const_cast<float4*>(A.xs), const_cast<int*>(H.slot),
                               s) != CL_OK)
      return CL_ERR_CUDA;
  }
  if (lists_half) *lists_half = half ? 1 : 0;
  if (half) {
    // every non-empty cell: fast-path or windowed half-shell sweep, then the
    // per-particle finish; partials [sweep][finish]
    // (the windowed kernel's CTAs exit at once when no cell needs it)
    int nhb = half_grid(mode);
    const int nfin = std::min(nrest, 152 * 8);
    if (nhb <= 0) return CL_ERR_CUDA;
    if (nhb > Hin.ncells) nhb = Hin.ncells;
    if (2 * nhb > partials_cap / NV - nfin) nhb = (int)((partials_cap / NV - nfin) / 2);
    if (nhb < 1) return CL_ERR_INVALID_ARG;
    double* pwin = partials + (size_t)nhb * NV;
    double* pfin = pwin + (size_t)nhb * NV;
    const size_t hsmem = sizeof(HalfSmem);
    if (mode == 0) {
      k_hood_half<0, false><<<nhb, kThreads, hsmem, s>>>(*Ahalf, H, partials);
      k_hood_half<0, true><<<nhb, kThreads, hsmem, s>>>(*Ahalf, H, pwin);
      k_half_finish<0><<<nfin, 256, 0, s>>>(*Ahalf, H, forces, grad, gE, pos, pfin);
    } else if (mode == 1) {
      k_hood_half<1, false><<<nhb, kThreads, hsmem, s>>>(*Ahalf, H, partials);
      k_hood_half<1, true><<<nhb, kThreads, hsmem, s>>>(*Ahalf, H, pwin);
      k_half_finish<1><<<nfin, 256, 0, s>>>(*Ahalf, H, forces, grad, gE, pos, pfin);
    } else {
      k_hood_half<3, false><<<nhb, kThreads, hsmem, s>>>(*Ahalf, H, partials);
      k_hood_half<3, true><<<nhb, kThreads, hsmem, s>>>(*Ahalf, H, pwin);
      k_half_finish<3><<<nfin, 256, 0, s>>>(*Ahalf, H, forces, grad, gE, pos, pfin);
    }
    return finish_reduction(final_mode, 3, hinv, 2 * nhb + nfin, NV, partials, sums, energy, virial, gradbox, gE, s);
  }
  // full-shell kernels (and the half-stencil energy, mode 2): partials
  // [neighbourhood sweep][companion][dense cells]
  const int ndc = dense_grid(mode);  // CTAs of the dense-cell sweep
  int nb = hood_grid(mode);
  if (nb <= 0 || ndc <= 0) return CL_ERR_CUDA;
  if (nb > Hin.ncells) nb = Hin.ncells;
  if (nb > partials_cap / NV - nrest - ndc) nb = (int)(partials_cap / NV - nrest - ndc);
  if (nb < 1) return CL_ERR_INVALID_ARG;
  double* rest = partials + (size_t)nb * NV;
  double* dpart = rest + (size_t)nrest * NV;
  const size_t smem = sizeof(Smem);
  const size_t dsmem = dense_smem_bytes(A.noff);
  if (mode == 0) {
    k_hood<0><<<nb, kThreads, smem, s>>>(A, H, forces, grad, gE, pos, partials);
    k_hood_rest<0><<<nrest, 256, 0, s>>>(A, H, forces, grad, gE, pos, rest);
    k_hood_dense<0><<<ndc, kDenseThreads, dsmem, s>>>(A, H, forces, grad, gE, pos, dpart);
  } else if (mode == 1) {
    k_hood<1><<<nb, kThreads, smem, s>>>(A, H, forces, grad, gE, pos, partials);
    k_hood_rest<1><<<nrest, 256, 0, s>>>(A, H, forces, grad, gE, pos, rest);
    k_hood_dense<1><<<ndc, kDenseThreads, dsmem, s>>>(A, H, forces, grad, gE, pos, dpart);
  } else if (mode == 2) {
    k_hood<2><<<nb, kThreads, smem, s>>>(A, H, forces, grad, gE, pos, partials);
    k_hood_rest<2><<<nrest, 256, 0, s>>>(A, H, forces, grad, gE, pos, rest);
    k_hood_dense<2><<<ndc, kDenseThreads, dsmem, s>>>(A, H, forces, grad, gE, pos, dpart);
  } else {
    k_hood<3><<<nb, kThreads, smem, s>>>(A, H, forces, grad, gE, pos, partials);
    k_hood_rest<3><<<nrest, 256, 0, s>>>(A, H, forces, grad, gE, pos, rest);
    k_hood_dense<3><<<ndc, kDenseThreads, dsmem, s>>>(A, H, forces, grad, gE, pos, dpart);
  }
  return finish_reduction(final_mode, 3, hinv, nb + nrest + ndc, NV, partials, sums, energy, virial, gradbox, gE,
                          s);
}

}  // namespace clk
