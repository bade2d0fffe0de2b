// cl_geom.cu -- host-side box preparation: lattice inverse, face distances,
// cell grid, and the neighbour-cell stencil with its per-offset shifts.
//
// Grid (Sec. 2.8 "partitioning the space into cells ... by integer division",
// lcell of Sec. 2.8 / Code 3): cells are a fractional grid of the lattice,
// n_k = max(1, floor(w_k lcell / rc)) cells along lattice vector k, w_k the
// distance between the two faces spanned by the other vectors. Each cell is
// then at least rc/lcell thick across every face, and two particles whose cells
// differ by more than m_k = ceil(rc n_k / w_k) along axis k are farther apart
// than rc. For an orthorhombic box this is the paper's Code 3 grid: sides
// [10,20,15] and rc 1.2 give [8,16,12] periodic cells of side 1.25 (the paper
// prints them with one ghost layer on each side, [10,18,14]).
//
// Stencil: every integer offset o with |o_k| <= m_k whose two cells can hold a
// pair closer than rc. The minimum distance between cell 0 and cell o is an
// exact box-constrained least-squares problem, min |sum_k d_k G_k| over
// d_k in [o_k - 1, o_k + 1] (G_k = H_k / n_k), solved by enumerating the 3^D
// active sets. Offsets whose cells stay at least rc apart are dropped; for a
// cubic box at lcell = 3 that removes the 3x3x3 corner offsets, for instance.
//
// Half shell (Sec. 2.8: "only half of the neighboring cells are evaluated"):
// the offsets that are lexicographically positive in (z, y, x) plus the own
// cell, where pairs are taken with j after i. Offset o covers the pair-image
// (i, j, T) and offset -o the same pair-image seen from j, so the half shell
// visits each pair-image once. This holds for any lattice, not only the
// orthorhombic one the paper uses it for.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cl_internal.cuh"

namespace clk {

static bool inv3(const double* a, double* o) {
  double c00 = a[4] * a[8] - a[5] * a[7];
  double c01 = a[5] * a[6] - a[3] * a[8];
  double c02 = a[3] * a[7] - a[4] * a[6];
  double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  if (!(std::fabs(det) > 0) || !std::isfinite(det)) return false;
  o[0] = c00 / det;
  o[3] = c01 / det;
  o[6] = c02 / det;
  o[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  o[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  o[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  o[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  o[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  o[8] = (a[0] * a[4] - a[1] * a[3]) / det;
  return true;
}

int prepare_geometry(const cl_box* box, Geo* g) {
  if (!box) return CL_ERR_INVALID_ARG;
  const int dim = box->dim;
  if (dim != 2 && dim != 3) return CL_ERR_INVALID_ARG;
  if (!(box->cutoff > 0) || !std::isfinite(box->cutoff)) return CL_ERR_INVALID_ARG;
  if (box->lcell < 1 || box->lcell > 4) return CL_ERR_INVALID_ARG;
  std::memset(g, 0, sizeof(*g));
  g->dim = dim;
  g->rc = box->cutoff;
  g->lcell = box->lcell;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g->h[a * 3 + b] = (a == b) ? 1.0 : 0.0;
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b) {
      double v = box->h[a * dim + b];
      if (!std::isfinite(v)) return CL_ERR_INVALID_BOX;
      g->h[a * 3 + b] = v;
    }
  if (!inv3(g->h, g->hinv)) return CL_ERR_INVALID_BOX;
  g->ortho = 1;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (a != b && g->h[a * 3 + b] != 0.0) g->ortho = 0;
  long long ncells = 1;
  for (int k = 0; k < 3; ++k) {
    double q = 0;
    for (int a = 0; a < 3; ++a) q += g->hinv[a * 3 + k] * g->hinv[a * 3 + k];
    g->w[k] = 1.0 / std::sqrt(q);
    if (k < dim) {
      if (!(g->rc < g->w[k])) return CL_ERR_CUTOFF_TOO_LARGE;
      double nk = std::floor(g->w[k] * g->lcell / g->rc);
      if (nk < 1) nk = 1;
      if (nk > kMaxAxis) nk = kMaxAxis;
      g->n[k] = (int)nk;
    } else {
      g->n[k] = 1;
    }
    ncells *= g->n[k];
  }
  if (ncells > (1LL << 28)) return CL_ERR_UNSUPPORTED;
  g->ncells = ncells;
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) g->m[a * 3 + k] = g->hinv[a * 3 + k] * g->n[k];
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) g->g[k * 3 + a] = (float)(g->h[k * 3 + a] / g->n[k]);
  return CL_OK;
}

// Squared minimum distance between cell 0 and cell o of the grid: the minimum
// of |sum_k d_k G_k|^2 with d_k in [o_k - 1, o_k + 1], k < dim.
static double min_dist2(const Geo& geo, const int* o) {
  const int dim = geo.dim;
  double G[3][3];
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) G[k][a] = geo.h[k * 3 + a] / geo.n[k];
  int npat = 1;
  for (int k = 0; k < dim; ++k) npat *= 3;
  double best = INFINITY;
  for (int p = 0; p < npat; ++p) {
    int st[3], q = p;
    for (int k = 0; k < dim; ++k) { st[k] = q % 3; q /= 3; }
    double lo[3], hi[3], d[3];
    int freek[3], nf = 0;
    double v0[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
      lo[k] = o[k] - 1.0;
      hi[k] = o[k] + 1.0;
      if (st[k] == 2) { freek[nf++] = k; continue; }
      d[k] = (st[k] == 0) ? lo[k] : hi[k];
      for (int a = 0; a < 3; ++a) v0[a] += d[k] * G[k][a];
    }
    // normal equations A df = -b for the free coordinates
    double A[3][3], b[3];
    for (int r = 0; r < nf; ++r) {
      b[r] = 0;
      for (int a = 0; a < 3; ++a) b[r] += G[freek[r]][a] * v0[a];
      for (int c = 0; c < nf; ++c) {
        A[r][c] = 0;
        for (int a = 0; a < 3; ++a) A[r][c] += G[freek[r]][a] * G[freek[c]][a];
      }
    }
    double sol[3] = {0, 0, 0};
    if (nf == 1) {
      sol[0] = -b[0] / A[0][0];
    } else if (nf == 2) {
      double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
      if (!(std::fabs(det) > 0)) continue;
      sol[0] = (-b[0] * A[1][1] + b[1] * A[0][1]) / det;
      sol[1] = (-b[1] * A[0][0] + b[0] * A[1][0]) / det;
    } else if (nf == 3) {
      double Af[9] = {A[0][0], A[0][1], A[0][2], A[1][0], A[1][1], A[1][2], A[2][0], A[2][1], A[2][2]}, Ai[9];
      if (!inv3(Af, Ai)) continue;
      for (int r = 0; r < 3; ++r) sol[r] = -(Ai[r * 3 + 0] * b[0] + Ai[r * 3 + 1] * b[1] + Ai[r * 3 + 2] * b[2]);
    }
    bool feasible = true;
    for (int r = 0; r < nf; ++r) {
      int k = freek[r];
      if (sol[r] < lo[k] - 1e-12 || sol[r] > hi[k] + 1e-12) feasible = false;
      d[k] = sol[r];
    }
    if (!feasible) continue;
    double v[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k)
      for (int a = 0; a < 3; ++a) v[a] += d[k] * G[k][a];
    double q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (q2 < best) best = q2;
  }
  return best;
}

void cell_halfwidths(const Geo& geo, float* e) {
  for (int a = 0; a < 3; ++a) {
    double s = 0.0;
    for (int k = 0; k < geo.dim; ++k) s += std::fabs(geo.h[k * 3 + a]) / geo.n[k];
    e[a] = (float)(0.5 * s + 1e-3 * geo.rc);
  }
}

int build_stencil(const Geo& geo, int half, Off* out, int cap, int* opk) {
  const int dim = geo.dim;
  int m[3] = {0, 0, 0};
  for (int k = 0; k < dim; ++k) m[k] = (int)std::ceil(geo.rc * geo.n[k] / geo.w[k]);
  const double keep2 = geo.rc * geo.rc * (1.0 + 1e-9);
  std::vector<Off> v;
  std::vector<int> pk;
  // own cell first
  for (int pass = 0; pass < 2; ++pass)
    for (int oz = -m[2]; oz <= m[2]; ++oz)
      for (int oy = -m[1]; oy <= m[1]; ++oy)
        for (int ox = -m[0]; ox <= m[0]; ++ox) {
          const bool self = (ox == 0 && oy == 0 && oz == 0);
          if ((pass == 0) != self) continue;
          if (half && !self) {
            bool positive = (oz > 0) || (oz == 0 && (oy > 0 || (oy == 0 && ox > 0)));
            if (!positive) continue;
          }
          int o[3] = {ox, oy, oz};
          if (!self && min_dist2(geo, o) >= keep2) continue;
          Off e;
          int d[3];
          for (int k = 0; k < 3; ++k) d[k] = ((o[k] % geo.n[k]) + geo.n[k]) % geo.n[k];
          e.dx = d[0];
          e.dy = d[1];
          e.dz = d[2];
          double s[3] = {0, 0, 0};
          for (int k = 0; k < dim; ++k)
            for (int a = 0; a < 3; ++a) s[a] += (double)o[k] / geo.n[k] * geo.h[k * 3 + a];
          e.sx = (float)s[0];
          e.sy = (float)s[1];
          e.sz = (float)s[2];
          v.push_back(e);
          pk.push_back((ox & 255) | ((oy & 255) << 8) | ((oz & 255) << 16));
        }
  if ((int)v.size() > cap) return CL_ERR_UNSUPPORTED;
  std::copy(v.begin(), v.end(), out);
  if (opk) std::copy(pk.begin(), pk.end(), opk);
  return (int)v.size();
}

}  // namespace clk
