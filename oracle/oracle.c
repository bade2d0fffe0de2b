/*
 * oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the cell-list
 * pair map of CellListMap.jl (Martinez, arXiv 2202.06427).
 *
 * TEST INFRASTRUCTURE. This file is the independent definition that the CUDA
 * path is checked against. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it. It shares no code, header, table or
 * constant with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, and where the paper states it:
 *
 *  - Sec. 2.3 (Code 2): the mapped function is evaluated once for every pair
 *    of particles closer than the cutoff, given the two positions under the
 *    periodic images and the squared distance.
 *  - Sec. 2.6 (Fig. 1): ghost copies of the real particles "guarantee the
 *    correct number of neighbours" under periodic boundaries. Read as the set
 *    of pair-images
 *        P = { (i, j, t) : i < j, t integer, |x_j - x_i + t.H| < rc },
 *    where the rows of H are the lattice vectors. When rc <= w_min/2 every
 *    pair has at most one such t (the minimum image).
 *  - Sec. 2.8: cells come from integer division of the coordinates, and a
 *    loop over cells and their neighbouring cells visits the candidates.
 *
 * Oracle algorithm (all FP64, no half shell, no projection, no FP32):
 *   1. fractional coordinates s = x.H^-1, wrapped s - floor(s);
 *   2. a fractional grid whose cells are at least rc wide across each face,
 *      n_k = max(1, floor(w_k / rc)), w_k the distance between lattice planes;
 *   3. for every particle i and every offset o of the FULL stencil
 *      {-m..m}^D with m_k = ceil(rc n_k / w_k): neighbour cell (c+o) mod n and
 *      image T = floor((c+o)/n);
 *   4. accept (i, j, T) when i < j and |x_j - x_i + T.H| < rc.
 *   When n_k < 2 m_k + 1 one cell is reached under several T: each is a
 *   distinct pair-image, as the definition of P requires.
 *
 * Reductions over P (the built-ins of the library):
 *   count, sum 1/r (Code 5), shifted-force energy
 *   u(r) = 1/r - 1/rc + (r - rc)/rc^2 with forces F = -dE/dx (Code 7 pattern:
 *   f[i] += g, f[j] -= g), virial W = -sum u'(r)/r r (x) r, the gradient of E
 *   with respect to H at fixed Cartesian positions, a distance histogram
 *   (Code 10 pattern) and the i<j neighbour list (Sec. 4.1).
 *
 * Band accounting. A pair whose FP64 distance lies within band*rc of the
 * cutoff, or of a histogram bin edge, may be classified either way by a
 * correct FP32 implementation. Such pairs are counted separately so that a
 * test can accept either classification and report how many there were.
 *
 * The brute-force routines (or_brute_*) loop over all i<j and all integer
 * image vectors with |t_k| <= ceil(rc/w_k)+1: O(n^2 * images), for n <= ~300.
 * They pin the cell-list oracle.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_BOX -2
#define OR_ERR_IMAGES -3   /* pair list asked for, but a pair has two images within rc */
#define OR_ERR_CAPACITY -4
#define OR_ERR_OOM -5

typedef struct {
  int dim;
  double h[3][3];    /* rows = lattice vectors */
  double hinv[3][3]; /* s = x . hinv */
  double w[3];       /* distances between opposite faces */
} geom;

/* Inverse of the lattice matrix, widths between faces. */
static int geom_init(geom* g, int dim, const double* h) {
  if (dim != 2 && dim != 3) return OR_ERR_ARG;
  memset(g, 0, sizeof(*g));
  g->dim = dim;
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b) g->h[a][b] = h[a * dim + b];
  double det;
  if (dim == 2) {
    det = g->h[0][0] * g->h[1][1] - g->h[0][1] * g->h[1][0];
    if (!(fabs(det) > 0) || !isfinite(det)) return OR_ERR_BOX;
    g->hinv[0][0] = g->h[1][1] / det;
    g->hinv[0][1] = -g->h[0][1] / det;
    g->hinv[1][0] = -g->h[1][0] / det;
    g->hinv[1][1] = g->h[0][0] / det;
  } else {
    double(*m)[3] = g->h;
    double c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
    double c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
    double c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
    det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
    if (!(fabs(det) > 0) || !isfinite(det)) return OR_ERR_BOX;
    /* inverse = adjugate / det; adjugate = transpose of the cofactor matrix */
    g->hinv[0][0] = c00 / det;
    g->hinv[1][0] = c01 / det;
    g->hinv[2][0] = c02 / det;
    g->hinv[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det;
    g->hinv[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det;
    g->hinv[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / det;
    g->hinv[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det;
    g->hinv[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det;
    g->hinv[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / det;
  }
  /* Column k of H^-1 is the reciprocal vector b_k (a_i . b_k = delta_ik); the
   * planes s_k = 0 and s_k = 1 are 1/|b_k| apart. */
  for (int k = 0; k < dim; ++k) {
    double q = 0;
    for (int a = 0; a < dim; ++a) q += g->hinv[a][k] * g->hinv[a][k];
    g->w[k] = 1.0 / sqrt(q);
  }
  return OR_OK;
}

static long long floordiv_ll(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

/* The oracle's own cell list: wrapped positions, integer wrap counts, and a
 * counting sort of particle indices by cell. */
typedef struct {
  int n[3], m[3];
  long long ncell;
  double* xw;      /* wrapped Cartesian positions, n*dim */
  double* fl;      /* floor(s) per particle and axis, n*dim */
  int* cell;       /* per particle: linear cell index */
  long long* start;/* ncell+1 */
  long long* order;/* particle indices sorted by cell */
} clist;

static void clist_free(clist* c) {
  free(c->xw); free(c->fl); free(c->cell); free(c->start); free(c->order);
  memset(c, 0, sizeof(*c));
}

static int clist_build(clist* cl, const geom* g, long long np, const double* x, double rc_grid) {
  const int dim = g->dim;
  memset(cl, 0, sizeof(*cl));
  long long ncell = 1;
  for (int k = 0; k < dim; ++k) {
    double nk = floor(g->w[k] / rc_grid);
    if (nk < 1) nk = 1;
    if (nk > 1024) nk = 1024; /* cells stay >= rc wide; the grid is only capped for memory */
    cl->n[k] = (int)nk;
    cl->m[k] = (int)ceil(rc_grid * cl->n[k] / g->w[k]);
    ncell *= cl->n[k];
  }
  cl->ncell = ncell;
  cl->xw = (double*)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1) * dim);
  cl->fl = (double*)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1) * dim);
  cl->cell = (int*)malloc(sizeof(int) * (size_t)(np > 0 ? np : 1));
  cl->start = (long long*)calloc((size_t)ncell + 1, sizeof(long long));
  cl->order = (long long*)malloc(sizeof(long long) * (size_t)(np > 0 ? np : 1));
  if (!cl->xw || !cl->fl || !cl->cell || !cl->start || !cl->order) { clist_free(cl); return OR_ERR_OOM; }
  for (long long i = 0; i < np; ++i) {
    double s[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k)
      for (int a = 0; a < dim; ++a) s[k] += x[i * dim + a] * g->hinv[a][k];
    long long lin = 0, stride = 1;
    for (int k = 0; k < dim; ++k) {
      double f = floor(s[k]);
      double sw = s[k] - f; /* in [0,1]; 1.0 only through rounding */
      cl->fl[i * dim + k] = f;
      int c = (int)floor(sw * cl->n[k]);
      if (c >= cl->n[k]) c = cl->n[k] - 1;
      if (c < 0) c = 0;
      lin += (long long)c * stride;
      stride *= cl->n[k];
      s[k] = sw;
    }
    for (int a = 0; a < dim; ++a) {
      double v = 0;
      for (int k = 0; k < dim; ++k) v += s[k] * g->h[k][a];
      cl->xw[i * dim + a] = v;
    }
    cl->cell[i] = (int)lin;
    cl->start[lin + 1]++;
  }
  for (long long c = 0; c < ncell; ++c) cl->start[c + 1] += cl->start[c];
  long long* fill = (long long*)malloc(sizeof(long long) * (size_t)(ncell > 0 ? ncell : 1));
  if (!fill) { clist_free(cl); return OR_ERR_OOM; }
  memcpy(fill, cl->start, sizeof(long long) * (size_t)ncell);
  for (long long i = 0; i < np; ++i) cl->order[fill[cl->cell[i]]++] = i;
  free(fill);
  return OR_OK;
}

/* Accumulators for one run over the pair-images. */
typedef struct {
  int dim;
  double rc, band, rmax;
  int nbins;
  long long count, band_in, band_out;
  double suminvr, energy;
  double* forces;   /* n*dim or NULL */
  double virial[9];
  double dedh[9];
  long long* hist_core;  /* nbins or NULL */
  long long* hist_maybe; /* nbins or NULL */
} acc;

/* shifted-force pair energy and its derivative */
static double u_sf(double r, double rc) { return 1.0 / r - 1.0 / rc + (r - rc) / (rc * rc); }
static double du_sf(double r, double rc) { return -1.0 / (r * r) + 1.0 / (rc * rc); }

/* Histogram range: bins of width rmax/nbins over [0, top), top = min(rc, rmax).
 * bin_of returns the bin of a distance, or -1 when it is not below top. */
static double hist_top(const acc* A) { return A->rmax < A->rc ? A->rmax : A->rc; }
static long long bin_of(double r, const acc* A) {
  if (!(r < hist_top(A))) return -1;
  if (r < 0) r = 0;
  long long k = (long long)floor(r * A->nbins / A->rmax);
  if (k >= A->nbins) k = A->nbins - 1;
  return k;
}
/* last bin that holds distances just below top */
static long long last_bin(const acc* A) {
  long long k = (long long)ceil(hist_top(A) * A->nbins / A->rmax) - 1;
  if (k >= A->nbins) k = A->nbins - 1;
  if (k < 0) k = 0;
  return k;
}

/* One pair-image (i, j, t) with displacement rv = x_j - x_i + t.H (raw
 * positions) and length r. Called for every pair-image with r < rc(1+4 band). */
static void visit(acc* A, long long i, long long j, const double* rv, double r, const double* t) {
  const int dim = A->dim;
  const double rc = A->rc, delta = A->band * rc;
  if (r < rc) {
    if (r >= rc - delta) A->band_in++;
  } else {
    if (r < rc + delta) A->band_out++;
  }
  if (A->nbins > 0 && A->hist_core) {
    /* bins reachable by the distance moved by at most delta either way */
    long long lo = bin_of(r - delta, A), hi = bin_of(r + delta, A);
    if (lo >= 0) {
      if (hi == lo) {
        A->hist_core[lo]++;
      } else {
        long long b = hi >= 0 ? hi : last_bin(A);
        for (long long k = lo; k <= b; ++k) A->hist_maybe[k]++;
      }
    }
  }
  if (!(r < rc)) return;
  A->count++;
  A->suminvr += 1.0 / r;
  A->energy += u_sf(r, rc);
  double up = du_sf(r, rc);
  if (A->forces) {
    for (int a = 0; a < dim; ++a) {
      double g = up * rv[a] / r; /* force on i: -dE/dx_i = u'(r) rv/r */
      A->forces[i * dim + a] += g;
      A->forces[j * dim + a] -= g;
    }
  }
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b) {
      A->virial[a * dim + b] += -up * rv[a] * rv[b] / r;
      A->dedh[a * dim + b] += up * rv[b] / r * t[a];
    }
}

static void acc_init(acc* A, int dim, double rc, double band, int nbins, double rmax, long long n,
                     double* forces, long long* hist_core, long long* hist_maybe) {
  memset(A, 0, sizeof(*A));
  A->dim = dim; A->rc = rc; A->band = band; A->nbins = nbins; A->rmax = rmax > 0 ? rmax : rc;
  A->forces = forces; A->hist_core = hist_core; A->hist_maybe = hist_maybe;
  if (forces) memset(forces, 0, sizeof(double) * (size_t)n * dim);
  if (hist_core) memset(hist_core, 0, sizeof(long long) * (size_t)nbins);
  if (hist_maybe) memset(hist_maybe, 0, sizeof(long long) * (size_t)nbins);
}

static void acc_out(const acc* A, long long* counts, double* sums, double* virial, double* dedh) {
  const int dd = A->dim * A->dim;
  if (counts) { counts[0] = A->count; counts[1] = A->band_in; counts[2] = A->band_out; }
  if (sums) { sums[0] = A->suminvr; sums[1] = A->energy; }
  if (virial) memcpy(virial, A->virial, sizeof(double) * dd);
  if (dedh) memcpy(dedh, A->dedh, sizeof(double) * dd);
}

/* Enumerate the pair-images (i, j, T) with i in [i_lo, i_hi), i < j and
 * |r| < rc_enum, following steps 1-4 of the header, and hand each one to
 * visit() (or to the pair-list collector when pl != NULL). */
typedef struct { long long i, j; double r; } pl_entry;
typedef struct { pl_entry* e; long long n, cap; int overflow; } pl_buf;

/* Sink of or_images / or_cross_images: every accepted pair-image with its
 * displacement vector (the mapped function of Code 2 receives the two
 * positions under the image, i.e. this vector). */
typedef struct {
  long long *i, *j;
  double* rv;   /* cap * dim */
  double* r;
  long long n, cap;
  int dim;
} img_buf;

static void img_put(img_buf* b, long long i, long long j, const double* rv, double r) {
  if (b->n < b->cap) {
    b->i[b->n] = i;
    b->j[b->n] = j;
    for (int a = 0; a < b->dim; ++a) b->rv[b->n * b->dim + a] = rv[a];
    b->r[b->n] = r;
  }
  b->n++;
}

static int enumerate(const geom* g, long long np, const double* x, double rc, double band,
                     long long i_lo, long long i_hi, acc* A, pl_buf* pl, img_buf* ib) {
  const int dim = g->dim;
  const double rc_enum = rc * (1.0 + 4.0 * band);
  clist cl;
  int err = clist_build(&cl, g, np, x, rc_enum);
  if (err) return err;
  if (i_lo < 0) i_lo = 0;
  if (i_hi > np) i_hi = np;
  int span[3] = {1, 1, 1};
  for (int k = 0; k < dim; ++k) span[k] = 2 * cl.m[k] + 1;
  for (long long i = i_lo; i < i_hi; ++i) {
    int ci[3] = {0, 0, 0};
    long long lin = cl.cell[i];
    for (int k = 0; k < dim; ++k) { ci[k] = (int)(lin % cl.n[k]); lin /= cl.n[k]; }
    const double* xi = cl.xw + i * dim;
    for (int oz = 0; oz < (dim == 3 ? span[2] : 1); ++oz)
      for (int oy = 0; oy < span[1]; ++oy)
        for (int ox = 0; ox < span[0]; ++ox) {
          int o[3] = {ox - cl.m[0], oy - cl.m[1], dim == 3 ? oz - cl.m[2] : 0};
          long long T[3] = {0, 0, 0}, cj = 0, stride = 1;
          for (int k = 0; k < dim; ++k) {
            long long u = (long long)ci[k] + o[k];
            T[k] = floordiv_ll(u, cl.n[k]);
            cj += (u - T[k] * cl.n[k]) * stride;
            stride *= cl.n[k];
          }
          double shift[3] = {0, 0, 0};
          for (int a = 0; a < dim; ++a)
            for (int k = 0; k < dim; ++k) shift[a] += (double)T[k] * g->h[k][a];
          for (long long q = cl.start[cj]; q < cl.start[cj + 1]; ++q) {
            long long j = cl.order[q];
            if (j <= i) continue;
            const double* xj = cl.xw + j * dim;
            double rv[3] = {0, 0, 0}, r2 = 0;
            for (int a = 0; a < dim; ++a) {
              rv[a] = xj[a] + shift[a] - xi[a];
              r2 += rv[a] * rv[a];
            }
            if (!(r2 < rc_enum * rc_enum)) continue;
            double r = sqrt(r2);
            /* integer image relative to the raw (unwrapped) input positions */
            double t[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k) t[k] = (double)T[k] - cl.fl[j * dim + k] + cl.fl[i * dim + k];
            if (ib) {
              img_put(ib, i, j, rv, r);
            } else if (pl) {
              if (pl->n == pl->cap) { pl->overflow = 1; continue; }
              pl->e[pl->n].i = i; pl->e[pl->n].j = j; pl->e[pl->n].r = r; pl->n++;
            } else {
              visit(A, i, j, rv, r, t);
            }
          }
        }
  }
  clist_free(&cl);
  return OR_OK;
}

/* ------------------------------------------------------------------ API -- */

/* Grid the oracle would use (cells >= rc wide) and the widths; for tests. */
int or_geom_info(int dim, const double* h, double rc, int lcell, double* w_out, int* n_out, int* m_out) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0) || lcell < 1) return OR_ERR_ARG;
  for (int k = 0; k < dim; ++k) {
    double nk = floor(g.w[k] * lcell / rc);
    if (nk < 1) nk = 1;
    w_out[k] = g.w[k];
    n_out[k] = (int)nk;
    m_out[k] = (int)ceil(rc * n_out[k] / g.w[k]);
  }
  return OR_OK;
}

/* All reductions over P for i in [i_lo, i_hi) (pass 0, n for all pairs).
 * counts[3]: pair count (r < rc), band pairs inside, band pairs outside.
 * sums[2]: sum 1/r, shifted-force energy.
 * forces (n*dim), virial (dim*dim), dedh (dim*dim): optional, may be NULL.
 * hist_core / hist_maybe (nbins): optional; bins over [0, rmax). */
int or_map(int dim, long long n, const double* x, const double* h, double rc, double band,
           long long i_lo, long long i_hi, int nbins, double rmax,
           long long* counts, double* sums, double* forces, double* virial, double* dedh,
           long long* hist_core, long long* hist_maybe) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0) || n < 0 || band < 0) return OR_ERR_ARG;
  for (int k = 0; k < dim; ++k)
    if (!(rc < g.w[k])) return OR_ERR_ARG; /* a particle would see its own image */
  acc A;
  acc_init(&A, dim, rc, band, nbins, rmax, n, forces, hist_core, hist_maybe);
  err = enumerate(&g, n, x, rc, band, i_lo, i_hi, &A, NULL, NULL);
  if (err) return err;
  acc_out(&A, counts, sums, virial, dedh);
  return OR_OK;
}

static int cmp_pair(const void* a, const void* b) {
  const pl_entry* p = (const pl_entry*)a;
  const pl_entry* q = (const pl_entry*)b;
  if (p->i != q->i) return p->i < q->i ? -1 : 1;
  if (p->j != q->j) return p->j < q->j ? -1 : 1;
  return (p->r < q->r) ? -1 : (p->r > q->r);
}

static int pairlist_finish(pl_buf* pl, double rc, double band, long long cap,
                           long long* pi, long long* pj, double* pd, signed char* pband, long long* npairs) {
  if (pl->overflow) { free(pl->e); return OR_ERR_CAPACITY; }
  qsort(pl->e, (size_t)pl->n, sizeof(pl_entry), cmp_pair);
  for (long long q = 1; q < pl->n; ++q)
    if (pl->e[q].i == pl->e[q - 1].i && pl->e[q].j == pl->e[q - 1].j) { free(pl->e); return OR_ERR_IMAGES; }
  *npairs = pl->n;
  if (pl->n > cap) { free(pl->e); return OR_ERR_CAPACITY; }
  const double delta = band * rc;
  for (long long q = 0; q < pl->n; ++q) {
    pi[q] = pl->e[q].i; pj[q] = pl->e[q].j; pd[q] = pl->e[q].r;
    pband[q] = (fabs(pl->e[q].r - rc) <= delta) ? 1 : 0;
  }
  free(pl->e);
  return OR_OK;
}

/* Neighbour list (Sec. 4.1): all i<j with r < rc(1+4 band), sorted by (i, j),
 * each flagged band=1 when |r - rc| <= band*rc (those with r >= rc are only
 * present so that a test can accept an FP32 inclusion). Requires that no pair
 * has two images inside the cutoff. */
int or_pairlist(int dim, long long n, const double* x, const double* h, double rc, double band,
                long long cap, long long* pi, long long* pj, double* pd, signed char* pband, long long* npairs) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0) || n < 0 || band < 0) return OR_ERR_ARG;
  pl_buf pl;
  pl.cap = cap + 1; pl.n = 0; pl.overflow = 0;
  pl.e = (pl_entry*)malloc(sizeof(pl_entry) * (size_t)pl.cap);
  if (!pl.e) return OR_ERR_OOM;
  err = enumerate(&g, n, x, rc, band, 0, n, NULL, &pl, NULL);
  if (err) { free(pl.e); return err; }
  return pairlist_finish(&pl, rc, band, cap, pi, pj, pd, pband, npairs);
}

/* Force (-dE/dx) and per-particle energy (half of its pair energies) of the
 * particles idx[0..k), each computed on its own over all its pair-images. */
int or_particles(int dim, long long n, const double* x, const double* h, double rc,
                 const long long* idx, long long k, double* f_out, double* e_out) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0)) return OR_ERR_ARG;
  for (int a = 0; a < dim; ++a)
    if (!(rc < g.w[a])) return OR_ERR_ARG;
  clist cl;
  err = clist_build(&cl, &g, n, x, rc);
  if (err) return err;
  int span[3] = {1, 1, 1};
  for (int a = 0; a < dim; ++a) span[a] = 2 * cl.m[a] + 1;
  for (long long q = 0; q < k; ++q) {
    long long i = idx[q];
    double f[3] = {0, 0, 0}, e = 0;
    if (i < 0 || i >= n) { clist_free(&cl); return OR_ERR_ARG; }
    int ci[3] = {0, 0, 0};
    long long lin = cl.cell[i];
    for (int a = 0; a < dim; ++a) { ci[a] = (int)(lin % cl.n[a]); lin /= cl.n[a]; }
    const double* xi = cl.xw + i * dim;
    for (int oz = 0; oz < (dim == 3 ? span[2] : 1); ++oz)
      for (int oy = 0; oy < span[1]; ++oy)
        for (int ox = 0; ox < span[0]; ++ox) {
          int o[3] = {ox - cl.m[0], oy - cl.m[1], dim == 3 ? oz - cl.m[2] : 0};
          long long T[3] = {0, 0, 0}, cj = 0, stride = 1;
          for (int a = 0; a < dim; ++a) {
            long long u = (long long)ci[a] + o[a];
            T[a] = floordiv_ll(u, cl.n[a]);
            cj += (u - T[a] * cl.n[a]) * stride;
            stride *= cl.n[a];
          }
          double shift[3] = {0, 0, 0};
          for (int a = 0; a < dim; ++a)
            for (int b = 0; b < dim; ++b) shift[a] += (double)T[b] * g.h[b][a];
          for (long long p = cl.start[cj]; p < cl.start[cj + 1]; ++p) {
            long long j = cl.order[p];
            if (j == i) continue;
            const double* xj = cl.xw + j * dim;
            double rv[3] = {0, 0, 0}, r2 = 0;
            for (int a = 0; a < dim; ++a) { rv[a] = xj[a] + shift[a] - xi[a]; r2 += rv[a] * rv[a]; }
            if (!(r2 < rc * rc)) continue;
            double r = sqrt(r2), up = du_sf(r, rc);
            for (int a = 0; a < dim; ++a) f[a] += up * rv[a] / r;
            e += 0.5 * u_sf(r, rc);
          }
        }
    for (int a = 0; a < dim; ++a) f_out[q * dim + a] = f[a];
    if (e_out) e_out[q] = e;
  }
  clist_free(&cl);
  return OR_OK;
}

/* Neighbours j > a of each query particle a (Sec. 4.1 list restricted to the
 * rows of chosen particles): every j > a with r < rc(1 + 4 band), sorted by
 * j, with its distance and band flag. Row q occupies out[offs[q] ..
 * offs[q+1]); offs has k + 1 entries. Returns OR_ERR_CAPACITY when the rows
 * need more than cap entries (offs[k] then holds the total). */
static int cmp_j(const void* a, const void* b) {
  const pl_entry* p = (const pl_entry*)a;
  const pl_entry* q = (const pl_entry*)b;
  return (p->j > q->j) - (p->j < q->j);
}

int or_neighbors(int dim, long long n, const double* x, const double* h, double rc, double band,
                 const long long* idx, long long k, long long cap, long long* offs, long long* out_j,
                 double* out_d, signed char* out_band) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0) || band < 0) return OR_ERR_ARG;
  const double rce = rc * (1.0 + 4.0 * band), delta = band * rc;
  clist cl;
  err = clist_build(&cl, &g, n, x, rce);
  if (err) return err;
  int span[3] = {1, 1, 1};
  for (int a = 0; a < dim; ++a) span[a] = 2 * cl.m[a] + 1;
  long long used = 0;
  pl_entry* row = (pl_entry*)malloc(sizeof(pl_entry) * (size_t)(n > 0 ? n : 1));
  if (!row) { clist_free(&cl); return OR_ERR_OOM; }
  for (long long q = 0; q < k; ++q) {
    long long i = idx[q], m = 0;
    offs[q] = used;
    if (i < 0 || i >= n) { free(row); clist_free(&cl); return OR_ERR_ARG; }
    int ci[3] = {0, 0, 0};
    long long lin = cl.cell[i];
    for (int a = 0; a < dim; ++a) { ci[a] = (int)(lin % cl.n[a]); lin /= cl.n[a]; }
    const double* xi = cl.xw + i * dim;
    for (int oz = 0; oz < (dim == 3 ? span[2] : 1); ++oz)
      for (int oy = 0; oy < span[1]; ++oy)
        for (int ox = 0; ox < span[0]; ++ox) {
          int o[3] = {ox - cl.m[0], oy - cl.m[1], dim == 3 ? oz - cl.m[2] : 0};
          long long T[3] = {0, 0, 0}, cj = 0, stride = 1;
          for (int a = 0; a < dim; ++a) {
            long long u = (long long)ci[a] + o[a];
            T[a] = floordiv_ll(u, cl.n[a]);
            cj += (u - T[a] * cl.n[a]) * stride;
            stride *= cl.n[a];
          }
          double shift[3] = {0, 0, 0};
          for (int a = 0; a < dim; ++a)
            for (int b = 0; b < dim; ++b) shift[a] += (double)T[b] * g.h[b][a];
          for (long long p = cl.start[cj]; p < cl.start[cj + 1]; ++p) {
            long long j = cl.order[p];
            if (j <= i) continue;
            const double* xj = cl.xw + j * dim;
            double r2 = 0;
            for (int a = 0; a < dim; ++a) {
              double d = xj[a] + shift[a] - xi[a];
              r2 += d * d;
            }
            if (!(r2 < rce * rce)) continue;
            row[m].i = i; row[m].j = j; row[m].r = sqrt(r2); m++;
          }
        }
    qsort(row, (size_t)m, sizeof(pl_entry), cmp_j);
    for (long long t = 0; t < m; ++t) {
      if (used < cap) {
        out_j[used] = row[t].j;
        out_d[used] = row[t].r;
        out_band[used] = fabs(row[t].r - rc) <= delta ? 1 : 0;
      }
      used++;
    }
  }
  offs[k] = used;
  free(row);
  clist_free(&cl);
  return used > cap ? OR_ERR_CAPACITY : OR_OK;
}

/* ---------------------------------------------------------- brute force -- */

static int brute_walk(const geom* g, long long n, const double* x, double rc, double band,
                      acc* A, pl_buf* pl, img_buf* ib) {
  const int dim = g->dim;
  const double rce = rc * (1.0 + 4.0 * band);
  int K[3] = {0, 0, 0};
  for (int k = 0; k < dim; ++k) K[k] = (int)ceil(rce / g->w[k]) + 1;
  double* sw = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * dim);
  double* fl = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * dim);
  if (!sw || !fl) { free(sw); free(fl); return OR_ERR_OOM; }
  /* wrapped fractional coordinates, computed independently of clist_build */
  for (long long i = 0; i < n; ++i)
    for (int k = 0; k < dim; ++k) {
      double s = 0;
      for (int a = 0; a < dim; ++a) s += x[i * dim + a] * g->hinv[a][k];
      fl[i * dim + k] = floor(s);
      sw[i * dim + k] = s - floor(s);
    }
  for (long long i = 0; i < n; ++i)
    for (long long j = i + 1; j < n; ++j)
      for (int tz = (dim == 3 ? -K[2] : 0); tz <= (dim == 3 ? K[2] : 0); ++tz)
        for (int ty = -K[1]; ty <= K[1]; ++ty)
          for (int tx = -K[0]; tx <= K[0]; ++tx) {
            double T[3] = {tx, ty, tz};
            double ds[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k) ds[k] = sw[j * dim + k] - sw[i * dim + k] + T[k];
            double rv[3] = {0, 0, 0}, r2 = 0;
            for (int a = 0; a < dim; ++a) {
              for (int k = 0; k < dim; ++k) rv[a] += ds[k] * g->h[k][a];
              r2 += rv[a] * rv[a];
            }
            if (!(r2 < rce * rce)) continue;
            double r = sqrt(r2);
            double t[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k) t[k] = T[k] - fl[j * dim + k] + fl[i * dim + k];
            if (ib) {
              img_put(ib, i, j, rv, r);
            } else if (pl) {
              if (pl->n == pl->cap) { pl->overflow = 1; continue; }
              pl->e[pl->n].i = i; pl->e[pl->n].j = j; pl->e[pl->n].r = r; pl->n++;
            } else {
              visit(A, i, j, rv, r, t);
            }
          }
  free(sw); free(fl);
  return OR_OK;
}

int or_brute_map(int dim, long long n, const double* x, const double* h, double rc, double band,
                 int nbins, double rmax, long long* counts, double* sums, double* forces,
                 double* virial, double* dedh, long long* hist_core, long long* hist_maybe) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0) || n < 0 || band < 0) return OR_ERR_ARG;
  acc A;
  acc_init(&A, dim, rc, band, nbins, rmax, n, forces, hist_core, hist_maybe);
  err = brute_walk(&g, n, x, rc, band, &A, NULL, NULL);
  if (err) return err;
  acc_out(&A, counts, sums, virial, dedh);
  return OR_OK;
}

int or_brute_pairlist(int dim, long long n, const double* x, const double* h, double rc, double band,
                      long long cap, long long* pi, long long* pj, double* pd, signed char* pband,
                      long long* npairs) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  pl_buf pl;
  pl.cap = cap + 1; pl.n = 0; pl.overflow = 0;
  pl.e = (pl_entry*)malloc(sizeof(pl_entry) * (size_t)pl.cap);
  if (!pl.e) return OR_ERR_OOM;
  err = brute_walk(&g, n, x, rc, band, NULL, &pl, NULL);
  if (err) { free(pl.e); return err; }
  return pairlist_finish(&pl, rc, band, cap, pi, pj, pd, pband, npairs);
}

/* ------------------------------------------------------------ pair-images */

/* Every pair-image (i < j, image t) with r < rc(1 + 4 band), with its
 * displacement rv = x_j - x_i + t.H (dim values each) and distance r, in the
 * order the cell-list enumeration meets them. This is what the mapped
 * function of Code 2 sees; any pair function (Code 5-7, 10) is a sum over it.
 * Returns OR_ERR_CAPACITY with *nimg = the number needed when cap is short. */
int or_images(int dim, long long n, const double* x, const double* h, double rc, double band, long long cap,
              long long* pi, long long* pj, double* rv, double* pr, long long* nimg) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0) || n < 0 || band < 0 || cap < 0) return OR_ERR_ARG;
  img_buf b = {pi, pj, rv, pr, 0, cap, dim};
  err = enumerate(&g, n, x, rc, band, 0, n, NULL, NULL, &b);
  if (err) return err;
  *nimg = b.n;
  return b.n > cap ? OR_ERR_CAPACITY : OR_OK;
}

/* The same set by brute force over all i < j and image vectors (n <= ~300). */
int or_brute_images(int dim, long long n, const double* x, const double* h, double rc, double band,
                    long long cap, long long* pi, long long* pj, double* rv, double* pr, long long* nimg) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0) || n < 0 || band < 0 || cap < 0) return OR_ERR_ARG;
  img_buf b = {pi, pj, rv, pr, 0, cap, dim};
  err = brute_walk(&g, n, x, rc, band, NULL, NULL, &b);
  if (err) return err;
  *nimg = b.n;
  return b.n > cap ? OR_ERR_CAPACITY : OR_OK;
}

/* Cross pair-images between two sets (Code 8: a cell list of x and y):
 *   { (a, b, t) : a < na, b < nb, |y_b - x_a + t.H| < rc },
 * every a paired with every b (no a < b rule), displacement rv = y_b - x_a + t.H.
 * A cell list of x on the oracle grid; every b visits the full stencil around
 * its cell. */
int or_cross_images(int dim, long long na, const double* xa, long long nb, const double* yb, const double* h,
                    double rc, double band, long long cap, long long* pa, long long* pb, double* rv, double* pr,
                    long long* nimg) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0) || na < 0 || nb < 0 || band < 0 || cap < 0) return OR_ERR_ARG;
  const double rce = rc * (1.0 + 4.0 * band);
  clist cl;
  err = clist_build(&cl, &g, na, xa, rce);
  if (err) return err;
  img_buf buf = {pa, pb, rv, pr, 0, cap, dim};
  int span[3] = {1, 1, 1};
  for (int k = 0; k < dim; ++k) span[k] = 2 * cl.m[k] + 1;
  for (long long b = 0; b < nb; ++b) {
    /* wrap y_b and find its cell on x's grid */
    double s[3] = {0, 0, 0}, yw[3] = {0, 0, 0};
    int cb[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
      for (int a = 0; a < dim; ++a) s[k] += yb[b * dim + a] * g.hinv[a][k];
      s[k] -= floor(s[k]);
      int c = (int)floor(s[k] * cl.n[k]);
      if (c >= cl.n[k]) c = cl.n[k] - 1;
      if (c < 0) c = 0;
      cb[k] = c;
    }
    for (int a = 0; a < dim; ++a)
      for (int k = 0; k < dim; ++k) yw[a] += s[k] * g.h[k][a];
    for (int oz = 0; oz < (dim == 3 ? span[2] : 1); ++oz)
      for (int oy = 0; oy < span[1]; ++oy)
        for (int ox = 0; ox < span[0]; ++ox) {
          int o[3] = {ox - cl.m[0], oy - cl.m[1], dim == 3 ? oz - cl.m[2] : 0};
          long long T[3] = {0, 0, 0}, cj = 0, stride = 1;
          for (int k = 0; k < dim; ++k) {
            long long u = (long long)cb[k] + o[k];
            T[k] = floordiv_ll(u, cl.n[k]);
            cj += (u - T[k] * cl.n[k]) * stride;
            stride *= cl.n[k];
          }
          double shift[3] = {0, 0, 0};
          for (int a = 0; a < dim; ++a)
            for (int k = 0; k < dim; ++k) shift[a] += (double)T[k] * g.h[k][a];
          for (long long q = cl.start[cj]; q < cl.start[cj + 1]; ++q) {
            long long ia = cl.order[q];
            double d[3] = {0, 0, 0}, r2 = 0;
            for (int a = 0; a < dim; ++a) {
              d[a] = yw[a] - (cl.xw[ia * dim + a] + shift[a]);
              r2 += d[a] * d[a];
            }
            if (!(r2 < rce * rce)) continue;
            img_put(&buf, ia, b, d, sqrt(r2));
          }
        }
  }
  clist_free(&cl);
  *nimg = buf.n;
  return buf.n > cap ? OR_ERR_CAPACITY : OR_OK;
}

/* The same set by brute force over all (a, b) and image vectors. */
int or_brute_cross_images(int dim, long long na, const double* xa, long long nb, const double* yb,
                          const double* h, double rc, double band, long long cap, long long* pa, long long* pb,
                          double* rv, double* pr, long long* nimg) {
  geom g;
  int err = geom_init(&g, dim, h);
  if (err) return err;
  if (!(rc > 0) || na < 0 || nb < 0 || band < 0 || cap < 0) return OR_ERR_ARG;
  const double rce = rc * (1.0 + 4.0 * band);
  int K[3] = {0, 0, 0};
  for (int k = 0; k < dim; ++k) K[k] = (int)ceil(rce / g.w[k]) + 1;
  img_buf buf = {pa, pb, rv, pr, 0, cap, dim};
  for (long long ia = 0; ia < na; ++ia)
    for (long long b = 0; b < nb; ++b) {
      double sa[3] = {0, 0, 0}, sb[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) {
        for (int a = 0; a < dim; ++a) {
          sa[k] += xa[ia * dim + a] * g.hinv[a][k];
          sb[k] += yb[b * dim + a] * g.hinv[a][k];
        }
        sa[k] -= floor(sa[k]);
        sb[k] -= floor(sb[k]);
      }
      for (int tz = (dim == 3 ? -K[2] : 0); tz <= (dim == 3 ? K[2] : 0); ++tz)
        for (int ty = -K[1]; ty <= K[1]; ++ty)
          for (int tx = -K[0]; tx <= K[0]; ++tx) {
            double T[3] = {tx, ty, tz};
            double d[3] = {0, 0, 0}, r2 = 0;
            for (int a = 0; a < dim; ++a) {
              for (int k = 0; k < dim; ++k) d[a] += (sb[k] - sa[k] + T[k]) * g.h[k][a];
              r2 += d[a] * d[a];
            }
            if (!(r2 < rce * rce)) continue;
            img_put(&buf, ia, b, d, sqrt(r2));
          }
    }
  *nimg = buf.n;
  return buf.n > cap ? OR_ERR_CAPACITY : OR_OK;
}
