/*
 * clustered.c -- seeded generator of a clustered 3D particle set in a cubic
 * periodic box: Gaussian clusters plus a uniform background, with a minimum
 * separation between any two particles enforced by rejection.
 *
 * Input generation only: no part of the cell-list method lives here.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna) seeded through splitmix64;
 * normal deviates by the Box-Muller transform.
 *
 * Cluster sizes follow a power law p(s) ~ s^-2 truncated to [s_min, s_max]
 * (inverse-CDF sampling), rescaled so they sum exactly to the clustered count
 * (largest-remainder rounding). A clustered point that fails max_tries
 * placements is redrawn in the uniform background instead.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t next_u64(rng_t* r) {
  uint64_t* s = r->s;
  uint64_t result = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl(s[3], 45);
  return result;
}
static double u01(rng_t* r) { return (double)(next_u64(r) >> 11) * (1.0 / 9007199254740992.0); }
static double gauss(rng_t* r) {
  double a = u01(r), b = u01(r);
  if (a < 1e-300) a = 1e-300;
  return sqrt(-2.0 * log(a)) * cos(6.283185307179586 * b);
}

typedef struct {
  double L, cell;
  int G;
  int32_t* head;
  int32_t* next;
  double* x;
  double min_sep2;
} grid_t;

static double wrap(double v, double L) {
  v -= L * floor(v / L);
  if (v >= L) v -= L;
  if (v < 0) v = 0;
  return v;
}

static int gidx(const grid_t* g, double v) {
  int c = (int)(v / g->cell);
  if (c >= g->G) c = g->G - 1;
  if (c < 0) c = 0;
  return c;
}

/* 1 when p keeps at least min_sep from every accepted point (periodic). */
static int free_at(const grid_t* g, const double* p) {
  int c[3] = {gidx(g, p[0]), gidx(g, p[1]), gidx(g, p[2])};
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int cx = (c[0] + dx + g->G) % g->G, cy = (c[1] + dy + g->G) % g->G, cz = (c[2] + dz + g->G) % g->G;
        int32_t q = g->head[((int64_t)cz * g->G + cy) * g->G + cx];
        while (q >= 0) {
          double d2 = 0;
          for (int a = 0; a < 3; ++a) {
            double d = g->x[3 * (int64_t)q + a] - p[a];
            d -= g->L * nearbyint(d / g->L);
            d2 += d * d;
          }
          if (d2 < g->min_sep2) return 0;
          q = g->next[q];
        }
      }
  return 1;
}

static void insert(grid_t* g, int32_t id, const double* p) {
  for (int a = 0; a < 3; ++a) g->x[3 * (int64_t)id + a] = p[a];
  int64_t c = ((int64_t)gidx(g, p[2]) * g->G + gidx(g, p[1])) * g->G + gidx(g, p[0]);
  g->next[id] = g->head[c];
  g->head[c] = id;
}

/* stats[0..3]: clustered placed, background placed, clustered redirected to
 * the background, largest cluster size. Returns 0, or -1 on bad arguments,
 * -2 on allocation failure, -3 when the background could not be placed. */
int synth_clustered(long long n, double L, int n_clusters, double sigma, double frac_clustered,
                    double s_min, double s_max, double min_sep, int max_tries, unsigned long long seed,
                    double* x, long long* stats) {
  if (n <= 0 || n >= 2147483647LL || !(L > 0) || n_clusters < 0 || !(s_min > 0) || !(s_max >= s_min) ||
      !(min_sep > 0) || max_tries < 1)
    return -1;
  uint64_t sm = seed;
  rng_t R;
  for (int k = 0; k < 4; ++k) R.s[k] = splitmix64(&sm);

  long long n_cl = (long long)llround(frac_clustered * (double)n);
  if (n_clusters == 0) n_cl = 0;
  long long* size = (long long*)calloc((size_t)(n_clusters > 0 ? n_clusters : 1), sizeof(long long));
  double* raw = (double*)calloc((size_t)(n_clusters > 0 ? n_clusters : 1), sizeof(double));
  double* centre = (double*)calloc((size_t)(n_clusters > 0 ? n_clusters : 1) * 3, sizeof(double));
  if (!size || !raw || !centre) { free(size); free(raw); free(centre); return -2; }
  double tot = 0;
  for (int k = 0; k < n_clusters; ++k) {
    double u = u01(&R);
    raw[k] = 1.0 / (1.0 / s_min - u * (1.0 / s_min - 1.0 / s_max));
    tot += raw[k];
  }
  long long assigned = 0;
  for (int k = 0; k < n_clusters; ++k) {
    raw[k] = raw[k] * (double)n_cl / tot;
    size[k] = (long long)floor(raw[k]);
    raw[k] -= (double)size[k];
    assigned += size[k];
  }
  for (long long left = n_cl - assigned; left > 0; --left) { /* largest remainder */
    int best = 0;
    for (int k = 1; k < n_clusters; ++k)
      if (raw[k] > raw[best]) best = k;
    size[best]++;
    raw[best] = -1.0;
  }
  for (int k = 0; k < n_clusters; ++k)
    for (int a = 0; a < 3; ++a) centre[3 * k + a] = u01(&R) * L;

  grid_t g;
  g.L = L;
  g.G = (int)floor(L / min_sep);
  if (g.G > 400) g.G = 400;
  if (g.G < 1) g.G = 1;
  g.cell = L / g.G;
  g.min_sep2 = min_sep * min_sep;
  g.x = x;
  g.head = (int32_t*)malloc(sizeof(int32_t) * (size_t)g.G * g.G * g.G);
  g.next = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!g.head || !g.next) { free(g.head); free(g.next); free(size); free(raw); free(centre); return -2; }
  memset(g.head, 0xff, sizeof(int32_t) * (size_t)g.G * g.G * g.G);

  int32_t id = 0;
  long long redirected = 0, biggest = 0;
  double p[3];
  for (int k = 0; k < n_clusters; ++k) {
    if (size[k] > biggest) biggest = size[k];
    for (long long q = 0; q < size[k]; ++q) {
      int ok = 0;
      for (int t = 0; t < max_tries && !ok; ++t) {
        for (int a = 0; a < 3; ++a) p[a] = wrap(centre[3 * k + a] + sigma * gauss(&R), L);
        ok = free_at(&g, p);
      }
      if (ok) insert(&g, id++, p);
      else redirected++;
    }
  }
  long long placed_cl = id;
  long long n_bg = n - placed_cl;
  for (long long q = 0; q < n_bg; ++q) {
    int ok = 0;
    for (int t = 0; t < 100000 && !ok; ++t) {
      for (int a = 0; a < 3; ++a) p[a] = wrap(u01(&R) * L, L);
      ok = free_at(&g, p);
    }
    if (!ok) { free(g.head); free(g.next); free(size); free(raw); free(centre); return -3; }
    insert(&g, id++, p);
  }
  stats[0] = placed_cl;
  stats[1] = n_bg;
  stats[2] = redirected;
  stats[3] = biggest;
  free(g.head); free(g.next); free(size); free(raw); free(centre);
  return 0;
}
