/*
 * Seeded synthetic graph generators.
 *
 * These stand in for the paper's datasets (Section 4, Table 1: mesh-like
 * finite-element graphs, power grids, heavy-tailed networks and a binary
 * tree), which are not available here.  Every generator returns an
 * undirected edge list (src[e], dst[e]) over nodes 0..n-1 and holds none of
 * the layout method's arithmetic: no distances, weights or positions of the
 * method are computed here (the edge lengths of gen_rgg_lengths are input
 * data, the Euclidean lengths of the generated points' edges).  Both the CUDA path and the CPU oracle consume
 * these edge lists, so this file is the only code the two sides share.
 *
 * Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), used here as a
 * plain sequential stream.
 *
 * Memory: every function that produces an edge list allocates it with
 * malloc and returns it through the out pointers; release with gen_free.
 * Return value 0 on success, negative on bad arguments or allocation failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } sm64;

static uint64_t sm64_next(sm64 *r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform integer in [0, n) by the multiply-shift map on the top 32 bits */
static uint32_t sm64_below(sm64 *r, uint32_t n) {
  return (uint32_t)(((sm64_next(r) >> 32) * (uint64_t)n) >> 32);
}

/* uniform double in [0, 1) from the top 53 bits */
static double sm64_unit(sm64 *r) {
  return (double)(sm64_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

void gen_free(void *p) { free(p); }

static int alloc_edges(int64_t m, int32_t **src, int32_t **dst) {
  *src = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  *dst = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!*src || !*dst) { free(*src); free(*dst); *src = *dst = NULL; return -2; }
  return 0;
}

/* rows x cols 4-neighbour grid, node id r*cols + c, unit edges */
int gen_grid(int32_t rows, int32_t cols, int32_t *n_out, int64_t *m_out,
             int32_t **src, int32_t **dst) {
  if (rows < 1 || cols < 1 || (int64_t)rows * cols > 0x7fffffff) return -1;
  int64_t m = (int64_t)rows * (cols - 1) + (int64_t)(rows - 1) * cols;
  if (alloc_edges(m, src, dst)) return -2;
  int64_t e = 0;
  for (int32_t r = 0; r < rows; ++r)
    for (int32_t c = 0; c < cols; ++c) {
      int32_t v = r * cols + c;
      if (c + 1 < cols) { (*src)[e] = v; (*dst)[e] = v + 1; ++e; }
      if (r + 1 < rows) { (*src)[e] = v; (*dst)[e] = v + cols; ++e; }
    }
  *n_out = rows * cols; *m_out = m;
  return 0;
}

/* path 0-1-...-(n-1) */
int gen_path(int32_t n, int32_t *n_out, int64_t *m_out, int32_t **src, int32_t **dst) {
  if (n < 1) return -1;
  if (alloc_edges(n - 1, src, dst)) return -2;
  for (int32_t i = 0; i + 1 < n; ++i) { (*src)[i] = i; (*dst)[i] = i + 1; }
  *n_out = n; *m_out = n - 1;
  return 0;
}

/* complete binary tree of the given depth: n = 2^(depth+1) - 1, children 2i+1, 2i+2 */
int gen_complete_btree(int32_t depth, int32_t *n_out, int64_t *m_out,
                       int32_t **src, int32_t **dst) {
  if (depth < 0 || depth > 29) return -1;
  int32_t n = (int32_t)((1u << (depth + 1)) - 1);
  if (alloc_edges(n - 1, src, dst)) return -2;
  for (int32_t i = 1; i < n; ++i) { (*src)[i - 1] = (i - 1) / 2; (*dst)[i - 1] = i; }
  *n_out = n; *m_out = n - 1;
  return 0;
}

/* random binary tree: node i (i >= 1) attaches to a uniformly chosen earlier
 * node that still has fewer than two children */
int gen_random_btree(int32_t n, uint64_t seed, int32_t *n_out, int64_t *m_out,
                     int32_t **src, int32_t **dst) {
  if (n < 1) return -1;
  if (alloc_edges(n - 1, src, dst)) return -2;
  int32_t *open = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  uint8_t *kids = (uint8_t *)calloc((size_t)n, 1);
  if (!open || !kids) { free(open); free(kids); gen_free(*src); gen_free(*dst); return -2; }
  sm64 r = {seed};
  int32_t nopen = 1; open[0] = 0;
  for (int32_t i = 1; i < n; ++i) {
    uint32_t j = sm64_below(&r, (uint32_t)nopen);
    int32_t p = open[j];
    (*src)[i - 1] = p; (*dst)[i - 1] = i;
    if (++kids[p] == 2) open[j] = open[--nopen];
    open[nopen++] = i;
  }
  free(open); free(kids);
  *n_out = n; *m_out = n - 1;
  return 0;
}

/* ---- largest connected component (input preparation: the paper keeps only
 * the largest component of disconnected inputs, Section 4 "Data") ---- */
static int32_t uf_find(int32_t *par, int32_t x) {
  while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
  return x;
}

/* keeps the largest component (ties: the one holding the smallest node id),
 * relabels its nodes in increasing original id, rewrites the edge list in place */
static int keep_lcc(int32_t n, int64_t *m, int32_t *src, int32_t *dst, float *len, int32_t *n_out) {
  int32_t *par = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *size = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  if (!par || !size) { free(par); free(size); return -2; }
  for (int32_t i = 0; i < n; ++i) par[i] = i;
  for (int64_t e = 0; e < *m; ++e) {
    int32_t a = uf_find(par, src[e]), b = uf_find(par, dst[e]);
    if (a != b) { if (a < b) par[b] = a; else par[a] = b; }
  }
  int32_t best = -1, bestsz = 0;
  for (int32_t i = 0; i < n; ++i) ++size[uf_find(par, i)];
  for (int32_t i = 0; i < n; ++i)
    if (par[i] == i && size[i] > bestsz) { bestsz = size[i]; best = i; }
  int32_t *lab = size; /* reuse */
  int32_t nn = 0;
  for (int32_t i = 0; i < n; ++i) lab[i] = (uf_find(par, i) == best) ? nn++ : -1;
  int64_t mm = 0;
  for (int64_t e = 0; e < *m; ++e) {
    if (lab[src[e]] >= 0) {
      src[mm] = lab[src[e]];
      dst[mm] = lab[dst[e]];
      if (len) len[mm] = len[e];
      ++mm;
    }
  }
  free(par); free(size);
  *m = mm; *n_out = nn;
  return 0;
}

/* random geometric graph: n points uniform in the unit square, an edge for
 * every pair at Euclidean distance < radius (radius = sqrt(mean_deg/(pi n))
 * when radius <= 0), built with a bucket grid; the largest component is kept. */
static int rgg_impl(int32_t n, double mean_deg, double radius, uint64_t seed,
                    int32_t *n_out, int64_t *m_out, int32_t **src, int32_t **dst, float **len) {
  if (n < 2) return -1;
  if (radius <= 0) radius = sqrt(mean_deg / (3.14159265358979323846 * (double)n));
  double *px = (double *)malloc((size_t)n * sizeof(double));
  double *py = (double *)malloc((size_t)n * sizeof(double));
  int32_t g = (int32_t)floor(1.0 / radius);
  if (g < 1) g = 1;
  if ((int64_t)g * g > 64LL * n) g = (int32_t)sqrt(64.0 * n);
  int64_t ncell = (int64_t)g * g;
  int32_t *head = (int32_t *)malloc((size_t)(ncell + 1) * sizeof(int32_t));
  int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *cellof = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!px || !py || !head || !order || !cellof) goto fail;
  sm64 r = {seed};
  for (int32_t i = 0; i < n; ++i) { px[i] = sm64_unit(&r); py[i] = sm64_unit(&r); }
  memset(head, 0, (size_t)(ncell + 1) * sizeof(int32_t));
  for (int32_t i = 0; i < n; ++i) {
    int32_t cx = (int32_t)(px[i] * g), cy = (int32_t)(py[i] * g);
    if (cx >= g) cx = g - 1;
    if (cy >= g) cy = g - 1;
    cellof[i] = cy * g + cx;
    ++head[cellof[i] + 1];
  }
  for (int64_t c = 0; c < ncell; ++c) head[c + 1] += head[c];
  {
    int32_t *fill = (int32_t *)malloc((size_t)ncell * sizeof(int32_t));
    if (!fill) goto fail;
    memcpy(fill, head, (size_t)ncell * sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) order[fill[cellof[i]]++] = i; /* ascending i per cell */
    free(fill);
  }
  /* two passes: count, then fill */
  double r2 = radius * radius;
  int64_t cap = 0;
  for (int pass = 0; pass < 2; ++pass) {
    int64_t e = 0;
    for (int32_t i = 0; i < n; ++i) {
      int32_t cx = cellof[i] % g, cy = cellof[i] / g;
      for (int32_t dy = -1; dy <= 1; ++dy)
        for (int32_t dx = -1; dx <= 1; ++dx) {
          int32_t x = cx + dx, y = cy + dy;
          if (x < 0 || y < 0 || x >= g || y >= g) continue;
          int32_t c = y * g + x;
          for (int32_t t = head[c]; t < head[c + 1]; ++t) {
            int32_t j = order[t];
            if (j <= i) continue;
            double ddx = px[i] - px[j], ddy = py[i] - py[j];
            if (ddx * ddx + ddy * ddy < r2) {
              if (pass == 1) {
                (*src)[e] = i;
                (*dst)[e] = j;
                if (len) (*len)[e] = (float)(sqrt(ddx * ddx + ddy * ddy) / radius);
              }
              ++e;
            }
          }
        }
    }
    if (pass == 0) {
      cap = e;
      if (alloc_edges(cap, src, dst)) goto fail;
      if (len) {
        *len = (float *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(float));
        if (!*len) { gen_free(*src); gen_free(*dst); goto fail; }
      }
    }
  }
  free(px); free(py); free(head); free(order); free(cellof);
  px = py = NULL;
  {
    int64_t m = cap;
    if (keep_lcc(n, &m, *src, *dst, len ? *len : NULL, n_out)) {
      gen_free(*src);
      gen_free(*dst);
      if (len) gen_free(*len);
      return -2;
    }
    *m_out = m;
  }
  return 0;
fail:
  free(px); free(py); free(head); free(order); free(cellof);
  return -2;
}

int gen_rgg(int32_t n, double mean_deg, double radius, uint64_t seed,
            int32_t *n_out, int64_t *m_out, int32_t **src, int32_t **dst) {
  return rgg_impl(n, mean_deg, radius, seed, n_out, m_out, src, dst, NULL);
}

/* the same graph with edge lengths: the Euclidean length of each edge divided
 * by the radius, as float (in (0, 1); a geometric stand-in for the paper's
 * weighted inputs); the lengths are released with gen_free */
int gen_rgg_lengths(int32_t n, double mean_deg, double radius, uint64_t seed,
                    int32_t *n_out, int64_t *m_out, int32_t **src, int32_t **dst, float **len) {
  return rgg_impl(n, mean_deg, radius, seed, n_out, m_out, src, dst, len);
}

/* Barabasi-Albert preferential attachment: a (m0)-clique seed with
 * m0 = attach + 1 nodes, then every new node joins `attach` distinct earlier
 * nodes, each drawn with probability proportional to its degree (uniform
 * draws from the list of all edge endpoints so far, repeated until distinct). */
int gen_ba(int32_t n, int32_t attach, uint64_t seed, int32_t *n_out, int64_t *m_out,
           int32_t **src, int32_t **dst) {
  int32_t m0 = attach + 1;
  if (attach < 1 || attach > 64 || n < m0) return -1;
  int64_t m = (int64_t)m0 * (m0 - 1) / 2 + (int64_t)attach * (n - m0);
  if (alloc_edges(m, src, dst)) return -2;
  int32_t *ends = (int32_t *)malloc((size_t)(2 * m) * sizeof(int32_t));
  if (!ends) { gen_free(*src); gen_free(*dst); return -2; }
  int64_t e = 0, ne = 0;
  for (int32_t i = 0; i < m0; ++i)
    for (int32_t j = i + 1; j < m0; ++j) {
      (*src)[e] = i; (*dst)[e] = j; ++e;
      ends[ne++] = i; ends[ne++] = j;
    }
  sm64 r = {seed};
  int32_t pick[64];
  for (int32_t v = m0; v < n; ++v) {
    int32_t got = 0;
    while (got < attach) {
      int32_t u = ends[(int64_t)(((sm64_next(&r) >> 11) * (double)ne) / 9007199254740992.0)];
      int dup = 0;
      for (int32_t t = 0; t < got; ++t) dup |= (pick[t] == u);
      if (!dup) pick[got++] = u;
    }
    for (int32_t t = 0; t < attach; ++t) {
      (*src)[e] = pick[t]; (*dst)[e] = v; ++e;
      ends[ne++] = pick[t]; ends[ne++] = v;
    }
  }
  free(ends);
  *n_out = n; *m_out = m;
  return 0;
}

/* the subgraph induced by nodes 0..n_keep-1 (edges with both ends below n_keep) */
int gen_induced_prefix(int32_t n_keep, int64_t m, const int32_t *src, const int32_t *dst,
                       int64_t *m_out, int32_t **osrc, int32_t **odst) {
  int64_t c = 0;
  for (int64_t e = 0; e < m; ++e) c += (src[e] < n_keep && dst[e] < n_keep);
  if (alloc_edges(c, osrc, odst)) return -2;
  c = 0;
  for (int64_t e = 0; e < m; ++e)
    if (src[e] < n_keep && dst[e] < n_keep) { (*osrc)[c] = src[e]; (*odst)[c] = dst[e]; ++c; }
  *m_out = c;
  return 0;
}
