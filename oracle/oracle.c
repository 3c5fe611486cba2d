/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, FP64 CPU restatement of the sparse stress model of
 * Ortmann, Klimenta and Brandes, "A Sparse Stress Model" (arxiv 1608.08909).
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * it; the product library never calls it, and it shares no code, header,
 * table or constant with the CUDA path.
 *
 * Every function follows the paper's definitions step by step, in the
 * paper's order, with no blocking, fusion or reordering:
 *   orc_build_csr        simple undirected graph G=(V,E)            (Section 1)
 *   orc_bfs              graph-theoretic distances d_ij, plain queue (Section 1, Eq. 1)
 *   orc_maxmin           "max/min sp" pivot sampling                 (Section 4.1)
 *   orc_kmeans_sp        "k-means sp" pivot sampling                 (Section 4.1)
 *   orc_pivot_dist       d_ip for all pivots, one BFS per pivot      (Algorithm 1, line 2)
 *   orc_regions          regions R(p): closest pivot                 (Section 3)
 *   orc_regions_smallest the same with the paper's smallest-partition ties (Section 3)
 *   orc_histograms       per-pivot distance counts over R(p)         (Section 3, w'_ip)
 *   orc_adapted_weights  w'_ip = s / d_ip^2 by direct count          (Section 3, after Eq. 4)
 *   orc_pivotmds         PivotMDS initial layout                     (Algorithm 1, line 3)
 *   orc_rescale          edge-length rescale                          (Algorithm 1, line 4)
 *   orc_sweep_jacobi     one update of Eq. 4 for all nodes from X^t  (Eq. 4)
 *                        (orc_sweep_jacobi_rows: the same for a node range)
 *   orc_sweep_gs         the same, in place node by node              (Algorithm 1, lines 6-10)
 *   orc_full_sweep       full stress majorization, Jacobi or in place (Section 3, before Eq. 4)
 *   orc_procrustes       Procrustes statistic of two layouts          (Section 4, "Sampling Evaluation")
 *   orc_hull_error       convex-hull error of k-neighbourhoods        (Section 4, Fig. 4)
 *   orc_gabriel(_jaccard) Gabriel graph, neighbourhood similarity    (Section 4, Fig. 3)
 *   orc_full_stress      Eq. 1 over all pairs, or over sampled pairs  (Eq. 1, Section 4)
 *   orc_build_wcsr, orc_sssp, orc_wmaxmin, orc_wpivot_dist, orc_wregions,
 *   orc_wcounts_rows, orc_wpivotmds, orc_wrescale, orc_wsweep_jacobi_rows,
 *   orc_wfull_stress     the same steps on weighted graphs            (Algorithm 1 line 2, Section 3)
 *                        (orc_stress_sums_range: its pair sums for a source range)
 *
 * Readings taken where the paper is silent (each is listed with its reason
 * in the design notes of the repository):
 *   - region ties go to the lowest pivot index (selection order);
 *   - the pivot sum skips p = i (d = 0) and pivots adjacent to i (d = 1);
 *   - s counts j in R(p) with 2*d_jp <= d_ip (exact integer form of d_jp <= d_ip/2);
 *   - a term with ||x_i - x_j|| == 0 contributes w*x_j only;
 *   - the update is applied Jacobi-style (all nodes from X^t) in
 *     orc_sweep_jacobi; orc_sweep_gs keeps the paper's in-place order;
 *   - relative positional change is ||X^{t+1}-X^t||_F / ||X^t||_F;
 *   - the rescale target is the sum of edge lengths, i.e. m for unit edges;
 *   - stress is reported with the optimal scale alpha* = S1/S2.
 *
 * Status codes: 0 ok, -1 bad argument, -2 bad graph (id out of range),
 * -3 disconnected, -4 distance above 65534, -5 out of memory,
 * -8 numerical failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_ARG -1
#define ORC_E_GRAPH -2
#define ORC_E_DISCONNECTED -3
#define ORC_E_DIST_OVERFLOW -4
#define ORC_E_NOMEM -5
#define ORC_E_NUMERIC -8

/* ------------------------------------------------------------------ */
/* graph                                                               */
/* ------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Simple undirected graph from an edge list: self-loops and repeated edges
 * are dropped, both directions are stored, each adjacency list is sorted
 * ascending.  colidx must hold 2*m_in entries; *m_out receives |E|. */
int orc_build_csr(int32_t n, int64_t m_in, const int32_t *src, const int32_t *dst,
                  int32_t *rowptr, int32_t *colidx, int64_t *m_out) {
  if (n < 1 || m_in < 0) return ORC_E_ARG;
  for (int64_t e = 0; e < m_in; ++e)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return ORC_E_GRAPH;
  int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t *tmp = (int32_t *)malloc((size_t)(2 * m_in + 1) * sizeof(int32_t));
  if (!deg || !fill || !tmp) { free(deg); free(fill); free(tmp); return ORC_E_NOMEM; }
  for (int64_t e = 0; e < m_in; ++e)
    if (src[e] != dst[e]) { deg[src[e] + 1]++; deg[dst[e] + 1]++; }
  for (int32_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
  memcpy(fill, deg, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t e = 0; e < m_in; ++e)
    if (src[e] != dst[e]) {
      tmp[fill[src[e]]++] = dst[e];
      tmp[fill[dst[e]]++] = src[e];
    }
  int64_t out = 0;
  rowptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int64_t b = deg[i], e = deg[i + 1];
    qsort(tmp + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
    for (int64_t t = b; t < e; ++t)
      if (t == b || tmp[t] != tmp[t - 1]) colidx[out++] = tmp[t];
    rowptr[i + 1] = (int32_t)out;
  }
  free(deg); free(fill); free(tmp);
  *m_out = out / 2;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* breadth-first search: d_ij for unit edges                           */
/* ------------------------------------------------------------------ */

/* dist[v] = number of edges on a shortest s-v path, -1 if unreachable */
int orc_bfs(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t s, int32_t *dist) {
  if (s < 0 || s >= n) return ORC_E_ARG;
  int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!queue) return ORC_E_NOMEM;
  for (int32_t v = 0; v < n; ++v) dist[v] = -1;
  int32_t head = 0, tail = 0;
  dist[s] = 0;
  queue[tail++] = s;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int32_t t = rowptr[u]; t < rowptr[u + 1]; ++t) {
      int32_t v = colidx[t];
      if (dist[v] < 0) { dist[v] = dist[u] + 1; queue[tail++] = v; }
    }
  }
  free(queue);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* pivot sampling: max/min sp (Section 4.1)                            */
/* ------------------------------------------------------------------ */

/* P = [start]; mind = BFS(start); then k-1 times: p = smallest i with
 * mind[i] = max(mind); append p; mind = min(mind, BFS(p)).  Each BFS is a
 * full, unpruned queue BFS. */
int orc_maxmin(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k,
               int32_t start, int32_t *pivots) {
  if (k < 1 || k > n || start < 0 || start >= n) return ORC_E_ARG;
  int32_t *mind = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *d = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!mind || !d) { free(mind); free(d); return ORC_E_NOMEM; }
  int rc = orc_bfs(n, rowptr, colidx, start, mind);
  for (int32_t v = 0; rc == ORC_OK && v < n; ++v)
    if (mind[v] < 0) rc = ORC_E_DISCONNECTED;
  if (rc == ORC_OK) pivots[0] = start;
  for (int32_t j = 1; rc == ORC_OK && j < k; ++j) {
    int32_t best = 0;
    for (int32_t v = 1; v < n; ++v)
      if (mind[v] > mind[best]) best = v;
    pivots[j] = best;
    rc = orc_bfs(n, rowptr, colidx, best, d);
    for (int32_t v = 0; v < n; ++v)
      if (d[v] < mind[v]) mind[v] = d[v];
  }
  free(mind); free(d);
  return rc;
}

/* ------------------------------------------------------------------ */
/* pivot sampling: k-means sp (Section 4.1)                             */
/* ------------------------------------------------------------------ */

/* k-means over the shortest-path entries of k max/min-sp pivots.  Node i is
 * the point y_i = (d_{0 i}, ..., d_{k-1 i}) of Z^k (column i of the pivot-
 * major table dip); cluster a starts with centre y_{pivots_in[a]}.  Lloyd
 * iterations, at most max_iter (the paper caps its k-means at 50):
 *   assignment: node i joins the cluster a minimising ||y_i - c_a||^2, ties to
 *     the lowest a; with c_a = S_a / n_a (S_a an integer vector, n_a > 0) the
 *     quantity compared is g(i,a) = alpha_a - beta_a * t_ia, where
 *     t_ia = y_i . S_a (an exact integer), beta_a = 2 / n_a and
 *     alpha_a = sum_b (S_ab / n_a)^2 summed in b order, all in FP64 with one
 *     rounding per operation -- ||y_i - c_a||^2 minus the common ||y_i||^2;
 *   stop when an assignment (after the first) changes no node;
 *   update: S_a = sum of the members' y, n_a = member count; a cluster left
 *     empty keeps its previous centre.
 * New pivot of cluster a: the member i minimising ||y_i - c_a||^2, compared
 * exactly as the integer n_a ||y_i||^2 - 2 t_ia, ties to the lowest node id; a
 * cluster empty at the end keeps pivots_in[a].  The exact-integer steps need
 * n * k * max(d)^2 < 2^53 (else ORC_E_ARG).  assign (optional) receives the
 * final cluster of every node, *iters the number of assignment passes. */
int orc_kmeans_sp(int32_t n, int32_t k, const uint16_t *dip, const int32_t *pivots_in, int32_t max_iter,
                  int32_t *pivots_out, int32_t *assign, int32_t *iters) {
  if (n < 1 || k < 1 || max_iter < 1) return ORC_E_ARG;
  int64_t dmax = 0;
  for (int64_t t = 0; t < (int64_t)k * n; ++t)
    if (dip[t] > dmax) dmax = dip[t];
  if ((double)n * (double)k * (double)dmax * (double)dmax >= 9007199254740992.0) return ORC_E_ARG;
  int64_t *S = (int64_t *)malloc((size_t)k * k * sizeof(int64_t));
  int64_t *Snew = (int64_t *)malloc((size_t)k * k * sizeof(int64_t));
  int64_t *cnt = (int64_t *)malloc((size_t)k * sizeof(int64_t));
  int64_t *cnew = (int64_t *)malloc((size_t)k * sizeof(int64_t));
  double *alpha = (double *)malloc((size_t)k * sizeof(double));
  double *beta = (double *)malloc((size_t)k * sizeof(double));
  int32_t *asg = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!S || !Snew || !cnt || !cnew || !alpha || !beta || !asg) {
    free(S); free(Snew); free(cnt); free(cnew); free(alpha); free(beta); free(asg);
    return ORC_E_NOMEM;
  }
  for (int32_t a = 0; a < k; ++a) {
    for (int32_t b = 0; b < k; ++b) S[(int64_t)a * k + b] = dip[(int64_t)b * n + pivots_in[a]];
    cnt[a] = 1;
  }
  for (int32_t i = 0; i < n; ++i) asg[i] = -1;
  int32_t it = 0;
  for (int32_t pass = 1; pass <= max_iter; ++pass) {
    for (int32_t a = 0; a < k; ++a) {
      double al = 0.0;
      for (int32_t b = 0; b < k; ++b) {
        double c = (double)S[(int64_t)a * k + b] / (double)cnt[a];
        al += c * c;
      }
      alpha[a] = al;
      beta[a] = 2.0 / (double)cnt[a];
    }
    int64_t changed = 0;
    for (int32_t i = 0; i < n; ++i) {
      int32_t best = -1;
      double gbest = 0.0;
      for (int32_t a = 0; a < k; ++a) {
        int64_t t = 0;
        for (int32_t b = 0; b < k; ++b) t += (int64_t)dip[(int64_t)b * n + i] * S[(int64_t)a * k + b];
        double g = alpha[a] - beta[a] * (double)t;
        if (best < 0 || g < gbest) { best = a; gbest = g; }
      }
      if (asg[i] != best) { asg[i] = best; ++changed; }
    }
    it = pass;
    if (pass > 1 && changed == 0) break;
    memset(Snew, 0, (size_t)k * k * sizeof(int64_t));
    memset(cnew, 0, (size_t)k * sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i) {
      int32_t a = asg[i];
      cnew[a] += 1;
      for (int32_t b = 0; b < k; ++b) Snew[(int64_t)a * k + b] += dip[(int64_t)b * n + i];
    }
    for (int32_t a = 0; a < k; ++a)
      if (cnew[a] > 0) {
        cnt[a] = cnew[a];
        for (int32_t b = 0; b < k; ++b) S[(int64_t)a * k + b] = Snew[(int64_t)a * k + b];
      }
  }
  for (int32_t a = 0; a < k; ++a) pivots_out[a] = -1;
  int64_t *vbest = cnew; /* reuse: best n_a ||y_i||^2 - 2 t_ia per cluster */
  for (int32_t i = 0; i < n; ++i) {
    int32_t a = asg[i];
    int64_t yy = 0, t = 0;
    for (int32_t b = 0; b < k; ++b) {
      int64_t y = dip[(int64_t)b * n + i];
      yy += y * y;
      t += y * S[(int64_t)a * k + b];
    }
    int64_t v = cnt[a] * yy - 2 * t;
    if (pivots_out[a] < 0 || v < vbest[a]) { pivots_out[a] = i; vbest[a] = v; }
  }
  for (int32_t a = 0; a < k; ++a)
    if (pivots_out[a] < 0) pivots_out[a] = pivots_in[a];
  if (assign) memcpy(assign, asg, (size_t)n * sizeof(int32_t));
  if (iters) *iters = it;
  free(S); free(Snew); free(cnt); free(cnew); free(alpha); free(beta); free(asg);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* d_ip table (Algorithm 1 line 2), pivot-major [k][n] uint16          */
/* ------------------------------------------------------------------ */

int orc_pivot_dist(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                   const int32_t *pivots, uint16_t *dip) {
  if (k < 1 || k > 65535) return ORC_E_ARG;
  int32_t *d = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!d) return ORC_E_NOMEM;
  int rc = ORC_OK;
  for (int32_t a = 0; rc == ORC_OK && a < k; ++a) {
    rc = orc_bfs(n, rowptr, colidx, pivots[a], d);
    for (int32_t v = 0; rc == ORC_OK && v < n; ++v) {
      if (d[v] < 0) rc = ORC_E_DISCONNECTED;
      else if (d[v] > 65534) rc = ORC_E_DIST_OVERFLOW;
      else dip[(int64_t)a * n + v] = (uint16_t)d[v];
    }
  }
  free(d);
  return rc;
}

/* ------------------------------------------------------------------ */
/* regions R(p) (Section 3)                                            */
/* ------------------------------------------------------------------ */

/* region[i] = the smallest pivot index a minimising d_ia */
int orc_regions(int32_t n, int32_t k, const uint16_t *dip, int32_t *region) {
  for (int32_t i = 0; i < n; ++i) {
    int32_t best = 0;
    for (int32_t a = 1; a < k; ++a)
      if (dip[(int64_t)a * n + i] < dip[(int64_t)best * n + i]) best = a;
    region[i] = best;
  }
  return ORC_OK;
}

/* Regions with the paper's tie rule (Section 3: R is built incrementally
 * while the distances are computed, a tie going to the smallest
 * partition).  Reading: nodes join in the order a multi-source search
 * settles them -- increasing distance L_i = min_a d_ia to their nearest
 * pivots, equal distances by increasing node id; a node with one nearest
 * pivot joins it, a node with several joins the one whose region has the
 * fewest members at that moment, equal sizes to the lowest pivot index. */
int orc_regions_smallest(int32_t n, int32_t k, const uint16_t *dip, int32_t *region) {
  int32_t *L = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int64_t *size = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  int64_t *start = NULL;
  int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!L || !size || !order) { free(L); free(size); free(order); return ORC_E_NOMEM; }
  int32_t lmax = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t m = 65535;
    for (int32_t a = 0; a < k; ++a)
      if (dip[(int64_t)a * n + i] < m) m = dip[(int64_t)a * n + i];
    L[i] = m;
    if (m > lmax) lmax = m;
  }
  /* stable counting sort of the nodes by L */
  start = (int64_t *)calloc((size_t)lmax + 2, sizeof(int64_t));
  if (!start) { free(L); free(size); free(order); return ORC_E_NOMEM; }
  for (int32_t i = 0; i < n; ++i) start[L[i] + 1] += 1;
  for (int32_t l = 0; l <= lmax; ++l) start[l + 1] += start[l];
  for (int32_t i = 0; i < n; ++i) order[start[L[i]]++] = i;
  for (int32_t q = 0; q < n; ++q) {
    int32_t v = order[q], best = -1;
    for (int32_t a = 0; a < k; ++a)
      if (dip[(int64_t)a * n + v] == L[v] && (best < 0 || size[a] < size[best])) best = a;
    region[v] = best;
    size[best] += 1;
  }
  free(L); free(size); free(start); free(order);
  return ORC_OK;
}

/* ecc[a] = max_{j in R(a)} d_ja;  cnt[cnt_off[a] + t] = #{j in R(a): d_ja <= t}
 * for t = 0..ecc[a].  With cnt_off == NULL only ecc is written. */
int orc_histograms(int32_t n, int32_t k, const uint16_t *dip, const int32_t *region,
                   int32_t *ecc, int64_t *cnt_off, uint32_t *cnt, int64_t cnt_cap) {
  for (int32_t a = 0; a < k; ++a) ecc[a] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t a = region[i], d = dip[(int64_t)a * n + i];
    if (d > ecc[a]) ecc[a] = d;
  }
  if (!cnt_off) return ORC_OK;
  cnt_off[0] = 0;
  for (int32_t a = 0; a < k; ++a) cnt_off[a + 1] = cnt_off[a] + ecc[a] + 1;
  if (cnt_off[k] > cnt_cap) return ORC_E_ARG;
  memset(cnt, 0, (size_t)cnt_off[k] * sizeof(uint32_t));
  for (int32_t i = 0; i < n; ++i) {
    int32_t a = region[i];
    cnt[cnt_off[a] + dip[(int64_t)a * n + i]] += 1; /* histogram H[a][t] */
  }
  for (int32_t a = 0; a < k; ++a) /* prefix sums over t */
    for (int64_t t = cnt_off[a] + 1; t < cnt_off[a + 1]; ++t) cnt[t] += cnt[t - 1];
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* adapted weights w'_ip = s / d_ip^2,  s = #{j in R(p): d_jp <= d_ip/2} */
/* ------------------------------------------------------------------ */

static int cmp_u16(const void *a, const void *b) {
  uint16_t x = *(const uint16_t *)a, y = *(const uint16_t *)b;
  return (x > y) - (x < y);
}

/* w[a][i] for every pivot index a and node i, by counting the members of
 * R(a) directly (a sorted list of their distances to p_a and a binary
 * search), independent of orc_histograms.  w = 0 where the pivot term is
 * skipped: d_ia <= 1 (i is p_a, or p_a is a neighbour of i). */
int orc_adapted_weights(int32_t n, int32_t k, const uint16_t *dip, const int32_t *region,
                        double *w) {
  uint16_t *lst = (uint16_t *)malloc((size_t)n * sizeof(uint16_t));
  if (!lst) return ORC_E_NOMEM;
  for (int32_t a = 0; a < k; ++a) {
    int32_t len = 0;
    for (int32_t j = 0; j < n; ++j)
      if (region[j] == a) lst[len++] = dip[(int64_t)a * n + j];
    qsort(lst, (size_t)len, sizeof(uint16_t), cmp_u16);
    for (int32_t i = 0; i < n; ++i) {
      int32_t d = dip[(int64_t)a * n + i];
      double wi = 0.0;
      if (d >= 2) {
        /* s = number of list entries e with 2*e <= d */
        int32_t lo = 0, hi = len;
        while (lo < hi) {
          int32_t mid = lo + (hi - lo) / 2;
          if (2 * (int32_t)lst[mid] <= d) lo = mid + 1; else hi = mid;
        }
        wi = (double)lo / ((double)d * (double)d);
      }
      w[(int64_t)a * n + i] = wi;
    }
  }
  free(lst);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* PivotMDS (Algorithm 1 line 3; Brandes and Pich 2007)                */
/* ------------------------------------------------------------------ */

/* cyclic Jacobi eigenvalue method for a symmetric k x k matrix A (row-major,
 * destroyed): on return diag(A) holds the eigenvalues and the columns of V
 * the eigenvectors.  Sweeps rotate every off-diagonal pair (p,q), p<q, in
 * row order, with the rotation angle chosen to zero A[p][q]. */
static int jacobi_eigen(int32_t k, double *A, double *V) {
  for (int32_t i = 0; i < k; ++i)
    for (int32_t j = 0; j < k; ++j) V[i * k + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int32_t i = 0; i < k; ++i)
      for (int32_t j = 0; j < k; ++j) {
        tot += A[i * k + j] * A[i * k + j];
        if (i != j) off += A[i * k + j] * A[i * k + j];
      }
    if (off <= 1e-30 * tot || off == 0.0) return ORC_OK;
    for (int32_t p = 0; p < k; ++p)
      for (int32_t q = p + 1; q < k; ++q) {
        double apq = A[p * k + q];
        if (apq == 0.0) continue;
        double app = A[p * k + p], aqq = A[q * k + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int32_t r = 0; r < k; ++r) { /* A <- A J (columns p, q) */
          double arp = A[r * k + p], arq = A[r * k + q];
          A[r * k + p] = c * arp - s * arq;
          A[r * k + q] = s * arp + c * arq;
        }
        for (int32_t r = 0; r < k; ++r) { /* A <- J^T A (rows p, q) */
          double apr = A[p * k + r], aqr = A[q * k + r];
          A[p * k + r] = c * apr - s * aqr;
          A[q * k + r] = s * apr + c * aqr;
        }
        for (int32_t r = 0; r < k; ++r) { /* V <- V J */
          double vrp = V[r * k + p], vrq = V[r * k + q];
          V[r * k + p] = c * vrp - s * vrq;
          V[r * k + q] = s * vrp + c * vrq;
        }
      }
  }
  return ORC_E_NUMERIC;
}

/* PivotMDS from the k x n pivot distances:
 *   delta_ia = d_ia^2;
 *   c_ia = -1/2 (delta_ia - rowmean_i - colmean_a + grandmean);
 *   B = C^T C (k x k);  v1, v2 = eigenvectors of the two largest eigenvalues;
 *   each v is signed so that its largest-magnitude entry (lowest index on a
 *   tie) is positive;  x_i = ((C v1)_i, (C v2)_i).
 * pos is [n][2]; eig (optional) receives the two eigenvalues, B (optional,
 * k*k) receives C^T C before the eigen-solve. */
/* the steps after delta: C ([n][k], holding delta_ia on entry) is centred
 * in place; C is released here */
static int pivotmds_from_delta(int32_t n, int32_t k, double *C, double *pos, double *eig, double *Bout) {
  double *rowm = (double *)calloc((size_t)n, sizeof(double));
  double *colm = (double *)calloc((size_t)k, sizeof(double));
  double *B = (double *)calloc((size_t)k * k, sizeof(double));
  double *V = (double *)malloc((size_t)k * k * sizeof(double));
  if (!C || !rowm || !colm || !B || !V) { free(C); free(rowm); free(colm); free(B); free(V); return ORC_E_NOMEM; }
  double grand = 0.0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t a = 0; a < k; ++a) {
      double delta = C[(int64_t)i * k + a];
      rowm[i] += delta;
      colm[a] += delta;
      grand += delta;
    }
  for (int32_t i = 0; i < n; ++i) rowm[i] /= (double)k;
  for (int32_t a = 0; a < k; ++a) colm[a] /= (double)n;
  grand /= (double)n * (double)k;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t a = 0; a < k; ++a)
      C[(int64_t)i * k + a] = -0.5 * (C[(int64_t)i * k + a] - rowm[i] - colm[a] + grand);
  for (int32_t a = 0; a < k; ++a)
    for (int32_t b = 0; b < k; ++b) {
      double s = 0.0;
      for (int32_t i = 0; i < n; ++i) s += C[(int64_t)i * k + a] * C[(int64_t)i * k + b];
      B[a * k + b] = s;
    }
  if (Bout) memcpy(Bout, B, (size_t)k * k * sizeof(double));
  int rc = jacobi_eigen(k, B, V);
  if (rc == ORC_OK) {
    int32_t top[2] = {-1, -1};
    for (int r = 0; r < 2; ++r)
      for (int32_t a = 0; a < k; ++a) {
        if (a == top[0]) continue;
        if (top[r] < 0 || B[a * k + a] > B[top[r] * k + top[r]]) top[r] = a;
      }
    for (int r = 0; r < 2; ++r) {
      int32_t c = top[r], big = 0;
      for (int32_t a = 1; a < k; ++a)
        if (fabs(V[a * k + c]) > fabs(V[big * k + c])) big = a;
      double sg = V[big * k + c] < 0 ? -1.0 : 1.0;
      if (eig) eig[r] = B[c * k + c];
      for (int32_t i = 0; i < n; ++i) {
        double x = 0.0;
        for (int32_t a = 0; a < k; ++a) x += C[(int64_t)i * k + a] * sg * V[a * k + c];
        pos[2 * (int64_t)i + r] = x;
      }
    }
  }
  free(C); free(rowm); free(colm); free(B); free(V);
  return rc;
}

int orc_pivotmds(int32_t n, int32_t k, const uint16_t *dip, double *pos, double *eig, double *Bout) {
  if (k < 2) return ORC_E_ARG;
  double *C = (double *)malloc((size_t)n * k * sizeof(double));
  if (!C) return ORC_E_NOMEM;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t a = 0; a < k; ++a) {
      double d = (double)dip[(int64_t)a * n + i];
      C[(int64_t)i * k + a] = d * d;
    }
  return pivotmds_from_delta(n, k, C, pos, eig, Bout);
}

/* PivotMDS on weighted distances: the same steps with delta_ia = d_ia^2
 * from the float32 table (squared in FP64, exactly) */
int orc_wpivotmds(int32_t n, int32_t k, const float *dip, double *pos, double *eig, double *Bout) {
  if (k < 2) return ORC_E_ARG;
  double *C = (double *)malloc((size_t)n * k * sizeof(double));
  if (!C) return ORC_E_NOMEM;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t a = 0; a < k; ++a) {
      double d = (double)dip[(int64_t)a * n + i];
      C[(int64_t)i * k + a] = d * d;
    }
  return pivotmds_from_delta(n, k, C, pos, eig, Bout);
}

/* ------------------------------------------------------------------ */
/* rescale (Algorithm 1 line 4): sum_E ||x_i - x_j|| = sum_E l_ij = m   */
/* ------------------------------------------------------------------ */

int orc_rescale(int32_t n, const int32_t *rowptr, const int32_t *colidx, double *pos) {
  double len = 0.0;
  int64_t m2 = 0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
      int32_t j = colidx[t];
      if (j <= i) continue;
      double dx = pos[2 * (int64_t)i] - pos[2 * (int64_t)j];
      double dy = pos[2 * (int64_t)i + 1] - pos[2 * (int64_t)j + 1];
      len += sqrt(dx * dx + dy * dy);
      ++m2;
    }
  if (!(len > 0.0)) return ORC_E_NUMERIC;
  double s = (double)m2 / len;
  for (int64_t t = 0; t < 2 * (int64_t)n; ++t) pos[t] *= s;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* the update of Eq. 4                                                 */
/* ------------------------------------------------------------------ */

/* new position of node i from the positions X (Eq. 4): neighbour terms with
 * w_ij = 1, d_ij = 1 (CSR order), then pivot terms a = 0..k-1 with
 * d = d_ia >= 2 and weight w[a][i]. */
static void eq4_update(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                       const int32_t *pivots, const uint16_t *dip, const double *w,
                       const double *X, int32_t i, double *out) {
  double xi = X[2 * (int64_t)i], yi = X[2 * (int64_t)i + 1];
  double nx = 0.0, ny = 0.0, den = 0.0;
  for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
    int32_t j = colidx[t];
    double xj = X[2 * (int64_t)j], yj = X[2 * (int64_t)j + 1];
    double dx = xi - xj, dy = yi - yj;
    double r = sqrt(dx * dx + dy * dy);
    if (r > 0.0) { nx += xj + dx / r; ny += yj + dy / r; }
    else { nx += xj; ny += yj; }
    den += 1.0;
  }
  for (int32_t a = 0; a < k; ++a) {
    int32_t d = dip[(int64_t)a * n + i];
    if (d < 2) continue;
    int32_t p = pivots[a];
    double wa = w[(int64_t)a * n + i];
    double xp = X[2 * (int64_t)p], yp = X[2 * (int64_t)p + 1];
    double dx = xi - xp, dy = yi - yp;
    double r = sqrt(dx * dx + dy * dy);
    if (r > 0.0) { nx += wa * (xp + d * dx / r); ny += wa * (yp + d * dy / r); }
    else { nx += wa * xp; ny += wa * yp; }
    den += wa;
  }
  if (den > 0.0) { out[0] = nx / den; out[1] = ny / den; }
  else { out[0] = xi; out[1] = yi; }
}

/* The Jacobi update of Eq. 4 for the nodes i0 <= i < i1 only (every node's
 * new position depends on X^t alone, so node ranges are independent). */
int orc_sweep_jacobi_rows(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                          const int32_t *pivots, const uint16_t *dip, const double *w,
                          const double *pos_in, double *pos_out, int32_t i0, int32_t i1) {
  if (i0 < 0 || i1 < i0 || i1 > n) return ORC_E_ARG;
  for (int32_t i = i0; i < i1; ++i)
    eq4_update(n, rowptr, colidx, k, pivots, dip, w, pos_in, i, pos_out + 2 * (int64_t)i);
  return ORC_OK;
}

/* relative positional change (Algorithm 1 line 5, read as a Frobenius ratio):
 * ||X^{t+1} - X^t||_F / ||X^t||_F, summed in coordinate order */
double orc_relchange(int32_t n, const double *pos_in, const double *pos_out) {
  double num = 0.0, den = 0.0;
  for (int64_t t = 0; t < 2 * (int64_t)n; ++t) {
    double dd = pos_out[t] - pos_in[t];
    num += dd * dd;
    den += pos_in[t] * pos_in[t];
  }
  return den > 0.0 ? sqrt(num) / sqrt(den) : 0.0;
}

/* Jacobi: X^{t+1}_i from X^t for every i; relchange (optional) receives
 * ||X^{t+1} - X^t||_F / ||X^t||_F. */
int orc_sweep_jacobi(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                     const int32_t *pivots, const uint16_t *dip, const double *w,
                     const double *pos_in, double *pos_out, double *relchange) {
  orc_sweep_jacobi_rows(n, rowptr, colidx, k, pivots, dip, w, pos_in, pos_out, 0, n);
  if (relchange) *relchange = orc_relchange(n, pos_in, pos_out);
  return ORC_OK;
}

/* Gauss-Seidel, the paper's order: x_i <- Eq. 4 for i = 0..n-1, in place */
int orc_sweep_gs(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                 const int32_t *pivots, const uint16_t *dip, const double *w, double *pos) {
  double t[2];
  for (int32_t i = 0; i < n; ++i) {
    eq4_update(n, rowptr, colidx, k, pivots, dip, w, pos, i, t);
    pos[2 * (int64_t)i] = t[0];
    pos[2 * (int64_t)i + 1] = t[1];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* full stress majorization (Section 3, the update before Eq. 4)        */
/* ------------------------------------------------------------------ */

/* new position of node i under full stress: every j != i with
 * w_ij = 1/d_ij^2, d_ij = D[i*n + j] (all-pairs hop distances), j ascending */
static void full_update(int32_t n, const uint16_t *D, const double *X, int32_t i, double *out) {
  double xi = X[2 * (int64_t)i], yi = X[2 * (int64_t)i + 1];
  double nx = 0.0, ny = 0.0, den = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    if (j == i) continue;
    double d = (double)D[(int64_t)i * n + j];
    double w = 1.0 / (d * d);
    double xj = X[2 * (int64_t)j], yj = X[2 * (int64_t)j + 1];
    double dx = xi - xj, dy = yi - yj;
    double r = sqrt(dx * dx + dy * dy);
    if (r > 0.0) { nx += w * (xj + d * dx / r); ny += w * (yj + d * dy / r); }
    else { nx += w * xj; ny += w * yj; }
    den += w;
  }
  if (den > 0.0) { out[0] = nx / den; out[1] = ny / den; }
  else { out[0] = xi; out[1] = yi; }
}

/* One sweep of full stress majorization over the n x n distance table D.
 * order 0: Jacobi (every node from pos_in); order 1: Gauss-Seidel, nodes
 * 0..n-1 in turn, each from the positions already moved (the node-at-a-time
 * order under which full stress decreases monotonically).  pos_out receives
 * the new layout; relchange (optional) ||X' - X||_F / ||X||_F. */
int orc_full_sweep(int32_t n, const uint16_t *D, const double *pos_in, double *pos_out, int32_t order,
                   double *relchange) {
  if (n < 1 || (order != 0 && order != 1)) return ORC_E_ARG;
  for (int64_t t = 0; t < (int64_t)n * n; ++t)
    if (D[t] == 0xFFFF) return ORC_E_DISCONNECTED;
  if (order == 0) {
    for (int32_t i = 0; i < n; ++i) full_update(n, D, pos_in, i, pos_out + 2 * (int64_t)i);
  } else {
    memcpy(pos_out, pos_in, 2 * (size_t)n * sizeof(double));
    double t[2];
    for (int32_t i = 0; i < n; ++i) {
      full_update(n, D, pos_out, i, t);
      pos_out[2 * (int64_t)i] = t[0];
      pos_out[2 * (int64_t)i + 1] = t[1];
    }
  }
  if (relchange) *relchange = orc_relchange(n, pos_in, pos_out);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* layout quality (Section 4)                                          */
/* ------------------------------------------------------------------ */

/* Procrustes statistic (Sibson 1978) of two layouts X and Y of the same n
 * nodes ([n][2]): both centred, Y fitted by a uniform scale s and a proper
 * rotation R (no reflection: Section 4 notes that the analysis cannot
 * resolve reflections),
 *   P = 1 - T^2 / (||Xc||^2 ||Yc||^2),  T = max_R tr(R Xc^T Yc)
 *     = sqrt((m11 + m22)^2 + (m12 - m21)^2),  m_ab = sum_i xc_ia yc_ib.
 * P is in [0, 1], 0 for a perfect match.  out = {P, s, theta} with
 * Y ~ s R(theta) X + translation, R(theta) = [[c, -s], [s, c]]. */
int orc_procrustes(int32_t n, const double *X, const double *Y, double *out) {
  if (n < 1) return ORC_E_ARG;
  double mx0 = 0.0, mx1 = 0.0, my0 = 0.0, my1 = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    mx0 += X[2 * (int64_t)i]; mx1 += X[2 * (int64_t)i + 1];
    my0 += Y[2 * (int64_t)i]; my1 += Y[2 * (int64_t)i + 1];
  }
  mx0 /= n; mx1 /= n; my0 /= n; my1 /= n;
  double m11 = 0.0, m12 = 0.0, m21 = 0.0, m22 = 0.0, xx = 0.0, yy = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    double x0 = X[2 * (int64_t)i] - mx0, x1 = X[2 * (int64_t)i + 1] - mx1;
    double y0 = Y[2 * (int64_t)i] - my0, y1 = Y[2 * (int64_t)i + 1] - my1;
    m11 += x0 * y0; m12 += x0 * y1; m21 += x1 * y0; m22 += x1 * y1;
    xx += x0 * x0 + x1 * x1;
    yy += y0 * y0 + y1 * y1;
  }
  double a = m11 + m22, b = m12 - m21;
  double T = sqrt(a * a + b * b);
  if (!(xx > 0.0) || !(yy > 0.0)) { out[0] = 1.0; out[1] = 0.0; out[2] = 0.0; return ORC_OK; }
  out[0] = 1.0 - T * T / (xx * yy);
  out[1] = T / xx;
  out[2] = atan2(b, a);
  return ORC_OK;
}

/* cross product (b - a) x (c - a), evaluated as written (the hull and the
 * inside test of orc_hull_error share it) */
static double cross3(const double *a, const double *b, const double *c) {
  double ux = b[0] - a[0], uy = b[1] - a[1], vx = c[0] - a[0], vy = c[1] - a[1];
  return ux * vy - uy * vx;
}

static const double *g_sort_pos; /* qsort context of the hull */
static int cmp_xy(const void *pa, const void *pb) {
  int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
  const double *A = g_sort_pos + 2 * (int64_t)a, *B = g_sort_pos + 2 * (int64_t)b;
  if (A[0] != B[0]) return A[0] < B[0] ? -1 : 1;
  if (A[1] != B[1]) return A[1] < B[1] ? -1 : 1;
  return (a > b) - (a < b);
}

/* convex hull of the points idx[0..m) of pos (Andrew's monotone chain: sort by
 * (x, y, index), lower then upper chain, a point is dropped while the turn
 * it makes is not strictly counter-clockwise); hull receives the vertex
 * indices counter-clockwise without repeating the first; returns their count */
static int32_t monotone_hull(const double *pos, int32_t *idx, int32_t m, int32_t *hull) {
  g_sort_pos = pos;
  qsort(idx, (size_t)m, sizeof(int32_t), cmp_xy);
  int32_t h = 0;
  for (int32_t t = 0; t < m; ++t) { /* lower chain */
    while (h >= 2 && cross3(pos + 2 * (int64_t)hull[h - 2], pos + 2 * (int64_t)hull[h - 1], pos + 2 * (int64_t)idx[t]) <= 0.0) --h;
    hull[h++] = idx[t];
  }
  int32_t lo = h + 1;
  for (int32_t t = m - 2; t >= 0; --t) { /* upper chain */
    while (h >= lo && cross3(pos + 2 * (int64_t)hull[h - 2], pos + 2 * (int64_t)hull[h - 1], pos + 2 * (int64_t)idx[t]) <= 0.0) --h;
    hull[h++] = idx[t];
  }
  if (h > 1) --h; /* the last point repeats the first */
  return h;
}

/* is q inside or on the convex polygon hull[0..h) (counter-clockwise)?  A
 * hull of one point: q equal to it; of two points: q on the segment */
static int in_hull(const double *pos, const int32_t *hull, int32_t h, const double *q) {
  if (h == 1) return q[0] == pos[2 * (int64_t)hull[0]] && q[1] == pos[2 * (int64_t)hull[0] + 1];
  if (h == 2) {
    const double *a = pos + 2 * (int64_t)hull[0], *b = pos + 2 * (int64_t)hull[1];
    if (cross3(a, b, q) != 0.0) return 0;
    return q[0] >= fmin(a[0], b[0]) && q[0] <= fmax(a[0], b[0]) && q[1] >= fmin(a[1], b[1]) && q[1] <= fmax(a[1], b[1]);
  }
  double x0 = pos[2 * (int64_t)hull[0]], x1 = x0, y0 = pos[2 * (int64_t)hull[0] + 1], y1 = y0;
  for (int32_t e = 1; e < h; ++e) { /* outside the hull's bounding box: outside */
    x0 = fmin(x0, pos[2 * (int64_t)hull[e]]); x1 = fmax(x1, pos[2 * (int64_t)hull[e]]);
    y0 = fmin(y0, pos[2 * (int64_t)hull[e] + 1]); y1 = fmax(y1, pos[2 * (int64_t)hull[e] + 1]);
  }
  if (q[0] < x0 || q[0] > x1 || q[1] < y0 || q[1] > y1) return 0;
  for (int32_t e = 0; e < h; ++e) {
    const double *a = pos + 2 * (int64_t)hull[e], *b = pos + 2 * (int64_t)hull[(e + 1) % h];
    if (cross3(a, b, q) < 0.0) return 0;
  }
  return 1;
}

/* Convex-hull error (Section 4, Fig. 4): for node v, B = {w : d_vw <= kh}
 * (graph distances D, [n][n]), H = convex hull of the positions of B;
 * err_v = |{u not in B : x_u inside or on H}| / (n - |B|) (0 when B = V).
 * per_node (optional) receives err_v; *mean their mean in node order. */
int orc_hull_error(int32_t n, const uint16_t *D, const double *pos, int32_t kh, double *per_node, double *mean) {
  if (n < 1 || kh < 0) return ORC_E_ARG;
  int32_t *ball = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *hull = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
  if (!ball || !hull) { free(ball); free(hull); return ORC_E_NOMEM; }
  double sum = 0.0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t m = 0;
    for (int32_t w = 0; w < n; ++w)
      if (D[(int64_t)v * n + w] <= kh) ball[m++] = w;
    double err = 0.0;
    if (m < n) {
      int32_t h = monotone_hull(pos, ball, m, hull);
      int64_t cnt = 0;
      for (int32_t u = 0; u < n; ++u)
        if (D[(int64_t)v * n + u] > kh && in_hull(pos, hull, h, pos + 2 * (int64_t)u)) ++cnt;
      err = (double)cnt / (double)(n - m);
    }
    if (per_node) per_node[v] = err;
    sum += err;
  }
  *mean = sum / (double)n;
  free(ball); free(hull);
  return ORC_OK;
}

/* Is w strictly inside the disc with diameter ab?  |2w - a - b|^2 < |a - b|^2,
 * evaluated as written with a the lower and b the higher node id, so that
 * the test for the pair (a, b) does not depend on the order it is asked in. */
static int in_diameter_disc(const double *pos, int32_t a, int32_t b, int32_t w) {
  if (a > b) { int32_t t = a; a = b; b = t; }
  const double *A = pos + 2 * (int64_t)a, *B = pos + 2 * (int64_t)b, *W = pos + 2 * (int64_t)w;
  double tx = 2.0 * W[0] - A[0] - B[0], ty = 2.0 * W[1] - A[1] - B[1];
  double ex = A[0] - B[0], ey = A[1] - B[1];
  return tx * tx + ty * ty < ex * ex + ey * ey;
}

/* Gabriel graph of a layout (Section 4, after Fig. 4): u and v adjacent iff
 * no other point lies inside the disc with diameter uv (read as the open
 * disc, so identical positions -- a disc of radius 0 -- are adjacent, as the
 * paper adds them).  adj[u*n + v] = 1 for an edge (n x n bytes). */
int orc_gabriel(int32_t n, const double *pos, uint8_t *adj) {
  if (n < 1) return ORC_E_ARG;
  memset(adj, 0, (size_t)n * n);
  for (int32_t u = 0; u < n; ++u)
    for (int32_t v = u + 1; v < n; ++v) {
      int ok = 1;
      for (int32_t w = 0; w < n && ok; ++w)
        if (w != u && w != v && in_diameter_disc(pos, u, v, w)) ok = 0;
      if (ok) adj[(int64_t)u * n + v] = adj[(int64_t)v * n + u] = 1;
    }
  return ORC_OK;
}

/* nodes within kh hops of s in the graph adj (n x n), s excluded; mark[]
 * receives 1 for them; returns their number */
static int32_t ball_adj(int32_t n, const uint8_t *adj, int32_t s, int32_t kh, int32_t *dist, int32_t *queue,
                        uint8_t *mark) {
  for (int32_t v = 0; v < n; ++v) { dist[v] = -1; mark[v] = 0; }
  int32_t head = 0, tail = 0, cnt = 0;
  dist[s] = 0;
  queue[tail++] = s;
  while (head < tail) {
    int32_t u = queue[head++];
    if (dist[u] == kh) continue;
    for (int32_t v = 0; v < n; ++v)
      if (adj[(int64_t)u * n + v] && dist[v] < 0) {
        dist[v] = dist[u] + 1;
        queue[tail++] = v;
        mark[v] = 1;
        ++cnt;
      }
  }
  return cnt;
}

/* Gabriel-graph similarity (Section 4, Fig. 3): the Gabriel graphs of two
 * layouts A and B of the same nodes, and for every node v the Jaccard
 * coefficient of its kh-neighbourhoods (nodes within kh hops, v itself
 * excluded) in the two graphs; 1 when both are empty.  per_node
 * (optional) receives them, *mean their mean in node order. */
int orc_gabriel_jaccard(int32_t n, const double *posA, const double *posB, int32_t kh, double *per_node,
                        double *mean) {
  if (n < 1 || kh < 1) return ORC_E_ARG;
  uint8_t *ga = (uint8_t *)malloc((size_t)n * n), *gb = (uint8_t *)malloc((size_t)n * n);
  uint8_t *ma = (uint8_t *)malloc((size_t)n), *mb = (uint8_t *)malloc((size_t)n);
  int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t)), *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!ga || !gb || !ma || !mb || !dist || !queue) {
    free(ga); free(gb); free(ma); free(mb); free(dist); free(queue);
    return ORC_E_NOMEM;
  }
  orc_gabriel(n, posA, ga);
  orc_gabriel(n, posB, gb);
  double sum = 0.0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t ca = ball_adj(n, ga, v, kh, dist, queue, ma);
    int32_t cb = ball_adj(n, gb, v, kh, dist, queue, mb);
    int32_t both = 0;
    for (int32_t w = 0; w < n; ++w) both += ma[w] & mb[w];
    int32_t uni = ca + cb - both;
    double j = uni > 0 ? (double)both / (double)uni : 1.0;
    if (per_node) per_node[v] = j;
    sum += j;
  }
  *mean = sum / (double)n;
  free(ga); free(gb); free(ma); free(mb); free(dist); free(queue);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* stress (Eq. 1) with optimal scaling                                 */
/* ------------------------------------------------------------------ */

/* splitmix64 as a counter-based generator: value c of stream `seed` is the
 * output mix of state seed + (c+1)*0x9E3779B97F4A7C15 (Steele, Lea, Flood 2014) */
static uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int orc_splitmix64(uint64_t seed, int64_t count, uint64_t *out) {
  for (int64_t c = 0; c < count; ++c) out[c] = splitmix64_at(seed, (uint64_t)c);
  return ORC_OK;
}

/* The sampled pair list: source j (0 <= j < S) is node
 * (hi32(u_j) * n) >> 32 with u_j = value j of the stream; target l of
 * source j uses u = value S + j*T + l, t' = (hi32(u) * (n-1)) >> 32 and
 * t = t' + (t' >= source), i.e. uniform over the other n-1 nodes. */
int orc_sample_pairs(int32_t n, int32_t S, int32_t T, uint64_t seed, int32_t *srcs, int32_t *tgts) {
  if (n < 2 || S < 1 || T < 1) return ORC_E_ARG;
  for (int32_t j = 0; j < S; ++j)
    srcs[j] = (int32_t)(((splitmix64_at(seed, (uint64_t)j) >> 32) * (uint64_t)n) >> 32);
  for (int32_t j = 0; j < S; ++j)
    for (int32_t l = 0; l < T; ++l) {
      uint64_t u = splitmix64_at(seed, (uint64_t)S + (uint64_t)j * T + l);
      int32_t t = (int32_t)(((u >> 32) * (uint64_t)(n - 1)) >> 32);
      tgts[(int64_t)j * T + l] = t + (t >= srcs[j]);
    }
  return ORC_OK;
}

/* Pair sums of Eq. 1 over the sources q0 <= q < q1 of the pair list that
 * orc_full_stress uses (S == 0: sources are the nodes, targets j > i; S > 0:
 * the S*T sampled pairs of orc_sample_pairs).  acc[4] receives
 * {sum (r-d)^2/d^2, S1 = sum r/d, S2 = sum r^2/d^2, N}, each summed pair by
 * pair in list order.  srcs/tgts are the sampled list (NULL when S == 0). */
static int stress_accumulate(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *pos,
                             int32_t S, int32_t T, const int32_t *srcs, const int32_t *tgts, int32_t q0,
                             int32_t q1, int32_t *dist, double *acc) {
  double raw = 0.0, s1 = 0.0, s2 = 0.0, np = 0.0;
  int rc = ORC_OK;
  for (int32_t q = q0; rc == ORC_OK && q < q1; ++q) {
    int32_t i = S > 0 ? srcs[q] : q;
    rc = orc_bfs(n, rowptr, colidx, i, dist);
    int32_t cnt = S > 0 ? T : n;
    for (int32_t l = 0; rc == ORC_OK && l < cnt; ++l) {
      int32_t j = S > 0 ? tgts[(int64_t)q * T + l] : l;
      if (S == 0 && j <= i) continue;
      if (dist[j] < 0) { rc = ORC_E_DISCONNECTED; break; }
      double d = (double)dist[j];
      double dx = pos[2 * (int64_t)i] - pos[2 * (int64_t)j];
      double dy = pos[2 * (int64_t)i + 1] - pos[2 * (int64_t)j + 1];
      double r = sqrt(dx * dx + dy * dy);
      raw += (r - d) * (r - d) / (d * d);
      s1 += r / d;
      s2 += r * r / (d * d);
      np += 1.0;
    }
  }
  acc[0] = raw; acc[1] = s1; acc[2] = s2; acc[3] = np;
  return rc;
}

/* Full stress of the layout pos.
 * S == 0: exhaustive, every pair i < j (a BFS from every node).
 * S > 0:  the S*T sampled pairs of orc_sample_pairs (a BFS from every source).
 * sums (optional) receives {sum (r-d)^2/d^2, S1 = sum r/d, S2 = sum r^2/d^2, N}.
 * out = {raw, alpha*, scaled, normalized}: raw = sum (r-d)^2/d^2 (sampled:
 * scaled to C(n,2) pairs by C(n,2)/N); alpha* = S1/S2 minimises
 * sum (alpha r - d)^2 / d^2; scaled = N - S1^2/S2 (sampled: times C(n,2)/N);
 * normalized = scaled / C(n,2). */
int orc_full_stress(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *pos,
                    int32_t S, int32_t T, uint64_t seed, double *out, double *sums) {
  if (n < 2 || S < 0 || (S > 0 && T < 1)) return ORC_E_ARG;
  int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *srcs = NULL, *tgts = NULL;
  if (!dist) return ORC_E_NOMEM;
  if (S > 0) {
    srcs = (int32_t *)malloc((size_t)S * sizeof(int32_t));
    tgts = (int32_t *)malloc((size_t)S * T * sizeof(int32_t));
    if (!srcs || !tgts) { free(dist); free(srcs); free(tgts); return ORC_E_NOMEM; }
    orc_sample_pairs(n, S, T, seed, srcs, tgts);
  }
  double acc[4];
  int rc = stress_accumulate(n, rowptr, colidx, pos, S, T, srcs, tgts, 0, S > 0 ? S : n, dist, acc);
  free(dist); free(srcs); free(tgts);
  if (rc != ORC_OK) return rc;
  double raw = acc[0], s1 = acc[1], s2 = acc[2], np = acc[3];
  double pairs = 0.5 * (double)n * (double)(n - 1);
  double f = S > 0 ? pairs / np : 1.0;
  if (sums) { sums[0] = raw; sums[1] = s1; sums[2] = s2; sums[3] = np; }
  out[0] = raw * f;
  out[1] = s2 > 0.0 ? s1 / s2 : 0.0;
  out[2] = (s2 > 0.0 ? np - s1 * s1 / s2 : np) * f;
  out[3] = out[2] / pairs;
  return ORC_OK;
}

/* The pair sums of orc_full_stress restricted to the sources q0 <= q < q1 of
 * its pair list (so that independent source ranges can be evaluated by
 * separate callers and added); sums[4] as in orc_full_stress. */
int orc_stress_sums_range(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *pos,
                          int32_t S, int32_t T, uint64_t seed, int32_t q0, int32_t q1, double *sums) {
  int32_t nsrc = S > 0 ? S : n;
  if (n < 2 || S < 0 || (S > 0 && T < 1) || q0 < 0 || q1 < q0 || q1 > nsrc) return ORC_E_ARG;
  int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *srcs = NULL, *tgts = NULL;
  if (!dist) return ORC_E_NOMEM;
  if (S > 0) {
    srcs = (int32_t *)malloc((size_t)S * sizeof(int32_t));
    tgts = (int32_t *)malloc((size_t)S * T * sizeof(int32_t));
    if (!srcs || !tgts) { free(dist); free(srcs); free(tgts); return ORC_E_NOMEM; }
    orc_sample_pairs(n, S, T, seed, srcs, tgts);
  }
  int rc = stress_accumulate(n, rowptr, colidx, pos, S, T, srcs, tgts, q0, q1, dist, sums);
  free(dist); free(srcs); free(tgts);
  return rc;
}

/* ------------------------------------------------------------------ */
/* weighted graphs (Algorithm 1 line 2: weighted MSSP; Section 3)        */
/* ------------------------------------------------------------------ */
/* Edge lengths l_ij are float32 (finite, at least FLT_MIN, n * max l below
 * 1e37 so no path sum overflows).  A distance is the least path sum over the
 * s-v paths with every partial sum rounded to float32 as the path is walked
 * from s (d(v) = fl(d(u) + l_uv)); rounding is monotone, so this minimum is
 * what any label-setting or label-correcting search reaches.  Stress weights
 * are w_ij = l_ij^-2 on edges and w'_ip = s / d_ip^2 on pivots, with s the
 * number of j in R(p) with 2 d_jp <= d_ip, decided in float32. */

typedef struct { float d; int32_t v; } wheap_item;

static void wheap_push(wheap_item *h, int64_t *len, float d, int32_t v) {
  int64_t i = (*len)++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].d <= d) break;
    h[i] = h[p];
    i = p;
  }
  h[i].d = d;
  h[i].v = v;
}

static wheap_item wheap_pop(wheap_item *h, int64_t *len) {
  wheap_item top = h[0], last = h[--(*len)];
  int64_t i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= *len) break;
    if (c + 1 < *len && h[c + 1].d < h[c].d) ++c;
    if (last.d <= h[c].d) break;
    h[i] = h[c];
    i = c;
  }
  if (*len > 0) h[i] = last;
  return top;
}

typedef struct { int32_t v; float l; } nbr_len;

static int cmp_nbr_len(const void *a, const void *b) {
  const nbr_len *x = (const nbr_len *)a, *y = (const nbr_len *)b;
  if (x->v != y->v) return (x->v > y->v) - (x->v < y->v);
  return (x->l > y->l) - (x->l < y->l);
}

/* Weighted simple undirected graph: as orc_build_csr, and elen[t] is the
 * length of the edge colidx[t]; a repeated edge keeps its shortest length.
 * Lengths must be finite, at least FLT_MIN, with n * max length < 1e37. */
int orc_build_wcsr(int32_t n, int64_t m_in, const int32_t *src, const int32_t *dst, const float *len,
                   int32_t *rowptr, int32_t *colidx, float *elen, int64_t *m_out) {
  if (n < 1 || m_in < 0) return ORC_E_ARG;
  double lmax = 0.0;
  for (int64_t e = 0; e < m_in; ++e) {
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return ORC_E_GRAPH;
    if (!(len[e] >= 1.17549435e-38f) || !(len[e] <= 3.4e38f)) return ORC_E_ARG;
    if (len[e] > lmax) lmax = len[e];
  }
  if ((double)n * lmax >= 1e37) return ORC_E_ARG;
  int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  nbr_len *tmp = (nbr_len *)malloc((size_t)(2 * m_in + 1) * sizeof(nbr_len));
  if (!deg || !fill || !tmp) { free(deg); free(fill); free(tmp); return ORC_E_NOMEM; }
  for (int64_t e = 0; e < m_in; ++e)
    if (src[e] != dst[e]) { deg[src[e] + 1]++; deg[dst[e] + 1]++; }
  for (int32_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
  memcpy(fill, deg, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t e = 0; e < m_in; ++e)
    if (src[e] != dst[e]) {
      nbr_len a = {dst[e], len[e]}, b = {src[e], len[e]};
      tmp[fill[src[e]]++] = a;
      tmp[fill[dst[e]]++] = b;
    }
  int64_t out = 0;
  rowptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int64_t b = deg[i], e = deg[i + 1];
    qsort(tmp + b, (size_t)(e - b), sizeof(nbr_len), cmp_nbr_len);
    for (int64_t t = b; t < e; ++t)
      if (t == b || tmp[t].v != tmp[t - 1].v) {  /* first of a group: the shortest */
        colidx[out] = tmp[t].v;
        elen[out] = tmp[t].l;
        ++out;
      }
    rowptr[i + 1] = (int32_t)out;
  }
  free(deg); free(fill); free(tmp);
  *m_out = out / 2;
  return ORC_OK;
}

/* Dijkstra's algorithm with a binary heap (lazy deletion), float32 sums:
 * dist[v] = least rounded path sum from s, +inf if unreachable. */
int orc_sssp(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t s, float *dist) {
  if (s < 0 || s >= n) return ORC_E_ARG;
  int64_t cap = (int64_t)rowptr[n] + 1;
  wheap_item *h = (wheap_item *)malloc((size_t)cap * sizeof(wheap_item));
  uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
  if (!h || !done) { free(h); free(done); return ORC_E_NOMEM; }
  for (int32_t v = 0; v < n; ++v) dist[v] = INFINITY;
  int64_t len = 0;
  dist[s] = 0.0f;
  wheap_push(h, &len, 0.0f, s);
  while (len > 0) {
    wheap_item it = wheap_pop(h, &len);
    int32_t u = it.v;
    if (done[u]) continue;
    done[u] = 1;
    for (int32_t t = rowptr[u]; t < rowptr[u + 1]; ++t) {
      int32_t v = colidx[t];
      float nd = dist[u] + elen[t];
      if (nd < dist[v]) {
        dist[v] = nd;
        wheap_push(h, &len, nd, v);
      }
    }
  }
  free(h); free(done);
  return ORC_OK;
}

/* max/min sp on weighted distances (Section 4.1): as orc_maxmin with one
 * Dijkstra per pivot; ties to the lowest node id. */
int orc_wmaxmin(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t k,
                int32_t start, int32_t *pivots) {
  if (k < 1 || k > n || start < 0 || start >= n) return ORC_E_ARG;
  float *mind = (float *)malloc((size_t)n * sizeof(float));
  float *d = (float *)malloc((size_t)n * sizeof(float));
  if (!mind || !d) { free(mind); free(d); return ORC_E_NOMEM; }
  int rc = orc_sssp(n, rowptr, colidx, elen, start, mind);
  for (int32_t v = 0; rc == ORC_OK && v < n; ++v)
    if (isinf(mind[v])) rc = ORC_E_DISCONNECTED;
  if (rc == ORC_OK) pivots[0] = start;
  for (int32_t j = 1; rc == ORC_OK && j < k; ++j) {
    int32_t best = 0;
    for (int32_t v = 1; v < n; ++v)
      if (mind[v] > mind[best]) best = v;
    pivots[j] = best;
    rc = orc_sssp(n, rowptr, colidx, elen, best, d);
    for (int32_t v = 0; v < n; ++v)
      if (d[v] < mind[v]) mind[v] = d[v];
  }
  free(mind); free(d);
  return rc;
}

/* weighted d_ip, pivot-major [k][n] float32, one Dijkstra per pivot */
int orc_wpivot_dist(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t k,
                    const int32_t *pivots, float *dip) {
  if (k < 1) return ORC_E_ARG;
  int rc = ORC_OK;
  for (int32_t a = 0; rc == ORC_OK && a < k; ++a) {
    rc = orc_sssp(n, rowptr, colidx, elen, pivots[a], dip + (int64_t)a * n);
    for (int32_t v = 0; rc == ORC_OK && v < n; ++v)
      if (isinf(dip[(int64_t)a * n + v])) rc = ORC_E_DISCONNECTED;
  }
  return rc;
}

/* region[i] = the smallest pivot index a minimising d_ia (float32) */
int orc_wregions(int32_t n, int32_t k, const float *dip, int32_t *region) {
  for (int32_t i = 0; i < n; ++i) {
    int32_t best = 0;
    for (int32_t a = 1; a < k; ++a)
      if (dip[(int64_t)a * n + i] < dip[(int64_t)best * n + i]) best = a;
    region[i] = best;
  }
  return ORC_OK;
}

static int row_has(const int32_t *rowptr, const int32_t *colidx, int32_t i, int32_t v) {
  for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t)
    if (colidx[t] == v) return 1;
  return 0;
}

/* s[a][i] = |{j in R(a) : 2 d_ja <= d_ia}| by direct count (Section 3,
 * after Eq. 4), for the nodes i0 <= i < i1; 0 where the pivot is i itself
 * or one of its neighbours (the pivot sum of Eq. 4 runs over P \ N(i) and
 * skips i). */
int orc_wcounts_rows(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k, const int32_t *pivots,
                     const float *dip, const int32_t *region, uint32_t *s, int32_t i0, int32_t i1) {
  if (i0 < 0 || i1 < i0 || i1 > n) return ORC_E_ARG;
  for (int32_t a = 0; a < k; ++a) {
    const float *row = dip + (int64_t)a * n;
    for (int32_t i = i0; i < i1; ++i) {
      uint32_t c = 0;
      if (pivots[a] != i && !row_has(rowptr, colidx, i, pivots[a]))
        for (int32_t j = 0; j < n; ++j)
          if (region[j] == a && 2.0f * row[j] <= row[i]) ++c;
      s[(int64_t)a * n + i] = c;
    }
  }
  return ORC_OK;
}

/* rescale with the weighted target: sum_E ||x_i - x_j|| = sum_E l_ij
 * (Algorithm 1 line 4; both sums over i < j in CSR order, FP64) */
int orc_wrescale(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, double *pos) {
  double len = 0.0, target = 0.0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
      int32_t j = colidx[t];
      if (j <= i) continue;
      double dx = pos[2 * (int64_t)i] - pos[2 * (int64_t)j];
      double dy = pos[2 * (int64_t)i + 1] - pos[2 * (int64_t)j + 1];
      len += sqrt(dx * dx + dy * dy);
      target += (double)elen[t];
    }
  if (!(len > 0.0)) return ORC_E_NUMERIC;
  double sc = target / len;
  for (int64_t t = 0; t < 2 * (int64_t)n; ++t) pos[t] *= sc;
  return ORC_OK;
}

/* Eq. 4 on a weighted graph, node i from X: neighbour terms with
 * d_ij = l_ij, w_ij = 1 / l_ij^2 (CSR order), then pivot terms a = 0..k-1
 * with d = d_ia, w' = s_ia / d^2, skipping the pivot when it is i or a
 * neighbour of i. */
static void eq4w_update(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t k,
                        const int32_t *pivots, const float *dip, const uint32_t *s, const double *X, int32_t i,
                        double *out) {
  double xi = X[2 * (int64_t)i], yi = X[2 * (int64_t)i + 1];
  double nx = 0.0, ny = 0.0, den = 0.0;
  for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
    int32_t j = colidx[t];
    double l = (double)elen[t], w = 1.0 / (l * l);
    double xj = X[2 * (int64_t)j], yj = X[2 * (int64_t)j + 1];
    double dx = xi - xj, dy = yi - yj;
    double r = sqrt(dx * dx + dy * dy);
    if (r > 0.0) { nx += w * (xj + l * dx / r); ny += w * (yj + l * dy / r); }
    else { nx += w * xj; ny += w * yj; }
    den += w;
  }
  for (int32_t a = 0; a < k; ++a) {
    int32_t p = pivots[a];
    if (p == i || row_has(rowptr, colidx, i, p)) continue;
    double d = (double)dip[(int64_t)a * n + i];
    double wa = (double)s[(int64_t)a * n + i] / (d * d);
    double xp = X[2 * (int64_t)p], yp = X[2 * (int64_t)p + 1];
    double dx = xi - xp, dy = yi - yp;
    double r = sqrt(dx * dx + dy * dy);
    if (r > 0.0) { nx += wa * (xp + d * dx / r); ny += wa * (yp + d * dy / r); }
    else { nx += wa * xp; ny += wa * yp; }
    den += wa;
  }
  if (den > 0.0) { out[0] = nx / den; out[1] = ny / den; }
  else { out[0] = xi; out[1] = yi; }
}

int orc_wsweep_jacobi_rows(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t k,
                           const int32_t *pivots, const float *dip, const uint32_t *s, const double *pos_in,
                           double *pos_out, int32_t i0, int32_t i1) {
  if (i0 < 0 || i1 < i0 || i1 > n) return ORC_E_ARG;
  for (int32_t i = i0; i < i1; ++i)
    eq4w_update(n, rowptr, colidx, elen, k, pivots, dip, s, pos_in, i, pos_out + 2 * (int64_t)i);
  return ORC_OK;
}

/* full stress (Eq. 1) with weighted distances: exhaustive (S == 0, a
 * Dijkstra from every node, pairs i < j) or over the S*T pairs of
 * orc_sample_pairs; out and sums as in orc_full_stress. */
int orc_wfull_stress(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen,
                     const double *pos, int32_t S, int32_t T, uint64_t seed, double *out, double *sums) {
  if (n < 2 || S < 0 || (S > 0 && T < 1)) return ORC_E_ARG;
  float *dist = (float *)malloc((size_t)n * sizeof(float));
  int32_t *srcs = NULL, *tgts = NULL;
  if (!dist) return ORC_E_NOMEM;
  if (S > 0) {
    srcs = (int32_t *)malloc((size_t)S * sizeof(int32_t));
    tgts = (int32_t *)malloc((size_t)S * T * sizeof(int32_t));
    if (!srcs || !tgts) { free(dist); free(srcs); free(tgts); return ORC_E_NOMEM; }
    orc_sample_pairs(n, S, T, seed, srcs, tgts);
  }
  double raw = 0.0, s1 = 0.0, s2 = 0.0, np = 0.0;
  int rc = ORC_OK;
  int32_t nsrc = S > 0 ? S : n;
  for (int32_t q = 0; rc == ORC_OK && q < nsrc; ++q) {
    int32_t i = S > 0 ? srcs[q] : q;
    rc = orc_sssp(n, rowptr, colidx, elen, i, dist);
    int32_t cnt = S > 0 ? T : n;
    for (int32_t l = 0; rc == ORC_OK && l < cnt; ++l) {
      int32_t j = S > 0 ? tgts[(int64_t)q * T + l] : l;
      if (S == 0 && j <= i) continue;
      if (isinf(dist[j])) { rc = ORC_E_DISCONNECTED; break; }
      double d = (double)dist[j];
      double dx = pos[2 * (int64_t)i] - pos[2 * (int64_t)j];
      double dy = pos[2 * (int64_t)i + 1] - pos[2 * (int64_t)j + 1];
      double r = sqrt(dx * dx + dy * dy);
      raw += (r - d) * (r - d) / (d * d);
      s1 += r / d;
      s2 += r * r / (d * d);
      np += 1.0;
    }
  }
  free(dist); free(srcs); free(tgts);
  if (rc != ORC_OK) return rc;
  double pairs = 0.5 * (double)n * (double)(n - 1);
  double f = S > 0 ? pairs / np : 1.0;
  if (sums) { sums[0] = raw; sums[1] = s1; sums[2] = s2; sums[3] = np; }
  out[0] = raw * f;
  out[1] = s2 > 0.0 ? s1 / s2 : 0.0;
  out[2] = (s2 > 0.0 ? np - s1 * s1 / s2 : np) * f;
  out[3] = out[2] / pairs;
  return ORC_OK;
}
