// Many small graphs prepared in two launches: Algorithm 1 lines 1-4 (graph,
// max/min pivots, d_ip, regions and counts, PivotMDS and the rescale) for a
// whole batch of independent layouts, feeding ssm_batch_iterate.
//
// One block owns one graph at a time (graphs handed out largest first from
// an atomic counter).  k_prep_pivots builds the graph's CSR in shared memory
// (degrees, scatter, rows sorted and deduplicated by one thread each), then
// runs the k breadth-first searches of max/min sp level by level in shared
// memory (distances and the running minimum as uint16, a visited bitmap,
// two frontier queues); each search's distance row is the pivot's d_ip row.
// Regions, the per-pivot eccentricities and the count-table length close
// the first launch; the host reads the lengths once for the whole batch and
// places the tables.  k_prep_layout then fills the cumulative counts, forms
// the exact integer Gram matrix Delta^T Delta of the squared distances
// (128-bit sums over 32-node chunks staged in shared memory), the FP64
// matrix B = 1/4 J (G - s s^T / n) J, its eigenpairs by a parallel cyclic
// Jacobi method (round-robin pairs, k/2 disjoint rotations per step, A and
// the eigenvectors in shared memory), projects, signs and rescales the
// layout.  Every reduction has a fixed order: results do not depend on
// timing.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace ssm {

constexpr int kPrepMaxN = 12288;
constexpr int kPrepMaxK = 100;
constexpr int kPrepThreads = 512;
constexpr int kPrepChunk = 32;     // nodes per staged chunk of the Gram

struct PrepDev {
  int32_t n, k;
  int64_t m_in, edge_off;
  int64_t node_off, row_off, col_off, piv_off, dip_off, cnt_off_off;
};

struct PrepArgs {
  int32_t G, nmax;
  const PrepDev *desc;
  const int32_t *order;
  const int32_t *src, *dst;
  int32_t *tmp;  // scatter area, capacity 2 m_in per graph at col_off
  int32_t *rowptr, *colidx, *pivots, *region;
  uint16_t *dip;
  int32_t *ecc;        // [sum k]
  int64_t *lens;       // [G] count-table lengths
  int64_t *medges;     // [G] edges after deduplication
  int32_t *pairq;      // per block: two queues of pair_cap (pivot, node) pairs
  int64_t pair_cap;
  int64_t ubytes;      // the shared region of the three phases
  unsigned *ctr;
  int32_t *status;
};

// exclusive block scan of a[0..len) in place (len <= 3 * kPrepMaxN), total returned
__device__ int block_exclusive_scan(int *a, int len, int *s_part) {
  const int per = (len + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per, e = min(len, b + per);
  int t = 0;
  for (int i = b; i < e; ++i) t += a[i];
  s_part[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < (int)blockDim.x; ++w) {
      const int v = s_part[w];
      s_part[w] = acc;
      acc += v;
    }
    s_part[blockDim.x] = acc;
  }
  __syncthreads();
  int acc = s_part[threadIdx.x];
  for (int i = b; i < e; ++i) {
    const int v = a[i];
    a[i] = acc;
    acc += v;
  }
  __syncthreads();
  const int total = s_part[blockDim.x];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kPrepThreads) k_prep_pivots(PrepArgs A) {
  extern __shared__ __align__(16) unsigned char psm[];
  const int NM = A.nmax;
  // one region serves the three phases in turn: the CSR build (degrees and
  // offsets), max/min (running minimum and two queues) and the lockstep
  // searches (a visited bit per (pivot, node) pair)
  int *deg = reinterpret_cast<int *>(psm);  // [NM + 1]
  int *off = deg + (NM + 1);                // [NM + 1]
  int *s_part = reinterpret_cast<int *>(psm + A.ubytes);  // [kPrepThreads + 1]
  int *s_ecc = s_part + kPrepThreads + 1;                  // [kPrepMaxK]
  __shared__ int s_task, s_next, s_piv[kPrepMaxK];
  __shared__ unsigned s_key;
  for (;;) {
    if (threadIdx.x == 0) s_task = (int)atomicAdd(A.ctr, 1u);
    __syncthreads();
    const int task = s_task;
    __syncthreads();
    if (task >= A.G) break;
    const int gi = A.order[task];
    const PrepDev D = A.desc[gi];
    const int n = D.n, k = D.k;
    const int32_t *src = A.src + D.edge_off, *dst = A.dst + D.edge_off;
    int32_t *tmp = A.tmp + D.col_off;
    int32_t *rowptr = A.rowptr + D.row_off;
    int32_t *colidx = A.colidx + D.col_off;
    // ---- CSR: degrees, scatter, rows sorted and deduplicated
    for (int i = threadIdx.x; i <= n; i += blockDim.x) deg[i] = 0;
    __syncthreads();
    for (int64_t e = threadIdx.x; e < D.m_in; e += blockDim.x) {
      const int u = src[e], v = dst[e];
      if (u < 0 || u >= n || v < 0 || v >= n) {
        dev_fail(A.status, SSM_E_GRAPH);
        continue;
      }
      if (u == v) continue;
      atomicAdd(deg + u, 1);
      atomicAdd(deg + v, 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= n; i += blockDim.x) off[i] = deg[i];
    __syncthreads();
    block_exclusive_scan(off, n + 1, s_part);
    for (int i = threadIdx.x; i <= n; i += blockDim.x) deg[i] = 0;  // cursors
    __syncthreads();
    for (int64_t e = threadIdx.x; e < D.m_in; e += blockDim.x) {
      const int u = src[e], v = dst[e];
      if (u < 0 || u >= n || v < 0 || v >= n || u == v) continue;
      tmp[off[u] + atomicAdd(deg + u, 1)] = v;
      tmp[off[v] + atomicAdd(deg + v, 1)] = u;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      int *row = tmp + off[i];
      const int len = off[i + 1] - off[i];
      for (int a = 1; a < len; ++a) {  // insertion sort (rows of these graphs are short)
        const int x = row[a];
        int b = a - 1;
        while (b >= 0 && row[b] > x) {
          row[b + 1] = row[b];
          --b;
        }
        row[b + 1] = x;
      }
      int u = 0;
      for (int a = 0; a < len; ++a) u += (a == 0 || row[a] != row[a - 1]) ? 1 : 0;
      deg[i] = u;
    }
    __syncthreads();
    const int m2 = block_exclusive_scan(deg, n + 1, s_part);
    for (int i = threadIdx.x; i <= n; i += blockDim.x) rowptr[i] = deg[i];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int *row = tmp + off[i];
      const int len = off[i + 1] - off[i];
      int o = deg[i];
      for (int a = 0; a < len; ++a)
        if (a == 0 || row[a] != row[a - 1]) colidx[o++] = row[a];
    }
    if (threadIdx.x == 0) A.medges[gi] = m2 / 2;
    __syncthreads();
    // ---- max/min sp (start node 0): each search lowers the running minimum
    // mind in place and only continues from nodes the new pivot is strictly
    // closer to (mind is 1-Lipschitz along edges, so nothing beyond them
    // can change); the first search reaches everything
    int *mindi = deg;                                       // [NM] (the CSR arrays are free now)
    uint16_t *qa = reinterpret_cast<uint16_t *>(off);       // [NM]
    uint16_t *qb = qa + NM;                                 // [NM]
    for (int i = threadIdx.x; i < n; i += blockDim.x) mindi[i] = 0x7FFFFFFF;
    __syncthreads();
    for (int a = 0; a < k; ++a) {
      int p = 0;
      if (a > 0) {
        if (threadIdx.x == 0) s_key = 0u;
        __syncthreads();
        unsigned best = 0u;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          const unsigned key = ((unsigned)mindi[i] << 16) | (0xFFFFu - (unsigned)i);
          best = key > best ? key : best;
        }
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&s_key, best);
        __syncthreads();
        p = (int)(0xFFFFu - (s_key & 0xFFFFu));
      }
      if (threadIdx.x == 0) {
        A.pivots[D.piv_off + a] = p;
        s_piv[a] = p;
        mindi[p] = 0;
        qa[0] = (uint16_t)p;
      }
      __syncthreads();
      int ncur = 1;
      uint16_t *qc = qa, *qn = qb;
      for (int level = 0; ncur > 0; ++level) {
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
        for (int t = threadIdx.x; t < ncur; t += blockDim.x) {
          const int v = qc[t];
          for (int j = rowptr[v]; j < rowptr[v + 1]; ++j) {
            const int u = colidx[j];
            if (atomicMin(mindi + u, level + 1) > level + 1) qn[atomicAdd(&s_next, 1)] = (uint16_t)u;
          }
        }
        __syncthreads();
        ncur = s_next;
        uint16_t *t_ = qc;
        qc = qn;
        qn = t_;
        __syncthreads();
      }
      if (a == 0)
        for (int i = threadIdx.x; i < n; i += blockDim.x)
          if (mindi[i] == 0x7FFFFFFF) dev_fail(A.status, SSM_E_DISCONNECTED);
      __syncthreads();
    }
    // ---- d_ip: the k searches in lockstep, one level for all pivots at a
    // time; (pivot, node) pairs in global queues, one visited bit per pair
    // in shared memory
    {
      unsigned *visk = reinterpret_cast<unsigned *>(psm);  // [(k n + 31) / 32], over the free CSR arrays
      int32_t *pq0 = A.pairq + (int64_t)blockIdx.x * 2 * A.pair_cap, *pq1 = pq0 + A.pair_cap;
      uint16_t *dipg = A.dip + D.dip_off;
      const int words = (k * n + 31) / 32;
      __syncthreads();
      for (int w = threadIdx.x; w < words; w += blockDim.x) visk[w] = 0u;
      __syncthreads();
      for (int a = threadIdx.x; a < k; a += blockDim.x) {
        const int p = s_piv[a];
        const int bit = a * n + p;
        atomicOr(visk + (bit >> 5), 1u << (bit & 31));
        dipg[(int64_t)a * n + p] = 0;
        pq0[a] = (a << 14) | p;
      }
      __syncthreads();
      int ncur = k;
      int32_t *qc = pq0, *qn = pq1;
      for (int level = 0; ncur > 0; ++level) {
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
        for (int t = threadIdx.x; t < ncur; t += blockDim.x) {
          const int pr = qc[t];
          const int a = pr >> 14, v = pr & 0x3FFF;
          for (int j = rowptr[v]; j < rowptr[v + 1]; ++j) {
            const int u = colidx[j];
            const int bit = a * n + u;
            const unsigned m = 1u << (bit & 31);
            if (!(atomicOr(visk + (bit >> 5), m) & m)) {
              dipg[(int64_t)a * n + u] = (uint16_t)(level + 1);
              qn[atomicAdd(&s_next, 1)] = (a << 14) | u;
            }
          }
        }
        __syncthreads();
        ncur = s_next;
        int32_t *t_ = qc;
        qc = qn;
        qn = t_;
        __syncthreads();
      }
    }
    // ---- regions (ties to the lowest pivot index) and eccentricities
    for (int a = threadIdx.x; a < k; a += blockDim.x) s_ecc[a] = 0;
    __syncthreads();
    const uint16_t *dip = A.dip + D.dip_off;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      int best = 0;
      unsigned bd = dip[i];
      for (int a = 1; a < k; ++a) {
        const unsigned d = dip[(int64_t)a * n + i];
        if (d < bd) {
          bd = d;
          best = a;
        }
      }
      A.region[D.node_off + i] = best;
      atomicMax(s_ecc + best, (int)bd);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t len = 0;
      for (int a = 0; a < k; ++a) {
        A.ecc[D.piv_off + a] = s_ecc[a];
        len += s_ecc[a] + 1;
      }
      A.lens[gi] = len;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ layout
struct LayoutDev {
  int32_t n, k;
  int64_t m;
  int64_t node_off, row_off, col_off, piv_off, dip_off, cnt_off_off, cnt_base;
};

struct LayoutArgs {
  int32_t G;
  const LayoutDev *desc;
  const int32_t *order;
  const int32_t *rowptr, *colidx, *region, *ecc;
  const uint16_t *dip;
  int32_t *cnt_off;
  uint32_t *cnt;
  float2 *pos;
  double *eig;  // [2 G] or null
  unsigned *ctr;
  int32_t *status;
};

// fixed-order block sum of one double per thread
__device__ double block_sum_d(double v, double *s_red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kPrepThreads) k_prep_layout(LayoutArgs L) {
  extern __shared__ __align__(16) unsigned char lsm[];
  double *Am = reinterpret_cast<double *>(lsm);              // [kPrepMaxK^2]
  double *V = Am + kPrepMaxK * kPrepMaxK;                     // [kPrepMaxK^2]
  uint32_t *chunk = reinterpret_cast<uint32_t *>(V + kPrepMaxK * kPrepMaxK);  // [kPrepChunk][kPrepMaxK]
  __shared__ double s_red[kPrepThreads / 32];
  __shared__ unsigned long long s_col[kPrepMaxK];
  __shared__ double s_rm[kPrepMaxK], s_v[2][kPrepMaxK];
  __shared__ int s_off[kPrepMaxK + 1];
  __shared__ double s_dg[kPrepMaxK], s_e[kPrepMaxK], s_p[kPrepMaxK], s_w[kPrepMaxK], s_lam[2];
  __shared__ double s_y[2][kPrepMaxK], s_fd[2][kPrepMaxK], s_fu[2][kPrepMaxK], s_fu2[2][kPrepMaxK], s_fl[2][kPrepMaxK];
  __shared__ double s_e2[kPrepMaxK];
  __shared__ int s_piv[2][kPrepMaxK];
  __shared__ int s_task, s_big[2];
  __shared__ double s_sig[2], s_kap[2];
  __shared__ int s_done;
  for (;;) {
    if (threadIdx.x == 0) s_task = (int)atomicAdd(L.ctr, 1u);
    __syncthreads();
    const int task = s_task;
    __syncthreads();
    if (task >= L.G) break;
    const int gi = L.order[task];
    const LayoutDev D = L.desc[gi];
    const int n = D.n, k = D.k;
    const uint16_t *dip = L.dip + D.dip_off;
    const int32_t *region = L.region + D.node_off;
    const int32_t *ecc = L.ecc + D.piv_off;
    // ---- Section 3's counts: cnt_off, histograms, prefix sums
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int a = 0; a < k; ++a) {
        s_off[a] = acc;
        acc += ecc[a] + 1;
      }
      s_off[k] = acc;
    }
    __syncthreads();
    uint32_t *cnt = L.cnt + D.cnt_base;
    for (int a = threadIdx.x; a <= k; a += blockDim.x) L.cnt_off[D.cnt_off_off + a] = s_off[a];
    for (int t = threadIdx.x; t < s_off[k]; t += blockDim.x) cnt[t] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int a = region[i];
      atomicAdd(cnt + s_off[a] + dip[(int64_t)a * n + i], 1u);
    }
    __syncthreads();
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
      uint32_t acc = 0;
      for (int t = s_off[a]; t < s_off[a + 1]; ++t) {
        acc += cnt[t];
        cnt[t] = acc;
      }
    }
    // ---- exact Gram G = Delta^T Delta (upper triangle, 128-bit) and s_a
    const int npairs = k * (k + 1) / 2;
    constexpr int kPairsPerThread = (kPrepMaxK * (kPrepMaxK + 1) / 2 + kPrepThreads - 1) / kPrepThreads;
    unsigned __int128 acc[kPairsPerThread];
    int pa[kPairsPerThread], pb[kPairsPerThread];
#pragma unroll
    for (int j = 0; j < kPairsPerThread; ++j) {
      acc[j] = 0;
      int p = threadIdx.x + j * blockDim.x;
      int a = 0;
      if (p < npairs) {
        while (p >= k - a) {
          p -= k - a;
          ++a;
        }
        pa[j] = a;
        pb[j] = a + p;
      } else {
        pa[j] = -1;
        pb[j] = -1;
      }
    }
    unsigned long long colsum = 0;
    for (int i0 = 0; i0 < n; i0 += kPrepChunk) {
      __syncthreads();
      for (int e = threadIdx.x; e < kPrepChunk * k; e += blockDim.x) {
        const int a = e / kPrepChunk, t = e % kPrepChunk;
        const int i = i0 + t;
        const uint32_t d = i < n ? dip[(int64_t)a * n + i] : 0u;
        chunk[t * kPrepMaxK + a] = d * d;
      }
      __syncthreads();
      if (threadIdx.x < k)
        for (int t = 0; t < kPrepChunk; ++t) colsum += chunk[t * kPrepMaxK + threadIdx.x];
#pragma unroll
      for (int j = 0; j < kPairsPerThread; ++j) {
        if (pa[j] < 0) continue;
        const int a = pa[j], b = pb[j];
        // a chunk's 32 products (each below 2^52) sum exactly in 64 bits;
        // the chunk sums go into the 128-bit total
        unsigned long long cs = 0;
        for (int t = 0; t < kPrepChunk; ++t)
          cs += (unsigned long long)chunk[t * kPrepMaxK + a] * (unsigned long long)chunk[t * kPrepMaxK + b];
        acc[j] += cs;
      }
    }
    if (threadIdx.x < k) s_col[threadIdx.x] = colsum;
    __syncthreads();
    // B = G - s s^T / n, then 1/4 J B J
    const double inv_n = 1.0 / (double)n;
    const double two64 = 18446744073709551616.0;
#pragma unroll
    for (int j = 0; j < kPairsPerThread; ++j) {
      if (pa[j] < 0) continue;
      const int a = pa[j], b = pb[j];
      const double g = (double)(unsigned long long)(acc[j] >> 64) * two64 + (double)(unsigned long long)acc[j];
      const double v = g - ((double)s_col[a] * (double)s_col[b]) * inv_n;
      Am[a * kPrepMaxK + b] = v;
      Am[b * kPrepMaxK + a] = v;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
      double r = 0.0;
      for (int b = 0; b < k; ++b) r += Am[a * kPrepMaxK + b];
      s_rm[a] = r / (double)k;
    }
    __syncthreads();
    double gm = 0.0;
    for (int a = 0; a < k; ++a) gm += s_rm[a];
    gm /= (double)k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int a = e / k, b = e % k;
      Am[a * kPrepMaxK + b] = 0.25 * (Am[a * kPrepMaxK + b] - s_rm[a] - s_rm[b] + gm);
      V[a * kPrepMaxK + b] = a == b ? 1.0 : 0.0;
    }
    __syncthreads();
    // ---- top-2 eigenpairs: Householder reduction of B to a tridiagonal T
    // (Q^T B Q = T, reflector vectors kept in V), the two largest
    // eigenvalues of T by Sturm-count bisection, their eigenvectors by
    // inverse iteration on T, and back through the reflectors
    double *Hv = V;  // row j: the unit reflector of step j (entries j+1 .. k-1)
    for (int j = 0; j + 2 < k; ++j) {
      // warp 0: the reflector of column j (norm by shuffles)
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double sig = 0.0;
        for (int r = j + 2 + lane; r < k; r += 32) sig += Am[r * kPrepMaxK + j] * Am[r * kPrepMaxK + j];
        for (int o = 16; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
        const double x0 = Am[(j + 1) * kPrepMaxK + j];
        if (sig == 0.0) {  // the column is already tridiagonal: H = I
          for (int r = lane; r < k; r += 32) Hv[j * kPrepMaxK + r] = 0.0;
          if (lane == 0) s_e[j] = x0;
        } else {
          const double nrm = sqrt(x0 * x0 + sig);
          const double alpha = x0 >= 0.0 ? -nrm : nrm;
          const double v0 = x0 - alpha;
          const double vinv = 1.0 / sqrt(v0 * v0 + sig);
          for (int r = lane; r < k; r += 32)
            Hv[j * kPrepMaxK + r] = r <= j ? 0.0 : (r == j + 1 ? v0 : Am[r * kPrepMaxK + j]) * vinv;
          if (lane == 0) s_e[j] = alpha;
        }
      }
      __syncthreads();
      const double *hv = Hv + j * kPrepMaxK;
      if (hv[j + 1] == 0.0) continue;  // H = I (the same decision in every thread)
      // p = A v over the trailing block (read down the columns: A is
      // symmetric and consecutive threads then touch consecutive words)
      for (int r = j + 1 + threadIdx.x; r < k; r += blockDim.x) {
        double t = 0.0;
        for (int c = j + 1; c < k; ++c) t += Am[c * kPrepMaxK + r] * hv[c];
        s_p[r] = t;
      }
      __syncthreads();
      // warp 0: K = v . p, w = 2 (p - K v)
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double kk = 0.0;
        for (int r = j + 1 + lane; r < k; r += 32) kk += hv[r] * s_p[r];
        for (int o = 16; o > 0; o >>= 1) kk += __shfl_xor_sync(0xffffffffu, kk, o);
        for (int r = j + 1 + lane; r < k; r += 32) s_w[r] = 2.0 * (s_p[r] - kk * hv[r]);
      }
      __syncthreads();
      const int L = k - j - 1;
      for (int e2 = threadIdx.x; e2 < L * L; e2 += blockDim.x) {
        const int r = j + 1 + e2 / L, c = j + 1 + e2 % L;
        Am[r * kPrepMaxK + c] -= hv[r] * s_w[c] + s_w[r] * hv[c];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      for (int a = 0; a < k; ++a) s_dg[a] = Am[a * kPrepMaxK + a];
      if (k >= 2) s_e[k - 2] = Am[(k - 1) * kPrepMaxK + (k - 2)];
    }
    __syncthreads();
    // eigenvalues number k-1 and k-2 (ascending) by bisection on Sturm counts,
    // 32 points per step evaluated by the lanes of warp 0 (the largest) and
    // warp 1 (the second); each step of the count's recurrence takes 1/q from
    // an FP32 reciprocal and one Newton step in FP64 (relative error near
    // 2^-46: only the signs of the q are used, and GB300's FP64 division is
    // the slow part of this loop)
    for (int a = threadIdx.x; a + 1 < k; a += blockDim.x) s_e2[a] = s_e[a] * s_e[a];
    __syncthreads();
    if (threadIdx.x < 64) {
      const int lane = threadIdx.x & 31, want = threadIdx.x >> 5;
      double lo = 0.0, hi = 0.0;
      for (int a = 0; a < k; ++a) {
        const double r = (a > 0 ? fabs(s_e[a - 1]) : 0.0) + (a + 1 < k ? fabs(s_e[a]) : 0.0);
        lo = a == 0 ? s_dg[a] - r : fmin(lo, s_dg[a] - r);
        hi = a == 0 ? s_dg[a] + r : fmax(hi, s_dg[a] + r);
      }
      const int idx = k - 1 - want;  // ascending index of the eigenvalue
      double a0 = lo - 1e-12 * (fabs(lo) + fabs(hi)), b0 = hi + 1e-12 * (fabs(lo) + fabs(hi));
      for (int it = 0; it < 40 && b0 - a0 > 4e-16 * fmax(fabs(a0), fabs(b0)); ++it) {
        const double x = a0 + (b0 - a0) * (double)(lane + 1) / 33.0;
        int cnt = 0;  // eigenvalues below x
        double q = s_dg[0] - x;
        cnt += q < 0.0;
        for (int a = 1; a < k; ++a) {
          double r;
          const double aq = fabs(q);
          if (aq > 1e-30 && aq < 1e30) {
            const double r0 = (double)__frcp_rn((float)q);
            r = r0 * fma(-q, r0, 2.0);
          } else {
            r = 1.0 / (q == 0.0 ? 1e-300 : q);
          }
          q = fma(-s_e2[a - 1], r, s_dg[a] - x);
          cnt += q < 0.0;
        }
        // the smallest lane point with more than idx eigenvalues below it
        const unsigned above = __ballot_sync(0xffffffffu, cnt > idx);
        const int first = above ? __ffs(above) - 1 : 32;
        const double nb = first < 32 ? a0 + (b0 - a0) * (double)(first + 1) / 33.0 : b0;
        const double na = first > 0 ? a0 + (b0 - a0) * (double)first / 33.0 : a0;
        a0 = na;
        b0 = nb;
      }
      if (lane == 0) s_lam[want] = 0.5 * (a0 + b0);
    }
    __syncthreads();
    // inverse iteration on T - lambda I (tridiagonal LU with partial
    // pivoting, factored once, two solves), one thread per eigenvalue; the
    // second vector is then made orthogonal to the first
    if (threadIdx.x == 0 || threadIdx.x == 32) {
      const int want = threadIdx.x >> 5;
      double *y = s_y[want];
      double *dd = s_fd[want], *du = s_fu[want], *du2 = s_fu2[want], *dl = s_fl[want];
      int *piv = s_piv[want];
      const double lam = s_lam[want];
      const double pert = 1e-14 * (fabs(lam) + 1e-300);
      for (int a = 0; a < k; ++a) {
        y[a] = 1.0 + 0.01 * (double)((a * 37) % 11);
        dd[a] = s_dg[a] - lam;
        du[a] = a + 1 < k ? s_e[a] : 0.0;
        dl[a] = a + 1 < k ? s_e[a] : 0.0;
        du2[a] = 0.0;
      }
      for (int a = 0; a + 1 < k; ++a) {
        if (fabs(dd[a]) >= fabs(dl[a])) {
          if (dd[a] == 0.0) dd[a] = pert;
          const double f = dl[a] / dd[a];
          dl[a] = f;
          dd[a + 1] -= f * du[a];
          piv[a] = 0;
        } else {
          const double f = dd[a] / dl[a];
          dd[a] = dl[a];
          dl[a] = f;
          const double t = du[a];
          du[a] = dd[a + 1];
          dd[a + 1] = t - f * dd[a + 1];
          if (a + 2 < k) {
            du2[a] = du[a + 1];
            du[a + 1] = -f * du[a + 1];
          }
          piv[a] = 1;
        }
      }
      if (dd[k - 1] == 0.0) dd[k - 1] = pert;
      for (int a = 0; a < k; ++a) dd[a] = 1.0 / dd[a];  // reciprocals for the solves
      for (int it = 0; it < 2; ++it) {
        for (int a = 0; a + 1 < k; ++a) {
          if (piv[a] == 0) {
            y[a + 1] -= dl[a] * y[a];
          } else {
            const double t = y[a];
            y[a] = y[a + 1];
            y[a + 1] = t - dl[a] * y[a];
          }
        }
        y[k - 1] *= dd[k - 1];
        if (k >= 2) y[k - 2] = (y[k - 2] - du[k - 2] * y[k - 1]) * dd[k - 2];
        for (int a = k - 3; a >= 0; --a) y[a] = (y[a] - du[a] * y[a + 1] - du2[a] * y[a + 2]) * dd[a];
        double nr = 0.0;
        for (int a = 0; a < k; ++a) nr += y[a] * y[a];
        nr = nr > 0.0 ? 1.0 / sqrt(nr) : 0.0;
        for (int a = 0; a < k; ++a) y[a] *= nr;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double dt = 0.0;
      for (int a = 0; a < k; ++a) dt += s_y[1][a] * s_y[0][a];
      double nr = 0.0;
      for (int a = 0; a < k; ++a) {
        s_y[1][a] -= dt * s_y[0][a];
        nr += s_y[1][a] * s_y[1][a];
      }
      nr = nr > 0.0 ? 1.0 / sqrt(nr) : 0.0;
      for (int a = 0; a < k; ++a) s_y[1][a] *= nr;
      s_done = s_lam[0] > 0.0;
      if (L.eig) {
        L.eig[2 * gi] = s_lam[0];
        L.eig[2 * gi + 1] = s_lam[1];
      }
    }
    __syncthreads();
    // z = H_0 H_1 ... H_{k-3} y, the reflectors applied last to first (one
    // warp: k <= 100 entries, dot products by shuffles, no block barrier)
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int j = k - 3; j >= 0; --j) {
        const double *hv = Hv + j * kPrepMaxK;
        double d0 = 0.0, d1 = 0.0;
        for (int r = j + 1 + lane; r < k; r += 32) {
          d0 += hv[r] * s_y[0][r];
          d1 += hv[r] * s_y[1][r];
        }
        for (int o = 16; o > 0; o >>= 1) {
          d0 += __shfl_xor_sync(0xffffffffu, d0, o);
          d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        }
        for (int r = j + 1 + lane; r < k; r += 32) {
          s_y[0][r] -= 2.0 * d0 * hv[r];
          s_y[1][r] -= 2.0 * d1 * hv[r];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (!s_done) dev_fail(L.status, SSM_E_NUMERIC);
    // each vector signed so that its largest-magnitude entry (lowest index on a tie) is positive
    if (threadIdx.x == 0)
      for (int r = 0; r < 2; ++r) {
        int big = 0;
        for (int a = 1; a < k; ++a)
          if (fabs(s_y[r][a]) > fabs(s_y[r][big])) big = a;
        s_big[r] = big;
      }
    __syncthreads();
    for (int a = threadIdx.x; a < k; a += blockDim.x)
      for (int r = 0; r < 2; ++r) s_v[r][a] = (s_y[r][s_big[r]] < 0 ? -1.0 : 1.0) * s_y[r][a];
    __syncthreads();
    if (threadIdx.x == 0) {
      double sg0 = 0.0, sg1 = 0.0, cv0 = 0.0, cv1 = 0.0, cb = 0.0;
      for (int a = 0; a < k; ++a) {
        const double cbar = (double)s_col[a] * inv_n;
        sg0 += s_v[0][a];
        sg1 += s_v[1][a];
        cv0 += cbar * s_v[0][a];
        cv1 += cbar * s_v[1][a];
        cb += cbar;
      }
      const double gbar = cb / (double)k;
      s_sig[0] = sg0;
      s_sig[1] = sg1;
      s_kap[0] = cv0 - gbar * sg0;
      s_kap[1] = cv1 - gbar * sg1;
    }
    __syncthreads();
    // ---- x_i = -1/2 (sum_a d_ia^2 v_a - rbar_i sigma - kappa), FP64
    float2 *pos = L.pos + D.node_off;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double x = 0.0, y = 0.0, rs = 0.0;
      for (int a = 0; a < k; ++a) {
        const double d = (double)dip[(int64_t)a * n + i];
        const double dd = d * d;
        rs += dd;
        x += dd * s_v[0][a];
        y += dd * s_v[1][a];
      }
      const double rbar = rs / (double)k;
      pos[i] = make_float2((float)(-0.5 * (x - rbar * s_sig[0] - s_kap[0])),
                           (float)(-0.5 * (y - rbar * s_sig[1] - s_kap[1])));
    }
    __syncthreads();
    // ---- rescale: sum_E ||x_i - x_j|| = m (lengths from the FP32 positions)
    const int32_t *rowptr = L.rowptr + D.row_off;
    const int32_t *colidx = L.colidx + D.col_off;
    double len = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float2 xi = pos[i];
      for (int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
        const int j = colidx[t];
        if (j <= i) continue;
        const float2 xj = pos[j];
        const float dx = xi.x - xj.x, dy = xi.y - xj.y;
        len += (double)sqrtf(dx * dx + dy * dy);
      }
    }
    len = block_sum_d(len, s_red);
    const bool okl = len > 0.0 && isfinite(len);
    if (!okl && threadIdx.x == 0) dev_fail(L.status, SSM_E_NUMERIC);
    const double sc = okl ? (double)D.m / len : 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float2 x = pos[i];
      pos[i] = make_float2((float)((double)x.x * sc), (float)((double)x.y * sc));
    }
    __syncthreads();
  }
}

// the workspace of both calls: descriptors, order, counter and lengths
// first (the layout call uses only this prefix), then the scatter area
struct PrepWs {
  PrepDev *pd;
  LayoutDev *ld;
  int32_t *order;
  unsigned *ctr;
  int64_t *lens;  // [2 G]: table lengths, then edge counts
  int32_t *tmp;
  int32_t *pairq;
};

static int prep_blocks(int32_t G) { return std::max(1, std::min(G, num_sms() * 4)); }

// cap < 0: the prefix only (what the layout call uses)
static void carve_prep(Carver &c, PrepWs &w, int32_t G, int64_t cap, int64_t kn_max) {
  w.pd = c.take<PrepDev>((size_t)G);
  w.ld = c.take<LayoutDev>((size_t)G);
  w.order = c.take<int32_t>((size_t)G);
  w.ctr = c.take<unsigned>(2);
  w.lens = c.take<int64_t>(2 * (size_t)G);
  w.tmp = cap >= 0 ? c.take<int32_t>((size_t)std::max<int64_t>(cap, 1)) : nullptr;
  w.pairq = cap >= 0 ? c.take<int32_t>((size_t)prep_blocks(G) * 2 * (size_t)std::max<int64_t>(kn_max, 1)) : nullptr;
}

// the shared region: CSR arrays 2 (nmax + 1) ints, or the visited bits of
// the lockstep searches, whichever is larger; then the scan and eccentricity
// scratch
static int64_t prep_region(int nmax, int64_t kn_max) {
  const int64_t csr = 2 * ((int64_t)nmax + 1) * (int64_t)sizeof(int);
  const int64_t bits = (kn_max + 31) / 32 * (int64_t)sizeof(unsigned);
  return (std::max(csr, bits) + 15) / 16 * 16;
}

static size_t prep_smem(int nmax, int64_t kn_max) {
  return (size_t)prep_region(nmax, kn_max) + (kPrepThreads + 1 + kPrepMaxK) * sizeof(int) + 16;
}

static size_t layout_smem() {
  return 2 * (size_t)kPrepMaxK * kPrepMaxK * sizeof(double) + (size_t)kPrepChunk * kPrepMaxK * sizeof(uint32_t);
}

}  // namespace ssm

// =========================================================== C ABI
SSM_API size_t ssm_batch_prepare_workspace(int32_t G, const ssm_batch_input *in) {
  if (G < 1 || !in) return 0;
  int64_t cap = 0, kn = 1;
  for (int32_t g = 0; g < G; ++g) {
    cap += 2 * std::max<int64_t>(0, in[g].m_in);
    kn = std::max<int64_t>(kn, (int64_t)std::max(in[g].k, 0) * std::max(in[g].n, 0));
  }
  ssm::Carver c(nullptr, 0);
  ssm::PrepWs w;
  ssm::carve_prep(c, w, G, cap, kn);
  return c.size();
}

SSM_API int ssm_batch_pivots(int32_t G, const ssm_batch_input *in, const int32_t *src, const int32_t *dst,
                             ssm_batch_graph *out, int32_t *rowptr, int32_t *colidx, int32_t *pivots, uint16_t *dip,
                             int32_t *region, int32_t *ecc, int64_t *m_out, int32_t *status, void *ws,
                             size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (G < 1 || !in || !out || !rowptr || !colidx || !pivots || !dip || !region || !ecc || !status || !ws)
    return fail(SSM_E_ARG, "ssm_batch_pivots: null pointer or G < 1");
  std::vector<PrepDev> pd((size_t)G);
  std::vector<int32_t> order((size_t)G);
  int64_t node = 0, row = 0, col = 0, piv = 0, dipo = 0, offo = 0, edges = 0, kn_max = 1;
  int nmax = 1;
  for (int32_t g = 0; g < G; ++g) {
    const ssm_batch_input &x = in[g];
    if (x.n < 1 || x.n > kPrepMaxN) return fail(SSM_E_ARG, "ssm_batch_pivots: graph %d has n = %d (1..%d)", g, x.n, kPrepMaxN);
    if (x.k < 2 || x.k > x.n || x.k > kPrepMaxK)
      return fail(SSM_E_ARG, "ssm_batch_pivots: graph %d has k = %d (2..min(n, %d))", g, x.k, kPrepMaxK);
    if (x.m_in < 0 || 2 * x.m_in >= ((int64_t)1 << 31)) return fail(SSM_E_ARG, "ssm_batch_pivots: graph %d edge count", g);
    if (x.m_in > 0 && (!src || !dst)) return fail(SSM_E_ARG, "ssm_batch_pivots: null edge arrays");
    PrepDev &d = pd[(size_t)g];
    d.n = x.n; d.k = x.k; d.m_in = x.m_in; d.edge_off = x.edge_off;
    d.node_off = node; d.row_off = row; d.col_off = col; d.piv_off = piv; d.dip_off = dipo; d.cnt_off_off = offo;
    ssm_batch_graph &o = out[g];
    o.n = x.n; o.k = x.k; o.cnt_len = 0; o.reserved = 0;
    o.node_off = node; o.row_off = row; o.col_off = col; o.piv_off = piv; o.dip_off = dipo; o.cnt_off_off = offo;
    o.cnt_base = 0;
    node += x.n; row += x.n + 1; col += 2 * x.m_in; piv += x.k; dipo += (int64_t)x.k * x.n; offo += x.k + 1;
    edges = std::max(edges, x.edge_off + x.m_in);
    nmax = std::max(nmax, x.n);
    kn_max = std::max<int64_t>(kn_max, (int64_t)x.k * x.n);
    order[(size_t)g] = g;
  }
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return (int64_t)pd[(size_t)a].n * pd[(size_t)a].k > (int64_t)pd[(size_t)b].n * pd[(size_t)b].k;
  });
  Carver c(ws, ws_bytes);
  PrepWs w;
  carve_prep(c, w, G, col, kn_max);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_batch_pivots: workspace %zu bytes, need %zu", ws_bytes, c.size());
  SSM_TRY_CUDA(cudaMemcpyAsync(w.pd, pd.data(), pd.size() * sizeof(PrepDev), cudaMemcpyHostToDevice, s));
  SSM_TRY_CUDA(cudaMemcpyAsync(w.order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  SSM_TRY_CUDA(cudaMemsetAsync(w.ctr, 0, 2 * sizeof(unsigned), s));
  PrepArgs A;
  A.G = G; A.nmax = nmax; A.desc = w.pd; A.order = w.order; A.src = src; A.dst = dst; A.tmp = w.tmp;
  A.rowptr = rowptr; A.colidx = colidx; A.pivots = pivots; A.region = region; A.dip = dip; A.ecc = ecc;
  A.lens = w.lens; A.medges = w.lens + G; A.ctr = w.ctr; A.status = status;
  A.pairq = w.pairq; A.pair_cap = kn_max; A.ubytes = prep_region(nmax, kn_max);
  const size_t smem = prep_smem(nmax, kn_max);
  SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_prep_pivots));
  int per_sm = 0;
  SSM_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prep_pivots, kPrepThreads, smem));
  if (per_sm < 1) return fail(SSM_E_ARG, "ssm_batch_pivots: %zu bytes of shared memory do not fit", smem);
  const int blocks = std::max(1, std::min(prep_blocks(G), per_sm * num_sms()));
  note_launch(), k_prep_pivots<<<blocks, kPrepThreads, smem, s>>>(A);
  SSM_TRY_CUDA(cudaGetLastError());
  std::vector<int64_t> h(2 * (size_t)G);
  int32_t hst = 0;
  SSM_TRY_CUDA(cudaMemcpyAsync(h.data(), w.lens, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SSM_TRY_CUDA(cudaMemcpyAsync(&hst, status, sizeof hst, cudaMemcpyDeviceToHost, s));
  SSM_TRY_CUDA(cudaStreamSynchronize(s));
  if (hst) return fail(hst, "ssm_batch_pivots: %s", ssm_status_string(hst));
  int64_t base = 0;
  for (int32_t g = 0; g < G; ++g) {
    if (h[(size_t)g] < in[g].k || h[(size_t)g] >= ((int64_t)1 << 30))
      return fail(SSM_E_DISCONNECTED, "ssm_batch_pivots: graph %d has no valid count table (disconnected?)", g);
    out[g].cnt_len = (int32_t)h[(size_t)g];
    out[g].cnt_base = base;
    base += h[(size_t)g];
    if (m_out) m_out[g] = h[(size_t)G + g];
  }
  return SSM_OK;
}

SSM_API int ssm_batch_layout_init(int32_t G, const ssm_batch_graph *graphs, const int64_t *m, const int32_t *rowptr,
                                  const int32_t *colidx, const uint16_t *dip, const int32_t *region,
                                  const int32_t *ecc, int32_t *cnt_off, uint32_t *cnt, float *pos, double *eig,
                                  int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (G < 1 || !graphs || !m || !rowptr || !colidx || !dip || !region || !ecc || !cnt_off || !cnt || !pos ||
      !status || !ws)
    return fail(SSM_E_ARG, "ssm_batch_layout_init: null pointer or G < 1");
  std::vector<LayoutDev> ld((size_t)G);
  std::vector<int32_t> order((size_t)G);
  for (int32_t g = 0; g < G; ++g) {
    const ssm_batch_graph &x = graphs[g];
    if (x.n < 1 || x.n > kPrepMaxN || x.k < 2 || x.k > kPrepMaxK || x.k > x.n || x.cnt_len < x.k)
      return fail(SSM_E_ARG, "ssm_batch_layout_init: graph %d has n = %d, k = %d, cnt_len = %d", g, x.n, x.k, x.cnt_len);
    if (m[g] < 1) return fail(SSM_E_ARG, "ssm_batch_layout_init: graph %d has no edges", g);
    LayoutDev &d = ld[(size_t)g];
    d.n = x.n; d.k = x.k; d.m = m[g];
    d.node_off = x.node_off; d.row_off = x.row_off; d.col_off = x.col_off; d.piv_off = x.piv_off;
    d.dip_off = x.dip_off; d.cnt_off_off = x.cnt_off_off; d.cnt_base = x.cnt_base;
    order[(size_t)g] = g;
  }
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    const LayoutDev &x = ld[(size_t)a], &y = ld[(size_t)b];
    return (int64_t)x.n * x.k * x.k > (int64_t)y.n * y.k * y.k;
  });
  Carver c(ws, ws_bytes);
  PrepWs w;
  carve_prep(c, w, G, -1, 0);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_batch_layout_init: workspace %zu bytes, need %zu", ws_bytes, c.size());
  LayoutDev *dd = w.ld;
  int32_t *dorder = w.order;
  unsigned *ctr = w.ctr + 1;
  SSM_TRY_CUDA(cudaMemcpyAsync(dd, ld.data(), ld.size() * sizeof(LayoutDev), cudaMemcpyHostToDevice, s));
  SSM_TRY_CUDA(cudaMemcpyAsync(dorder, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  SSM_TRY_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned), s));
  LayoutArgs L;
  L.G = G; L.desc = dd; L.order = dorder; L.rowptr = rowptr; L.colidx = colidx; L.region = region; L.ecc = ecc;
  L.dip = dip; L.cnt_off = cnt_off; L.cnt = cnt; L.pos = reinterpret_cast<float2 *>(pos); L.eig = eig; L.ctr = ctr;
  L.status = status;
  const size_t smem = layout_smem();
  SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_prep_layout));
  int per_sm = 0;
  SSM_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prep_layout, kPrepThreads, smem));
  if (per_sm < 1) return fail(SSM_E_ARG, "ssm_batch_layout_init: %zu bytes of shared memory do not fit", smem);
  const int blocks = std::max(1, std::min(G, per_sm * num_sms()));
  note_launch(), k_prep_layout<<<blocks, kPrepThreads, smem, s>>>(L);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
