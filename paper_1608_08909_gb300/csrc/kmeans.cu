// Pivot sampling "k-means sp" (Section 4.1): k max/min-sp pivots are refined
// by k-means over the shortest-path entries of those pivots.
//
// Node i is the point y_i = (d_0i, ..., d_{k-1,i}) of Z^k (column i of the
// pivot-major d_ip table); cluster a starts with centre y_{p_a}.  A centre is
// kept as an exact integer sum S_a (k entries) and a member count n_a, so
// every data-dependent sum is an exact integer and does not depend on the
// order in which the GPU forms it:
//   t_ia = y_i . S_a                                   (exact, 64-bit)
//   g(i,a) = alpha_a - beta_a * t_ia                   (FP64, two roundings)
//   alpha_a = sum_b (S_ab / n_a)^2 in b order, beta_a = 2 / n_a
// g(i,a) is ||y_i - S_a/n_a||^2 minus the common ||y_i||^2; node i joins the
// cluster with the least g, ties to the lowest a.  Passes repeat (at most
// max_iter; the paper caps its k-means at 50) until a pass after the first
// changes no node; between passes S_a, n_a become the members' sum and count
// (a cluster left empty keeps its centre).  The new pivot of cluster a is the
// member minimising the exact integer n_a ||y_i||^2 - 2 t_ia, ties to the
// lowest node id; an empty cluster keeps its max/min pivot.
//
// GB300 layout.  The assignment is the dense part (n k^2 multiply-adds per
// pass): a block takes 64 nodes and, for 64 clusters at a time, stages the
// nodes' distances and the clusters' sums 64 pivots at a time in shared
// memory (as 32-bit words); every thread forms
// a 4 x 4 block of (node, cluster) dot products in 64-bit integer
// multiply-adds; g is then formed in FP64 and the per-node argmin is reduced
// in shared memory in (g, a) order.  The centre update is a histogram per
// pivot row (shared-memory 64-bit atomics, one global atomic per cluster and
// block); integer sums make it order-free.  Every pass is launched up front
// and stops on the device (no host round trip), so the call is asynchronous.
// Exactness needs n * max(d) < 2^32 (32-bit centre sums) and
// n * k * max(d)^2 < 2^53 (t and n_a ||y||^2 exact in FP64 / int64); both are
// checked on the device (SSM_E_ARG).
#include <algorithm>

#include "common.cuh"

namespace ssm {

constexpr int kKmMaxK = 1024;
constexpr int kKmNodes = 64;     // nodes per assignment block
constexpr int kKmClusters = 64;  // clusters per shared-memory chunk
constexpr int kKmThreads = 256;  // 16 node groups x 16 cluster groups, 4 x 4 each
constexpr int kKmChunk = 64;     // pivots (entries of y) staged at a time
constexpr int kKmUpdNodes = 8192;  // nodes per update block

struct KmState {
  unsigned long long *S;     // [k][k] centre sums (row a = cluster a)
  unsigned long long *ST;    // [k][k] the same transposed (row b = pivot b), read by the assignment
  unsigned long long *Snew;  // [k][k]
  unsigned long long *cnt;   // [k] member counts of the centres
  unsigned long long *cnew;  // [k]
  double *alpha, *beta;      // [k]
  unsigned *changed;         // nodes that changed cluster in the current pass
  int32_t *stop;             // set when the passes are over (or on an error)
  unsigned *dmax;            // largest d_ip entry
  long long *vbest;          // [k] pivot choice: least n_a ||y||^2 - 2 t
  int32_t *pbest;            // [k] lowest node id attaining it
  long long *vnode;          // [n] that value per node
};

__global__ void k_km_dmax(int64_t count, const uint16_t *__restrict__ dip, unsigned *__restrict__ out) {
  unsigned m = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned)__ldg(dip + t));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// centre a = y of pivot a; the exactness bounds are checked here
__global__ void k_km_init(int32_t n, int32_t k, const uint16_t *__restrict__ dip, const int32_t *__restrict__ piv,
                          KmState W, int32_t *__restrict__ status) {
  const double dm = (double)*W.dmax;
  if ((double)n * dm >= 4294967296.0 || (double)n * (double)k * dm * dm >= 9007199254740992.0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      dev_fail(status, SSM_E_ARG);
      *W.stop = 1;
    }
    return;
  }
  for (int a = blockIdx.x; a < k; a += gridDim.x) {
    int p = __ldg(piv + a);
    if ((unsigned)p >= (unsigned)n) {
      if (threadIdx.x == 0) {
        dev_fail(status, SSM_E_ARG);
        *W.stop = 1;
      }
      p = 0;
    }
    for (int b = threadIdx.x; b < k; b += blockDim.x) {
      const unsigned long long v = __ldg(dip + (size_t)b * n + p);
      W.S[(size_t)a * k + b] = v;
      W.ST[(size_t)b * k + a] = v;
    }
    if (threadIdx.x == 0) W.cnt[a] = 1ull;
  }
}

// alpha_a, beta_a of the current centres, in the order the definition states
__global__ void k_km_centres(int32_t k, KmState W) {
  if (__ldcg(W.stop)) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x) {
    const double c = (double)W.cnt[a];
    double al = 0.0;
    for (int b = 0; b < k; ++b) {
      const double q = __ddiv_rn((double)W.S[(size_t)a * k + b], c);
      al = __dadd_rn(al, __dmul_rn(q, q));
    }
    W.alpha[a] = al;
    W.beta[a] = __ddiv_rn(2.0, c);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *W.changed = 0u;
}

// one assignment pass over a 64-node tile: the distances of the tile and the
// sums of 64 clusters are staged 64 pivots at a time
__global__ void __launch_bounds__(kKmThreads) k_km_assign(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                                                         KmState W, int32_t *__restrict__ assign) {
  __shared__ __align__(16) unsigned Y[kKmChunk][kKmNodes];     // d of the tile's nodes, pivots b0 .. b0+63
  __shared__ __align__(16) unsigned Sc[kKmChunk][kKmClusters];  // S_ab of 64 clusters, same pivots
  __shared__ double bg[16][kKmNodes];                          // per cluster group: best g of each node
  __shared__ int ba[16][kKmNodes];                             // and its cluster
  __shared__ double s_best[kKmNodes];
  __shared__ int s_arg[kKmNodes];
  if (__ldcg(W.stop)) return;
  const int tid = threadIdx.x;
  const int tn = tid & 15, ta = tid >> 4;  // node group (4 nodes), cluster group (4 clusters)
  const int n0 = blockIdx.x * kKmNodes;
  if (tid < kKmNodes) {
    s_best[tid] = 0.0;
    s_arg[tid] = -1;
  }
  for (int c0 = 0; c0 < k; c0 += kKmClusters) {
    unsigned long long acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0ull;
    for (int b0 = 0; b0 < k; b0 += kKmChunk) {
      __syncthreads();  // the previous chunk is consumed
      for (int t = tid; t < kKmChunk * kKmNodes; t += kKmThreads) {
        const int b = t / kKmNodes, v = t - b * kKmNodes;
        Y[b][v] = (b0 + b < k && n0 + v < n) ? (unsigned)__ldg(dip + (size_t)(b0 + b) * n + n0 + v) : 0u;
      }
      for (int t = tid; t < kKmChunk * kKmClusters; t += kKmThreads) {
        const int b = t / kKmClusters, q = t - b * kKmClusters;
        Sc[b][q] = (b0 + b < k && c0 + q < k) ? (unsigned)W.ST[(size_t)(b0 + b) * k + c0 + q] : 0u;
      }
      __syncthreads();
      const int nb = min(kKmChunk, k - b0);
#pragma unroll 4
      for (int b = 0; b < nb; ++b) {
        const uint4 y = reinterpret_cast<const uint4 *>(Y[b])[tn];
        const uint4 sv4 = reinterpret_cast<const uint4 *>(Sc[b])[ta];
        const unsigned yv[4] = {y.x, y.y, y.z, y.w}, sv[4] = {sv4.x, sv4.y, sv4.z, sv4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += (unsigned long long)yv[i] * sv[j];
      }
    }
    // per node, the best of this thread's 4 clusters (ascending a, strict <)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      double best = 0.0;
      int arg = -1;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int a = c0 + 4 * ta + j;
        if (a < k) {
          const double g = __dsub_rn(W.alpha[a], __dmul_rn(W.beta[a], (double)acc[i][j]));
          if (arg < 0 || g < best) {
            best = g;
            arg = a;
          }
        }
      }
      bg[ta][4 * tn + i] = best;
      ba[ta][4 * tn + i] = arg;
    }
    __syncthreads();
    // cluster groups in ascending a after the running best (strict <)
    if (tid < kKmNodes) {
      double best = s_best[tid];
      int arg = s_arg[tid];
      for (int q = 0; q < 16; ++q) {
        const int a = ba[q][tid];
        if (a < 0) continue;
        const double g = bg[q][tid];
        if (arg < 0 || g < best) {
          best = g;
          arg = a;
        }
      }
      s_best[tid] = best;
      s_arg[tid] = arg;
    }
  }
  __syncthreads();
  if (tid < kKmNodes) {  // warps 0 and 1, whole
    unsigned diff = 0u;
    if (n0 + tid < n) {
      const int a = s_arg[tid];
      diff = assign[n0 + tid] != a ? 1u : 0u;
      assign[n0 + tid] = a;
    }
    const unsigned c = __reduce_add_sync(0xffffffffu, diff);
    if ((tid & 31) == 0 && c) atomicAdd(W.changed, c);
  }
}

// after a pass: stop once a pass after the first changed nothing; otherwise
// clear the next centre sums
__global__ void k_km_after_assign(int32_t k, int32_t pass, KmState W, int32_t *__restrict__ iters) {
  if (__ldcg(W.stop)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *iters = pass;
    if (pass > 1 && __ldcg(W.changed) == 0u) *W.stop = 1;
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += gridDim.x * blockDim.x) W.Snew[t] = 0ull;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) W.cnew[t] = 0ull;
}

// Snew[a][b] = sum over the members i of a of d_bi (and, for b = 0, the member
// counts): block (b, node range) builds a histogram by cluster in shared memory
__global__ void __launch_bounds__(256) k_km_update(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                                                   const int32_t *__restrict__ assign, KmState W) {
  __shared__ unsigned long long hs[kKmMaxK];
  __shared__ unsigned hc[kKmMaxK];
  if (__ldcg(W.stop)) return;
  const int nchunks = (n + kKmUpdNodes - 1) / kKmUpdNodes;
  const int b = blockIdx.x / nchunks, ch = blockIdx.x - b * nchunks;
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    hs[a] = 0ull;
    hc[a] = 0u;
  }
  __syncthreads();
  const int i0 = ch * kKmUpdNodes, i1 = min(n, i0 + kKmUpdNodes);
  const uint16_t *row = dip + (size_t)b * n;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const int a = assign[i];
    atomicAdd(hs + a, (unsigned long long)__ldg(row + i));
    if (b == 0) atomicAdd(hc + a, 1u);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    if (hs[a]) atomicAdd(W.Snew + (size_t)a * k + b, hs[a]);
    if (b == 0 && hc[a]) atomicAdd(W.cnew + a, (unsigned long long)hc[a]);
  }
}

// the members' sums become the centres; an emptied cluster keeps its centre
__global__ void k_km_commit(int32_t k, KmState W) {
  if (__ldcg(W.stop)) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += gridDim.x * blockDim.x) {
    const int a = t / k;
    const unsigned long long c = W.cnew[a];
    if (c > 0ull) {
      W.S[t] = W.Snew[t];
      W.ST[(size_t)(t - a * k) * k + a] = W.Snew[t];
      if (t == a * k) W.cnt[a] = c;
    }
  }
}

// new pivots, step 1: v_i = n_a ||y_i||^2 - 2 t_ia for the node's cluster a,
// and the least v per cluster
__global__ void k_km_pick_value(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                                const int32_t *__restrict__ assign, KmState W) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int a = assign[i];
    if (a < 0) continue;
    const unsigned long long *Sa = W.S + (size_t)a * k;
    unsigned long long yy = 0ull, t = 0ull;
    for (int b = 0; b < k; ++b) {
      const unsigned long long y = __ldg(dip + (size_t)b * n + i);
      yy += y * y;
      t += y * Sa[b];
    }
    const long long v = (long long)(W.cnt[a] * yy) - 2ll * (long long)t;
    W.vnode[i] = v;
    atomicMin(W.vbest + a, v);
  }
}

// step 2: the lowest node id attaining the least v
__global__ void k_km_pick_node(int32_t n, const int32_t *__restrict__ assign, KmState W) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int a = assign[i];
    if (a >= 0 && W.vnode[i] == W.vbest[a]) atomicMin(W.pbest + a, (int)i);
  }
}

__global__ void k_km_pick_out(int32_t k, const int32_t *__restrict__ piv_in, const KmState W,
                              int32_t *__restrict__ piv_out) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x) {
    const int p = W.pbest[a];
    piv_out[a] = p != 0x7FFFFFFF ? p : __ldg(piv_in + a);
  }
}

__global__ void k_km_fill(int32_t k, KmState W) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x) {
    W.vbest[a] = 0x7FFFFFFFFFFFFFFFll;
    W.pbest[a] = 0x7FFFFFFF;
  }
}

static size_t carve_kmeans(Carver &c, KmState &W, int32_t **assign_ws, int32_t n, int32_t k) {
  W.S = c.take<unsigned long long>((size_t)k * k);
  W.ST = c.take<unsigned long long>((size_t)k * k);
  W.Snew = c.take<unsigned long long>((size_t)k * k);
  W.cnt = c.take<unsigned long long>((size_t)k);
  W.cnew = c.take<unsigned long long>((size_t)k);
  W.alpha = c.take<double>((size_t)k);
  W.beta = c.take<double>((size_t)k);
  W.changed = c.take<unsigned>(1);
  W.stop = c.take<int32_t>(1);
  W.dmax = c.take<unsigned>(1);
  W.vbest = c.take<long long>((size_t)k);
  W.pbest = c.take<int32_t>((size_t)k);
  W.vnode = c.take<long long>((size_t)n);
  *assign_ws = c.take<int32_t>((size_t)n);
  return c.size();
}

}  // namespace ssm

SSM_API size_t ssm_kmeans_pivots_workspace(int32_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::KmState W;
  int32_t *a;
  return ssm::carve_kmeans(c, W, &a, n, k);
}

SSM_API int ssm_kmeans_pivots(int32_t n, int32_t k, const uint16_t *dip, const int32_t *pivots_in, int32_t max_iter,
                              int32_t *pivots_out, int32_t *assign, int32_t *iters, int32_t *status, void *ws,
                              size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !dip || !pivots_in || !pivots_out || !iters || !status || !ws)
    return fail(SSM_E_ARG, "ssm_kmeans_pivots: null pointer or bad size");
  if (k < 1 || k > kKmMaxK || k > n) return fail(SSM_E_ARG, "ssm_kmeans_pivots: need 1 <= k <= min(n, %d)", kKmMaxK);
  if (max_iter < 1) return fail(SSM_E_ARG, "ssm_kmeans_pivots: max_iter must be >= 1");
  Carver c(ws, ws_bytes);
  KmState W;
  int32_t *asg_ws = nullptr;
  carve_kmeans(c, W, &asg_ws, n, k);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_kmeans_pivots: workspace %zu bytes, need %zu", ws_bytes, c.size());
  int32_t *asg = assign ? assign : asg_ws;
  const int sms = num_sms();
  SSM_TRY_CUDA(cudaMemsetAsync(W.dmax, 0, sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(W.stop, 0, sizeof(int32_t), s));
  SSM_TRY_CUDA(cudaMemsetAsync(iters, 0, sizeof(int32_t), s));
  SSM_TRY_CUDA(cudaMemsetAsync(asg, 0xFF, (size_t)n * sizeof(int32_t), s));  // -1: no cluster yet
  const int64_t kn = (int64_t)k * n;
  note_launch(), k_km_dmax<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((kn + 255) / 256, sms * 8)), 256, 0, s>>>(
      kn, dip, W.dmax);
  note_launch(), k_km_init<<<std::min(k, sms * 4), 256, 0, s>>>(n, k, dip, pivots_in, W, status);
  const unsigned tiles = (unsigned)((n + kKmNodes - 1) / kKmNodes);
  const unsigned upd_blocks = (unsigned)k * (unsigned)((n + kKmUpdNodes - 1) / kKmUpdNodes);
  const unsigned kk_blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)k * k + 255) / 256, sms * 4));
  for (int pass = 1; pass <= max_iter; ++pass) {
    note_launch(), k_km_centres<<<(k + 127) / 128, 128, 0, s>>>(k, W);
    note_launch(), k_km_assign<<<tiles, kKmThreads, 0, s>>>(n, k, dip, W, asg);
    note_launch(), k_km_after_assign<<<kk_blocks, 256, 0, s>>>(k, pass, W, iters);
    note_launch(), k_km_update<<<upd_blocks, 256, 0, s>>>(n, k, dip, asg, W);
    note_launch(), k_km_commit<<<kk_blocks, 256, 0, s>>>(k, W);
  }
  note_launch(), k_km_fill<<<(k + 255) / 256, 256, 0, s>>>(k, W);
  const int nb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)sms * 8);
  note_launch(), k_km_pick_value<<<nb, 256, 0, s>>>(n, k, dip, asg, W);
  note_launch(), k_km_pick_node<<<nb, 256, 0, s>>>(n, asg, W);
  note_launch(), k_km_pick_out<<<(k + 255) / 256, 256, 0, s>>>(k, pivots_in, W, pivots_out);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
