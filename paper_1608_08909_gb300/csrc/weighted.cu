// Weighted graphs (Algorithm 1 line 2: "weighted MSSP"; Section 3's weights
// with general edge lengths).
//
// Edge lengths l_ij are float32.  A distance is the least float32 path sum:
// d(v) = fl(d(u) + l_uv) along a path walked from the source, minimised over
// paths.  Rounding is monotone and never decreases a sum, so every search
// that only lowers labels and stops when no edge can lower one reaches that
// same minimum; the label-correcting search below and a Dijkstra therefore
// agree bit for bit.
//
//   ssm_edge_lengths        lengths of the CSR edges from the input list
//                           (a repeated edge keeps its shortest length)
//   k_sssp                  one block per source: rounds of relaxations of
//                           a frontier queue, labels lowered by atomicMin
//                           on their bit patterns (non-negative floats order
//                           like their bits); with the label row holding
//                           min over the earlier pivots it is max/min's
//                           pruned search
//   k_wmm_argmax            the next max/min pivot: max over v of
//                           (mind_v, -v) as one 64-bit key
//   k_wregion_keys, bitonic sort, k_wcounts
//                           regions (ties to the lowest pivot index) and
//                           s_ia = |{j in R(a) : 2 d_ja <= d_ia}| by binary
//                           search in each region's sorted distances; s = 0
//                           where the pivot is i or a neighbour of i
//   k_wsweep, k_wsweep_f32  Eq. 4 with w_ij = l_ij^-2 and w'_ia = s_ia/d_ia^2
//                           (FP64 as written; FP32 with w' formed once per
//                           call and one rsqrt per term)
#include <algorithm>

#include "common.cuh"
#include "weighted.cuh"

namespace ssm {

constexpr unsigned kInfBits = 0x7f800000u;
constexpr int kSsspThreads = 512;       // the max/min search: one block, the whole graph
constexpr int kSsspMultiThreads = 512;  // one source per block, up to three blocks per SM

// ------------------------------------------------------------ edge lengths
__global__ void k_fill_u32(int64_t count, unsigned *__restrict__ p, unsigned v) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    p[t] = v;
}

__device__ __forceinline__ int find_in_row(const int32_t *__restrict__ colidx, int b, int e, int v) {
  while (b < e) {
    const int mid = b + ((e - b) >> 1);
    const int c = __ldg(colidx + mid);
    if (c == v) return mid;
    if (c < v) b = mid + 1;
    else e = mid;
  }
  return -1;
}

__global__ void k_elen_set(int32_t n, int64_t m_in, const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                           const float *__restrict__ len, const int32_t *__restrict__ rowptr,
                           const int32_t *__restrict__ colidx, unsigned *__restrict__ elen,
                           unsigned *__restrict__ lmax, int32_t *__restrict__ status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m_in; e += (int64_t)gridDim.x * blockDim.x) {
    const int u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n) {
      dev_fail(status, SSM_E_GRAPH);
      continue;
    }
    if (u == v) continue;
    const float l = len[e];
    if (!(l >= 1.17549435e-38f) || !(l <= 3.4e38f)) {
      dev_fail(status, SSM_E_ARG);
      continue;
    }
    const unsigned lb = __float_as_uint(l);
    atomicMax(lmax, lb);
    const int tu = find_in_row(colidx, rowptr[u], rowptr[u + 1], v);
    const int tv = find_in_row(colidx, rowptr[v], rowptr[v + 1], u);
    if (tu < 0 || tv < 0) {
      dev_fail(status, SSM_E_GRAPH);
      continue;
    }
    atomicMin(elen + tu, lb);
    atomicMin(elen + tv, lb);
  }
}

__global__ void k_elen_check(int32_t n, int64_t m2, const unsigned *__restrict__ elen,
                             const unsigned *__restrict__ lmax, int32_t *__restrict__ status) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && (double)n * (double)__uint_as_float(*lmax) >= 1e37)
    dev_fail(status, SSM_E_ARG);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m2; t += (int64_t)gridDim.x * blockDim.x)
    if (elen[t] == kInfBits) dev_fail(status, SSM_E_GRAPH);  // a CSR edge missing from the list
}

// ------------------------------------------------------------ SSSP
// Near-far label-correcting search (two-bucket Delta-stepping): only labels
// below a threshold T are relaxed in a round ("near"); a node lowered to a
// label at or above T waits in the far pile; when the near queue is empty
// T grows by Delta (at least to the smallest far label plus Delta) and the
// far pile is split again.  Plain rounds over every improved node (the
// first form) re-relaxed each node about 20 times on a 262K-node geometric
// graph; the threshold keeps the search close to label-setting order while
// each round still relaxes a whole band of nodes.  Any order that relaxes
// until nothing improves reaches the same least path sums.
//
// Per block: near queues (current, next), two far piles (ping-pong), and
// membership bitmaps: one per near queue (the next queue's bits are set by
// the relaxations of a round, the current queue's bits cleared as its nodes
// are taken) and one for the far pile.
struct SsspSlot {
  int32_t *nq[2];
  int32_t *fq[2];
  unsigned *in_near[2], *in_far;
};

__host__ __device__ inline size_t sssp_qbytes(int32_t n) { return (((size_t)n * 4) + 255) & ~size_t(255); }
__host__ __device__ inline size_t sssp_bbytes(int32_t n) { return ((((size_t)n + 31) / 32) * 4 + 255) & ~size_t(255); }

__device__ __forceinline__ SsspSlot sssp_slot(char *base, size_t slot_bytes, int b, int32_t n) {
  char *p = base + (size_t)b * slot_bytes;
  const size_t qb = sssp_qbytes(n), bb = sssp_bbytes(n);
  SsspSlot s;
  s.nq[0] = (int32_t *)p;
  s.nq[1] = (int32_t *)(p + qb);
  s.fq[0] = (int32_t *)(p + 2 * qb);
  s.fq[1] = (int32_t *)(p + 3 * qb);
  s.in_near[0] = (unsigned *)(p + 4 * qb);
  s.in_near[1] = (unsigned *)(p + 4 * qb + bb);
  s.in_far = (unsigned *)(p + 4 * qb + 2 * bb);
  return s;
}

size_t sssp_slot_bytes(int32_t n) { return 4 * sssp_qbytes(n) + 3 * sssp_bbytes(n); }

__device__ __forceinline__ bool set_bit(unsigned *bm, int v) {
  const unsigned bit = 1u << (v & 31);
  return !(atomicOr(bm + (v >> 5), bit) & bit);
}

// One search from `source` into row (labels as float bits).  init: set every
// label to +inf first; otherwise the row's labels stay (max/min's pruned
// search: only nodes the new pivot is strictly closer to change).  delta is
// the band width.  The bitmaps are clear on entry and on return.
__device__ void sssp_block(int32_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                           const unsigned *__restrict__ elen, int32_t source, unsigned *__restrict__ row, bool init,
                           float delta, SsspSlot sl, int32_t *__restrict__ status) {
  __shared__ unsigned s_nnext, s_nfar, s_nfar2, s_minfar;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (init)
    for (int v = threadIdx.x; v < n; v += blockDim.x) row[v] = kInfBits;
  __syncthreads();
  if (threadIdx.x == 0) {
    row[source] = 0u;
    sl.nq[0][0] = source;
    s_nfar = 0;
  }
  __syncthreads();
  unsigned nnear = 1, nfar = 0;
  int cur = 0, fcur = 0;
  float T = delta;
  // every pass relaxes at least one node whose label is then final for the
  // band, so the passes are bounded; the cap only guards against a fault
  const int64_t cap = 64ll * ((int64_t)n + 16);
  for (int64_t pass = 0;; ++pass) {
    if (pass > cap) {
      if (threadIdx.x == 0) dev_fail(status, SSM_E_NUMERIC);
      break;
    }
    if (nnear == 0) {
      if (nfar == 0) break;
      // next band: T >= smallest far label + delta; split the far pile
      const int32_t *fq = fcur ? sl.fq[1] : sl.fq[0];
      int32_t *fq2 = fcur ? sl.fq[0] : sl.fq[1];
      int32_t *nq = cur ? sl.nq[1] : sl.nq[0];
      if (threadIdx.x == 0) {
        s_minfar = kInfBits;
        s_nnext = 0;
        s_nfar2 = 0;
      }
      __syncthreads();
      for (unsigned t = threadIdx.x; t < nfar; t += blockDim.x) atomicMin(&s_minfar, __ldcg(row + fq[t]));
      __syncthreads();
      T = fmaxf(T + delta, __uint_as_float(s_minfar) + delta);
      // where delta vanishes against the labels, take the next float above
      // the smallest far label so that at least that node moves on
      if (!(T > __uint_as_float(s_minfar))) T = __uint_as_float(s_minfar + 1u);
      for (unsigned t = threadIdx.x; t < nfar; t += blockDim.x) {
        const int v = fq[t];
        atomicAnd(sl.in_far + (v >> 5), ~(1u << (v & 31)));
        if (__uint_as_float(__ldcg(row + v)) < T) nq[atomicAdd(&s_nnext, 1u)] = v;
        else {
          set_bit(sl.in_far, v);
          fq2[atomicAdd(&s_nfar2, 1u)] = v;
        }
      }
      __syncthreads();
      nnear = s_nnext;
      nfar = s_nfar2;
      fcur ^= 1;
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) {
      s_nnext = 0;
      s_nfar = nfar;
    }
    __syncthreads();
    const int32_t *qc = cur ? sl.nq[1] : sl.nq[0];
    int32_t *qn = cur ? sl.nq[0] : sl.nq[1];
    unsigned *inc = cur ? sl.in_near[1] : sl.in_near[0];
    unsigned *inn = cur ? sl.in_near[0] : sl.in_near[1];
    int32_t *fq = fcur ? sl.fq[1] : sl.fq[0];
    // a warp takes 32 near entries at a time and walks their rows together,
    // 32 edge slots per step (hubs spread over the lanes)
    for (unsigned base = (unsigned)warp * 32u; base < nnear; base += blockDim.x) {
      const unsigned idx = base + (unsigned)lane;
      int b = 0, e = 0;
      unsigned dvb = kInfBits;
      if (idx < nnear) {
        const int v = qc[idx];
        atomicAnd(inc + (v >> 5), ~(1u << (v & 31)));
        b = __ldg(rowptr + v);
        e = __ldg(rowptr + v + 1);
        dvb = __ldcg(row + v);
      }
      const int deg = e - b;
      int incl = deg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      for (int s0 = 0; s0 < total; s0 += 32) {
        const int slot = s0 + lane;
        int lo = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int pv = __shfl_sync(0xffffffffu, incl, lo + step - 1);
          if (pv <= slot) lo += step;
        }
        const int owner = lo > 31 ? 31 : lo;
        const int o_incl = __shfl_sync(0xffffffffu, incl, owner);
        const int o_deg = __shfl_sync(0xffffffffu, deg, owner);
        const int o_beg = __shfl_sync(0xffffffffu, b, owner);
        const unsigned o_d = __shfl_sync(0xffffffffu, dvb, owner);
        if (slot < total) {
          const int t = o_beg + (slot - (o_incl - o_deg));
          const int u = __ldg(colidx + t);
          const float nd = __fadd_rn(__uint_as_float(o_d), __uint_as_float(__ldg(elen + t)));
          const unsigned ndb = __float_as_uint(nd);
          const unsigned old = atomicMin(row + u, ndb);
          if (ndb < old) {
            if (nd < T) {
              if (set_bit(inn, u)) qn[atomicAdd(&s_nnext, 1u)] = u;
            } else if (set_bit(sl.in_far, u)) {
              fq[atomicAdd(&s_nfar, 1u)] = u;
            }
          }
        }
      }
    }
    __syncthreads();
    nnear = s_nnext;
    nfar = s_nfar;
    cur ^= 1;
    __syncthreads();
  }
}

// band width of the near-far search: kDeltaScale times the mean edge length
constexpr float kDeltaScale = 8.0f;

__global__ void k_mean_length(int32_t n, const int32_t *__restrict__ rowptr, const float *__restrict__ elen,
                              float *__restrict__ delta) {
  __shared__ double red[32];
  const int64_t m2 = rowptr[n];
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < m2; t += blockDim.x) acc += (double)elen[t];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    const float mean = m2 > 0 ? (float)(t / (double)m2) : 1.0f;
    *delta = mean > 0.0f ? kDeltaScale * mean : 1.0f;
  }
}

// d_ip mode: block b takes sources b, b + grid, ...; dist rows [k][n]
__global__ void __launch_bounds__(kSsspMultiThreads, 3) k_sssp_multi(int32_t n, const int32_t *__restrict__ rowptr,
                                                             const int32_t *__restrict__ colidx,
                                                             const unsigned *__restrict__ elen, int32_t k,
                                                             const int32_t *__restrict__ sources,
                                                             unsigned *__restrict__ dist, const float *__restrict__ delta,
                                                             char *slots, size_t slot_bytes,
                                                             int32_t *__restrict__ status) {
  const SsspSlot sl = sssp_slot(slots, slot_bytes, blockIdx.x, n);
  const float dl = *delta;
  for (int a = blockIdx.x; a < k; a += gridDim.x) {
    const int s = sources[a];
    if (s < 0 || s >= n) {
      if (threadIdx.x == 0) dev_fail(status, SSM_E_ARG);
      continue;
    }
    sssp_block(n, rowptr, colidx, elen, s, dist + (size_t)a * n, true, dl, sl, status);
  }
}

// max/min mode (one block): the source is the pivot encoded in *key (or
// `start` when key is null); the search lowers mind in place
__global__ void __launch_bounds__(kSsspThreads) k_sssp_maxmin(int32_t n, const int32_t *__restrict__ rowptr,
                                                              const int32_t *__restrict__ colidx,
                                                              const unsigned *__restrict__ elen, int32_t start,
                                                              const unsigned long long *__restrict__ key,
                                                              int32_t *__restrict__ pivot_out,
                                                              unsigned *__restrict__ mind,
                                                              const float *__restrict__ delta, char *slots,
                                                              size_t slot_bytes, bool init,
                                                              int32_t *__restrict__ status) {
  const SsspSlot sl = sssp_slot(slots, slot_bytes, 0, n);
  const int s = key ? (int)(0xFFFFFFFFu - (unsigned)(*key & 0xFFFFFFFFull)) : start;
  if (s < 0 || s >= n) {
    if (threadIdx.x == 0) dev_fail(status, SSM_E_ARG);
    return;
  }
  if (threadIdx.x == 0) *pivot_out = s;
  sssp_block(n, rowptr, colidx, elen, s, mind, init, *delta, sl, status);
}

// *key = max over v of (bits(mind_v) << 32 | (2^32 - 1 - v)): the largest
// label, ties to the lowest node id; an unreachable node (+inf) is an error
__global__ void k_wmm_argmax(int32_t n, const unsigned *__restrict__ mind, unsigned long long *__restrict__ key,
                             int32_t *__restrict__ status) {
  unsigned long long best = 0;
  bool inf = false;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const unsigned b = mind[v];
    inf |= b >= kInfBits;
    const unsigned long long kk = ((unsigned long long)b << 32) | (0xFFFFFFFFu - (unsigned)v);
    best = kk > best ? kk : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
    best = t > best ? t : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(key, best);
  if (inf) dev_fail(status, SSM_E_DISCONNECTED);
}

__global__ void k_check_finite_rows(int64_t count, const unsigned *__restrict__ dist, int32_t *__restrict__ status) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    if (dist[t] >= kInfBits) {
      dev_fail(status, SSM_E_DISCONNECTED);
      return;
    }
}

size_t sssp_ws_bytes(int32_t n, int32_t k) { return 256 + sssp_slot_bytes(n) * (size_t)sssp_blocks(k); }

int launch_sssp(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t k,
                const int32_t *sources, float *dist, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  const int blocks = sssp_blocks(k);
  const size_t sb = sssp_slot_bytes(n);
  if (ws_bytes < sssp_ws_bytes(n, k))
    return fail(SSM_E_NOMEM, "sssp: workspace %zu bytes, need %zu", ws_bytes, sssp_ws_bytes(n, k));
  float *delta = (float *)ws;
  char *slots = (char *)ws + 256;
  SSM_TRY_CUDA(cudaMemsetAsync(slots, 0, sb * (size_t)blocks, s));
  note_launch(), k_mean_length<<<1, 1024, 0, s>>>(n, rowptr, elen, delta);
  note_launch(), k_sssp_multi<<<blocks, kSsspMultiThreads, 0, s>>>(n, rowptr, colidx, (const unsigned *)elen, k, sources,
                                                            (unsigned *)dist, delta, slots, sb, status);
  const int64_t cnt = (int64_t)k * n;
  note_launch(), k_check_finite_rows<<<(unsigned)std::min<int64_t>((cnt + 255) / 256, (int64_t)num_sms() * 8), 256, 0,
                                       s>>>(cnt, (const unsigned *)dist, status);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

int sssp_blocks(int32_t k) { return std::max(1, std::min<int>(k, num_sms() * 3)); }

// ------------------------------------------------------------ regions and s
__global__ void k_wregion_keys(int32_t n, int32_t k, const float *__restrict__ dist, int32_t *__restrict__ region,
                               unsigned long long *__restrict__ keys, int64_t npad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
    if (i >= n) {
      keys[i] = ~0ull;
      continue;
    }
    int best = 0;
    float bd = __ldg(dist + i);
    for (int a = 1; a < k; ++a) {
      const float d = __ldg(dist + (size_t)a * n + i);
      if (d < bd) {
        bd = d;
        best = a;
      }
    }
    region[i] = best;
    keys[i] = ((unsigned long long)best << 32) | __float_as_uint(bd);
  }
}

// bitonic sort of npad (a power of two, at least 2048) 64-bit keys, ascending
constexpr int kSortChunk = 2048;

__device__ __forceinline__ void cmp_swap(unsigned long long &x, unsigned long long &y, bool up) {
  if ((x > y) == up) {
    const unsigned long long t = x;
    x = y;
    y = t;
  }
}

// stages kk = 2 .. 2048 inside each 2048-key chunk (directions by global index)
__global__ void __launch_bounds__(1024) k_bitonic_local(unsigned long long *__restrict__ keys) {
  __shared__ unsigned long long sk[kSortChunk];
  const int64_t base = (int64_t)blockIdx.x * kSortChunk;
  sk[threadIdx.x] = keys[base + threadIdx.x];
  sk[threadIdx.x + 1024] = keys[base + threadIdx.x + 1024];
  __syncthreads();
  for (int kk = 2; kk <= kSortChunk; kk <<= 1)
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const int t = threadIdx.x;
      const int i = ((t / j) * 2 * j) + (t % j);
      const bool up = (((base + i) & kk) == 0);
      cmp_swap(sk[i], sk[i + j], up);
      __syncthreads();
    }
  keys[base + threadIdx.x] = sk[threadIdx.x];
  keys[base + threadIdx.x + 1024] = sk[threadIdx.x + 1024];
}

__global__ void k_bitonic_global(unsigned long long *__restrict__ keys, int64_t npad, int64_t kk, int64_t j) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npad / 2; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = ((t / j) * 2 * j) + (t % j);
    const bool up = ((i & kk) == 0);
    unsigned long long x = keys[i], y = keys[i + j];
    cmp_swap(x, y, up);
    keys[i] = x;
    keys[i + j] = y;
  }
}

// the steps j = 1024 .. 1 of stage kk inside each chunk
__global__ void __launch_bounds__(1024) k_bitonic_merge_local(unsigned long long *__restrict__ keys, int64_t kk) {
  __shared__ unsigned long long sk[kSortChunk];
  const int64_t base = (int64_t)blockIdx.x * kSortChunk;
  sk[threadIdx.x] = keys[base + threadIdx.x];
  sk[threadIdx.x + 1024] = keys[base + threadIdx.x + 1024];
  __syncthreads();
  for (int j = kSortChunk >> 1; j > 0; j >>= 1) {
    const int t = threadIdx.x;
    const int i = ((t / j) * 2 * j) + (t % j);
    const bool up = (((base + i) & kk) == 0);
    cmp_swap(sk[i], sk[i + j], up);
    __syncthreads();
  }
  keys[base + threadIdx.x] = sk[threadIdx.x];
  keys[base + threadIdx.x + 1024] = sk[threadIdx.x + 1024];
}

static int launch_sort(unsigned long long *keys, int64_t npad, cudaStream_t s) {
  const unsigned chunks = (unsigned)(npad / kSortChunk);
  note_launch(), k_bitonic_local<<<chunks, 1024, 0, s>>>(keys);
  const unsigned gb = (unsigned)std::min<int64_t>((npad / 2 + 255) / 256, (int64_t)num_sms() * 16);
  for (int64_t kk = 2 * kSortChunk; kk <= npad; kk <<= 1) {
    for (int64_t j = kk >> 1; j >= kSortChunk; j >>= 1) note_launch(), k_bitonic_global<<<gb, 256, 0, s>>>(keys, npad, kk, j);
    note_launch(), k_bitonic_merge_local<<<chunks, 1024, 0, s>>>(keys, kk);
  }
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

// seg[a] = first key position of region a (a = 0..k; padding keys sort last)
__global__ void k_seg_start(int32_t k, const unsigned long long *__restrict__ keys, int64_t npad,
                            int64_t *__restrict__ seg) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a <= k; a += gridDim.x * blockDim.x) {
    const unsigned long long want = (unsigned long long)a << 32;
    int64_t lo = 0, hi = npad;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (keys[mid] < want) lo = mid + 1;
      else hi = mid;
    }
    seg[a] = lo;
  }
}

__global__ void k_wcounts(int32_t n, int32_t k, const int32_t *__restrict__ rowptr,
                          const int32_t *__restrict__ colidx, const int32_t *__restrict__ pivots,
                          const float *__restrict__ dist, const unsigned long long *__restrict__ keys,
                          const int64_t *__restrict__ seg, uint32_t *__restrict__ s_out) {
  const int64_t total = (int64_t)k * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / n), i = (int)(t - (int64_t)a * n);
    const int p = __ldg(pivots + a);
    uint32_t c = 0;
    if (p != i && find_in_row(colidx, __ldg(rowptr + i), __ldg(rowptr + i + 1), p) < 0) {
      const float d = __ldg(dist + t);
      // entries of region a with 2 * d_ja <= d_ia: a prefix of the sorted segment
      int64_t lo = seg[a], hi = seg[a + 1];
      const int64_t b0 = lo;
      while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        const float dj = __uint_as_float((unsigned)(keys[mid] & 0xFFFFFFFFull));
        if (__fmul_rn(2.0f, dj) <= d) lo = mid + 1;
        else hi = mid;
      }
      c = (uint32_t)(lo - b0);
    }
    s_out[t] = c;
  }
}

// ------------------------------------------------------------ the sweep
constexpr int kWSweepThreads = 256;

// Eq. 4 for one node in FP64, every operation rounded on its own in the
// order of the plain FP64 definition (bit-identical to it)
template <class T2>
struct WArith;

template <>
struct WArith<double2> {
  using R = double;
  __device__ static R add(R a, R b) { return __dadd_rn(a, b); }
  __device__ static R sub(R a, R b) { return __dsub_rn(a, b); }
  __device__ static R mul(R a, R b) { return __dmul_rn(a, b); }
  __device__ static R div(R a, R b) { return __ddiv_rn(a, b); }
  __device__ static R sqrt_(R a) { return __dsqrt_rn(a); }
};

template <class T2>
__global__ void __launch_bounds__(kWSweepThreads) k_wsweep(int32_t n, const int32_t *__restrict__ rowptr,
                                                           const int32_t *__restrict__ colidx,
                                                           const float *__restrict__ elen, int32_t k,
                                                           const int32_t *__restrict__ pivots,
                                                           const float *__restrict__ dist,
                                                           const uint32_t *__restrict__ s_tab,
                                                           const T2 *__restrict__ X, T2 *__restrict__ Y,
                                                           double *__restrict__ part, unsigned *__restrict__ done,
                                                           double *__restrict__ rel) {
  using A = WArith<T2>;
  using R = typename A::R;
  extern __shared__ __align__(16) unsigned char wsm[];
  T2 *xp = reinterpret_cast<T2 *>(wsm);
  for (int a = threadIdx.x; a < k; a += blockDim.x) xp[a] = X[__ldg(pivots + a)];
  __syncthreads();
  double dn = 0.0, dd = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T2 xi = X[i];
    R nx = 0, ny = 0, den = 0;
    for (int t = __ldg(rowptr + i); t < __ldg(rowptr + i + 1); ++t) {
      const int j = __ldg(colidx + t);
      const R l = (R)__ldg(elen + t);
      const R w = A::div((R)1, A::mul(l, l));
      const T2 xj = X[j];
      const R dx = A::sub(xi.x, xj.x), dy = A::sub(xi.y, xj.y);
      const R r = A::sqrt_(A::add(A::mul(dx, dx), A::mul(dy, dy)));
      if (r > (R)0) {
        nx = A::add(nx, A::mul(w, A::add(xj.x, A::div(A::mul(l, dx), r))));
        ny = A::add(ny, A::mul(w, A::add(xj.y, A::div(A::mul(l, dy), r))));
      } else {
        nx = A::add(nx, A::mul(w, xj.x));
        ny = A::add(ny, A::mul(w, xj.y));
      }
      den = A::add(den, w);
    }
    for (int a = 0; a < k; ++a) {
      const uint32_t sc = __ldg(s_tab + (size_t)a * n + i);
      if (sc == 0) continue;  // the pivot is i itself or one of its neighbours
      const R d = (R)__ldg(dist + (size_t)a * n + i);
      const R w = A::div((R)sc, A::mul(d, d));
      const T2 xq = xp[a];
      const R dx = A::sub(xi.x, xq.x), dy = A::sub(xi.y, xq.y);
      const R r = A::sqrt_(A::add(A::mul(dx, dx), A::mul(dy, dy)));
      if (r > (R)0) {
        nx = A::add(nx, A::mul(w, A::add(xq.x, A::div(A::mul(d, dx), r))));
        ny = A::add(ny, A::mul(w, A::add(xq.y, A::div(A::mul(d, dy), r))));
      } else {
        nx = A::add(nx, A::mul(w, xq.x));
        ny = A::add(ny, A::mul(w, xq.y));
      }
      den = A::add(den, w);
    }
    T2 y = xi;
    if (den > (R)0) {
      y.x = A::div(nx, den);
      y.y = A::div(ny, den);
    }
    Y[i] = y;
    const double ex = (double)y.x - (double)xi.x, ey = (double)y.y - (double)xi.y;
    dn += ex * ex + ey * ey;
    dd += (double)xi.x * (double)xi.x + (double)xi.y * (double)xi.y;
  }
  // relative change: block sums, then the last block adds them in block order
  __shared__ double red[2][kWSweepThreads / 32];
  __shared__ unsigned s_ticket;
  for (int o = 16; o > 0; o >>= 1) {
    dn += __shfl_xor_sync(0xffffffffu, dn, o);
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = dn;
    red[1][threadIdx.x >> 5] = dd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < kWSweepThreads / 32; ++w) {
      a0 += red[0][w];
      a1 += red[1][w];
    }
    part[2 * blockIdx.x] = a0;
    part[2 * blockIdx.x + 1] = a1;
    __threadfence();
    s_ticket = atomicAdd(done, 1u);
  }
  __syncthreads();
  if (s_ticket != gridDim.x - 1 || threadIdx.x != 0) return;
  __threadfence();
  double a0 = 0.0, a1 = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) {
    a0 += __ldcg(part + 2 * b);
    a1 += __ldcg(part + 2 * b + 1);
  }
  *rel = a1 > 0.0 ? sqrt(a0) / sqrt(a1) : 0.0;
  *done = 0;
}

// FP32 form: w'_ia = s_ia / d_ia^2 formed once per call into wtab (0 where
// the pivot term is skipped), then per term one rsqrt and multiply-adds:
// u = 1/r, B = w' d u, numerator = sum w' x_p + sum B (x_i - x_p) (kept as
// two sums so that nothing cancels); r = 0 contributes w' x_p only.  A thread
// owns one node; eight pivots' (d, w') pairs are loaded before they are used.
__global__ void k_wprep(int64_t count, const float *__restrict__ dist, const uint32_t *__restrict__ s_tab,
                        float *__restrict__ wtab) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t sc = s_tab[t];
    const float d = dist[t];
    wtab[t] = sc ? (float)sc / (d * d) : 0.0f;
  }
}

constexpr int kWPrefetch = 8;

__global__ void __launch_bounds__(kWSweepThreads) k_wsweep_f32(int32_t n, const int32_t *__restrict__ rowptr,
                                                               const int32_t *__restrict__ colidx,
                                                               const float *__restrict__ elen, int32_t k,
                                                               const int32_t *__restrict__ pivots,
                                                               const float *__restrict__ dist,
                                                               const float *__restrict__ wtab,
                                                               const float2 *__restrict__ X, float2 *__restrict__ Y,
                                                               double *__restrict__ part, unsigned *__restrict__ done,
                                                               double *__restrict__ rel) {
  extern __shared__ __align__(16) unsigned char wsm[];
  float2 *xp = reinterpret_cast<float2 *>(wsm);
  for (int a = threadIdx.x; a < k; a += blockDim.x) xp[a] = X[__ldg(pivots + a)];
  __syncthreads();
  double dn = 0.0, dd = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 xi = X[i];
    float wx = 0.f, wy = 0.f, bx = 0.f, by = 0.f, den = 0.f;
    const float *dcol = dist + i;
    const float *wcol = wtab + i;
    // the first pivots' (d, w') are requested before the neighbour gathers,
    // and every batch's loads are issued before the previous batch is used
    float dq[kWPrefetch], wq[kWPrefetch];
#pragma unroll
    for (int q = 0; q < kWPrefetch; ++q) {
      const bool ok = q < k;
      dq[q] = ok ? __ldg(dcol + (size_t)q * n) : 0.f;
      wq[q] = ok ? __ldg(wcol + (size_t)q * n) : 0.f;
    }
    for (int t = __ldg(rowptr + i); t < __ldg(rowptr + i + 1); ++t) {
      const float l = __ldg(elen + t);
      const float w = 1.0f / (l * l);
      const float2 xj = X[__ldg(colidx + t)];
      const float dx = xi.x - xj.x, dy = xi.y - xj.y;
      const float r2 = dx * dx + dy * dy;
      const float B = r2 > 0.f ? w * l * rsqrtf(r2) : 0.f;
      wx += w * xj.x;
      wy += w * xj.y;
      bx += B * dx;
      by += B * dy;
      den += w;
    }
    for (int a0 = 0; a0 < k; a0 += kWPrefetch) {
      float dn_[kWPrefetch], wn_[kWPrefetch];
#pragma unroll
      for (int q = 0; q < kWPrefetch; ++q) {
        const bool ok = a0 + kWPrefetch + q < k;
        dn_[q] = ok ? __ldg(dcol + (size_t)(a0 + kWPrefetch + q) * n) : 0.f;
        wn_[q] = ok ? __ldg(wcol + (size_t)(a0 + kWPrefetch + q) * n) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < kWPrefetch; ++q) {
        if (a0 + q >= k) break;
        const float2 p = xp[a0 + q];
        const float w = wq[q];
        const float dx = xi.x - p.x, dy = xi.y - p.y;
        const float r2 = dx * dx + dy * dy;
        const float B = r2 > 0.f ? w * dq[q] * rsqrtf(r2) : 0.f;
        wx += w * p.x;
        wy += w * p.y;
        bx += B * dx;
        by += B * dy;
        den += w;
      }
#pragma unroll
      for (int q = 0; q < kWPrefetch; ++q) {
        dq[q] = dn_[q];
        wq[q] = wn_[q];
      }
    }
    float2 y = xi;
    if (den > 0.f) {
      y.x = (wx + bx) / den;
      y.y = (wy + by) / den;
    }
    Y[i] = y;
    const double ex = (double)y.x - (double)xi.x, ey = (double)y.y - (double)xi.y;
    dn += ex * ex + ey * ey;
    dd += (double)xi.x * (double)xi.x + (double)xi.y * (double)xi.y;
  }
  __shared__ double red[2][kWSweepThreads / 32];
  __shared__ unsigned s_ticket;
  for (int o = 16; o > 0; o >>= 1) {
    dn += __shfl_xor_sync(0xffffffffu, dn, o);
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = dn;
    red[1][threadIdx.x >> 5] = dd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < kWSweepThreads / 32; ++w) {
      a0 += red[0][w];
      a1 += red[1][w];
    }
    part[2 * blockIdx.x] = a0;
    part[2 * blockIdx.x + 1] = a1;
    __threadfence();
    s_ticket = atomicAdd(done, 1u);
  }
  __syncthreads();
  if (s_ticket != gridDim.x - 1 || threadIdx.x != 0) return;
  __threadfence();
  double a0 = 0.0, a1 = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) {
    a0 += __ldcg(part + 2 * b);
    a1 += __ldcg(part + 2 * b + 1);
  }
  *rel = a1 > 0.0 ? sqrt(a0) / sqrt(a1) : 0.0;
  *done = 0;
}

}  // namespace ssm

// =========================================================== C ABI
SSM_API int ssm_edge_lengths(int32_t n, int64_t m_in, const int32_t *src, const int32_t *dst, const float *len,
                             int64_t m, const int32_t *rowptr, const int32_t *colidx, float *elen, int32_t *status,
                             void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || m_in < 0 || m < 0 || !rowptr || !colidx || !elen || !status || !ws || (m_in > 0 && (!src || !dst || !len)))
    return fail(SSM_E_ARG, "ssm_edge_lengths: null pointer or bad size");
  if (ws_bytes < 256) return fail(SSM_E_NOMEM, "ssm_edge_lengths: workspace %zu bytes, need 256", ws_bytes);
  unsigned *lmax = (unsigned *)ws;
  const int64_t m2 = 2 * m;
  const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((std::max(m2, m_in) + 255) / 256,
                                                                        (int64_t)num_sms() * 8));
  SSM_TRY_CUDA(cudaMemsetAsync(lmax, 0, sizeof(unsigned), s));
  if (m2 > 0) note_launch(), k_fill_u32<<<gb, 256, 0, s>>>(m2, (unsigned *)elen, kInfBits);
  if (m_in > 0)
    note_launch(), k_elen_set<<<gb, 256, 0, s>>>(n, m_in, src, dst, len, rowptr, colidx, (unsigned *)elen, lmax, status);
  note_launch(), k_elen_check<<<gb, 256, 0, s>>>(n, m2, (const unsigned *)elen, lmax, status);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

SSM_API size_t ssm_pivot_sssp_workspace(int32_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  return ssm::sssp_ws_bytes(n, k);
}

SSM_API int ssm_pivot_sssp(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, const float *elen,
                           int32_t k, const int32_t *sources, float *dist, int32_t *status, void *ws, size_t ws_bytes,
                           cudaStream_t s) {
  using namespace ssm;
  (void)m;
  if (n < 1 || k < 1 || !rowptr || !colidx || !elen || !sources || !dist || !status || !ws)
    return fail(SSM_E_ARG, "ssm_pivot_sssp: null pointer or bad size");
  return launch_sssp(n, rowptr, colidx, elen, k, sources, dist, status, ws, ws_bytes, s);
}

namespace ssm {
struct WmmWs {
  unsigned *mind;
  unsigned long long *keys;
  float *delta;
  char *slot;
};
static size_t carve_wmm(Carver &c, WmmWs &w, int32_t n, int32_t k) {
  w.mind = c.take<unsigned>((size_t)n);
  w.keys = c.take<unsigned long long>((size_t)k);
  w.delta = c.take<float>(1);
  w.slot = c.take<char>(sssp_slot_bytes(n));
  return c.size();
}
}  // namespace ssm

SSM_API size_t ssm_select_pivots_weighted_workspace(int32_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::WmmWs w;
  return ssm::carve_wmm(c, w, n, k);
}

SSM_API int ssm_select_pivots_weighted(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx,
                                       const float *elen, int32_t k, int32_t start, int32_t *pivots,
                                       int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  (void)m;
  if (n < 1 || !rowptr || !colidx || !elen || !pivots || !status || !ws)
    return fail(SSM_E_ARG, "ssm_select_pivots_weighted: null pointer or n < 1");
  if (k < 1 || k > n || start < 0 || start >= n)
    return fail(SSM_E_ARG, "ssm_select_pivots_weighted: need 1 <= k <= n and 0 <= start < n");
  Carver c(ws, ws_bytes);
  WmmWs w;
  carve_wmm(c, w, n, k);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_select_pivots_weighted: workspace %zu bytes, need %zu", ws_bytes, c.size());
  SSM_TRY_CUDA(cudaMemsetAsync(w.keys, 0, (size_t)k * sizeof(unsigned long long), s));
  SSM_TRY_CUDA(cudaMemsetAsync(w.slot, 0, sssp_slot_bytes(n), s));
  const size_t sb = sssp_slot_bytes(n);
  note_launch(), k_mean_length<<<1, 1024, 0, s>>>(n, rowptr, elen, w.delta);
  note_launch(), k_sssp_maxmin<<<1, kSsspThreads, 0, s>>>(n, rowptr, colidx, (const unsigned *)elen, start, nullptr,
                                                        pivots, w.mind, w.delta, w.slot, sb, true, status);
  const unsigned ab = (unsigned)std::max(1, std::min((n + 255) / 256, num_sms() * 4));
  for (int a = 1; a < k; ++a) {
    note_launch(), k_wmm_argmax<<<ab, 256, 0, s>>>(n, w.mind, w.keys + a, status);
    note_launch(), k_sssp_maxmin<<<1, kSsspThreads, 0, s>>>(n, rowptr, colidx, (const unsigned *)elen, 0, w.keys + a,
                                                          pivots + a, w.mind, w.delta, w.slot, sb, false, status);
  }
  if (k == 1) note_launch(), k_wmm_argmax<<<ab, 256, 0, s>>>(n, w.mind, w.keys, status);  // reachability check
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

namespace ssm {
static int64_t sort_size(int32_t n) {
  int64_t p = kSortChunk;
  while (p < n) p <<= 1;
  return p;
}
struct WcntWs {
  unsigned long long *keys;
  int64_t *seg;
};
static size_t carve_wcnt(Carver &c, WcntWs &w, int32_t n, int32_t k) {
  w.keys = c.take<unsigned long long>((size_t)sort_size(n));
  w.seg = c.take<int64_t>((size_t)k + 1);
  return c.size();
}
}  // namespace ssm

SSM_API size_t ssm_weighted_counts_workspace(int32_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::WcntWs w;
  return ssm::carve_wcnt(c, w, n, k);
}

SSM_API int ssm_weighted_counts(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                                const int32_t *pivots, const float *dist, int32_t *region, uint32_t *s_tab,
                                int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || k < 1 || !rowptr || !colidx || !pivots || !dist || !region || !s_tab || !status || !ws)
    return fail(SSM_E_ARG, "ssm_weighted_counts: null pointer or bad size");
  Carver c(ws, ws_bytes);
  WcntWs w;
  carve_wcnt(c, w, n, k);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_weighted_counts: workspace %zu bytes, need %zu", ws_bytes, c.size());
  const int64_t npad = sort_size(n);
  const int sms = num_sms();
  note_launch(), k_wregion_keys<<<(unsigned)std::min<int64_t>((npad + 255) / 256, (int64_t)sms * 8), 256, 0, s>>>(
      n, k, dist, region, w.keys, npad);
  if (int rc = launch_sort(w.keys, npad, s)) return rc;
  note_launch(), k_seg_start<<<std::max(1, (k + 256) / 256), 256, 0, s>>>(k, w.keys, npad, w.seg);
  const int64_t total = (int64_t)k * n;
  note_launch(), k_wcounts<<<(unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 16), 256, 0, s>>>(
      n, k, rowptr, colidx, pivots, dist, w.keys, w.seg, s_tab);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

namespace ssm {
static int wsweep_blocks(int32_t n) { return std::max(1, std::min((n + kWSweepThreads - 1) / kWSweepThreads, num_sms() * 8)); }
struct WSweepWs {
  void *buf;
  double *part;
  unsigned *done;
  float *wtab;
};
static size_t carve_wsweep(Carver &c, WSweepWs &w, int32_t n, int32_t k, int32_t precision) {
  w.buf = c.take<char>((size_t)n * (precision == 64 ? 16 : 8));
  w.part = c.take<double>(2 * (size_t)wsweep_blocks(n));
  w.done = c.take<unsigned>(1);
  w.wtab = precision == 32 ? c.take<float>((size_t)k * n) : nullptr;
  return c.size();
}
}  // namespace ssm

SSM_API size_t ssm_iterate_weighted_workspace(int32_t n, int32_t k, int32_t precision) {
  if (n < 1 || k < 1 || (precision != 32 && precision != 64)) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::WSweepWs w;
  return ssm::carve_wsweep(c, w, n, k, precision);
}

SSM_API int ssm_iterate_weighted(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen,
                                 int32_t k, const int32_t *pivots, const float *dist, const uint32_t *s_tab, void *pos,
                                 int32_t precision, int32_t iters, double *rel_change, int32_t *status, void *ws,
                                 size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || k < 1 || !rowptr || !colidx || !elen || !pivots || !dist || !s_tab || !pos || !status || !ws ||
      !rel_change || iters < 0)
    return fail(SSM_E_ARG, "ssm_iterate_weighted: null pointer or bad size");
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_iterate_weighted: precision must be 32 or 64");
  const size_t esz = precision == 64 ? 16 : 8;
  if ((size_t)k * esz > 200 * 1024) return fail(SSM_E_ARG, "ssm_iterate_weighted: k too large for the pivot stage");
  Carver c(ws, ws_bytes);
  WSweepWs w;
  carve_wsweep(c, w, n, k, precision);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_iterate_weighted: workspace %zu bytes, need %zu", ws_bytes, c.size());
  SSM_TRY_CUDA(cudaMemsetAsync(w.done, 0, sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(rel_change, 0, sizeof(double), s));
  const int nb = wsweep_blocks(n);
  const size_t smem = (size_t)k * esz;
  if (precision == 64) {
    SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_wsweep<double2>));
  } else {
    SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_wsweep_f32));
    if (iters > 0) {
      const int64_t cnt = (int64_t)k * n;
      note_launch(), k_wprep<<<(unsigned)std::min<int64_t>((cnt + 255) / 256, (int64_t)num_sms() * 8), 256, 0, s>>>(
          cnt, dist, s_tab, w.wtab);
    }
  }
  void *bufs[2] = {pos, w.buf};
  for (int it = 0; it < iters; ++it) {
    void *in = bufs[it & 1], *out = bufs[(it & 1) ^ 1];
    if (precision == 64)
      note_launch(), k_wsweep<double2><<<nb, kWSweepThreads, smem, s>>>(n, rowptr, colidx, elen, k, pivots, dist, s_tab,
                                                                  (const double2 *)in, (double2 *)out, w.part, w.done,
                                                                  rel_change);
    else
      note_launch(), k_wsweep_f32<<<nb, kWSweepThreads, smem, s>>>(n, rowptr, colidx, elen, k, pivots, dist, w.wtab,
                                                             (const float2 *)in, (float2 *)out, w.part, w.done,
                                                             rel_change);
  }
  if (iters & 1) SSM_TRY_CUDA(cudaMemcpyAsync(pos, w.buf, (size_t)n * esz, cudaMemcpyDeviceToDevice, s));
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
