// Max/min-sp pivot sampling (Section 4.1) inside one thread-block cluster.
//
// The sampling is a chain of k pruned BFS (expand v at level L+1 only if
// L+1 < mind[v]), each a few dozen levels deep on large-diameter graphs, so
// its cost is the latency of one level times the number of levels.  Here the
// whole chain runs in one cluster of C CTAs (C = 8 or 16):
//   * node v belongs to CTA v mod C; its mind sits in that CTA's shared
//     memory at slot v div C, so claiming a node is one DSMEM atomicMin
//     (about 0.1 us) instead of an L2 atomic.  Graphs too large for 4 bytes
//     per node keep mind in 2 bytes (distances stay below 65535 like d_ip):
//     two nodes share a 32-bit word and a claim is a DSMEM compare-and-swap
//     on it (within one level every claim writes the same value, so a word
//     changes at most twice per level and the retry loop is short);
//   * a claimed node is pushed, with its row range, into the frontier queue
//     of its owner (a DSMEM atomicAdd for the slot and a DSMEM store), so the
//     next level reads every entry from local shared memory and the levels
//     are balanced over the CTAs by node id;
//   * every CTA publishes how many nodes it pushed to all CTAs, so each one
//     knows the size of the next level; levels are separated by the hardware
//     cluster barrier (no device-wide barrier, no spin-wait);
//   * a warp takes one entry of a small level and spreads its row over its
//     lanes; larger levels give a warp up to 32 entries whose edges are
//     balanced over the lanes;
//   * the argmax of mind (ties to the lowest node id) is a scan of each
//     CTA's own slice plus an exchange of C packed keys.
// A search deeper than a 2-byte mind holds stops the kernel and leaves the
// whole selection to the grid kernel, queued behind it on the same stream.
// Queue entries beyond the shared-memory capacity go to a global spill area
// (node ids only), so any frontier size is handled.
#include <algorithm>
#include <type_traits>

#include "bfs.cuh"
#include "cluster.cuh"

namespace ssm {

#ifndef SSM_MC_THREADS
#define SSM_MC_THREADS 512
#endif
constexpr int kMcThreads = SSM_MC_THREADS;
constexpr int kMcMaxCluster = 16;
constexpr int kMcQcapMax = 8192;  // queue entries per level parity kept in shared memory
constexpr int kMcQcapMin = 1024;
#ifndef SSM_MC_U
#define SSM_MC_U 2
#endif
constexpr int kMcU = SSM_MC_U;  // edge slots per lane in flight
constexpr unsigned kMcInf = 0xFFFFFFFFu;
constexpr unsigned kMcInf16 = 0xFFFFu;
constexpr int kMcCasTries = 64;  // a claim gives up (SSM_E_TIMEOUT) after this many failed swaps

struct McArgs {
  int32_t n;
  const int32_t *rowptr;
  const int4 *adj;  // [2m] (v, rowptr[v], rowptr[v+1], 0)
  int32_t k;
  int32_t start;
  int32_t *pivots;
  int32_t *status;
  unsigned *spill;  // [C][2][n] node ids of queue entries at index >= qcap
  unsigned *fallback;  // 2-byte mind: set to 1 when a search went deeper than 65534 levels
  // non-null: the first search (from start) was run on the whole GPU: mind
  // after it, 4 bytes per node, and its packed (mind << 32 | ~node) maximum
  const unsigned *init_mind;
  const unsigned long long *init_best;
  const unsigned *init_gaveup;  // the first search stopped early: ignore init_mind and search from start
  int32_t cshift;   // C = 1 << cshift
  int32_t slots;    // shared-memory mind slots per CTA (>= ceil(n / C), multiple of 8)
  int32_t qcap;     // queue entries per parity in shared memory
};

// 2-byte mind: lowers the half h of the DSMEM word at a to nd if it is above
// nd; returns the value it held (0 when pred is false, or when the swap kept
// failing, which records SSM_E_TIMEOUT)
__device__ __forceinline__ unsigned dsmem_claim16_if(bool pred, uint32_t a, unsigned h, unsigned nd, int32_t *status) {
  if (!pred) return 0u;
  const unsigned sh = 16u * h, mask = 0xFFFFu << sh;
  unsigned w = dsmem_ld_u32(a);
  for (int t = 0; t < kMcCasTries; ++t) {
    const unsigned cur = (w & mask) >> sh;
    if (cur <= nd) return cur;
    const unsigned prev = dsmem_cas_u32(a, w, (w & ~mask) | (nd << sh));
    if (prev == w) return cur;
    w = prev;
  }
  dev_fail(status, SSM_E_TIMEOUT);
  return 0u;
}

// ----------------------------------------------------------------- kernel
struct McSmem {
  void *mind;      // [slots] hop distance to the closest chosen pivot, nodes r, r + C, ... (MB bytes each)
  int4 *q;         // [2][qcap] own frontier entries (v, rowptr[v], rowptr[v+1], 0) by level parity
  unsigned *cnts;  // [2][16] nodes pushed by every CTA, by level parity (published)
  unsigned *t3;    // [3] own queue lengths, rotating with the level (raised by the pushing CTAs)
  unsigned *p3;    // [3] nodes this CTA pushed, rotating with the level
};

// One round of kMcU edge slots per lane at level L: claim each slot's node
// (a DSMEM atomicMin on its owner's mind) and push the new ones to their
// owners' queues of level L+1.
template <int MB>
__device__ __forceinline__ void mc_round(const McArgs &A, const McSmem &S, unsigned cs, unsigned L,
                                         const int4 (&e)[kMcU], bool (&act)[kMcU]) {
  const unsigned lane = threadIdx.x & 31u, cmask = (1u << cs) - 1u, nd = L + 1u, nxt = nd & 1u;
  const unsigned n = (unsigned)A.n, qcap = (unsigned)A.qcap;
  unsigned old[kMcU];
#pragma unroll
  for (int u = 0; u < kMcU; ++u) {
    const unsigned v = (unsigned)e[u].x, slot = v >> cs;
    if constexpr (MB == 4)
      old[u] = dsmem_atomic_min_if(act[u], dsmem_addr(static_cast<unsigned *>(S.mind) + slot, v & cmask), nd);
    else
      old[u] = dsmem_claim16_if(act[u], dsmem_addr(static_cast<unsigned *>(S.mind) + (slot >> 1), v & cmask), slot & 1u,
                                nd, A.status);
  }
#pragma unroll
  for (int u = 0; u < kMcU; ++u) act[u] = act[u] && old[u] > nd;
  unsigned slot[kMcU];
#pragma unroll
  for (int u = 0; u < kMcU; ++u)
    slot[u] = dsmem_atomic_add_if(act[u], dsmem_addr(S.t3 + nd % 3u, (unsigned)e[u].x & cmask), 1u);
  unsigned pushed = 0;
#pragma unroll
  for (int u = 0; u < kMcU; ++u) {
    const unsigned v = (unsigned)e[u].x, o = v & cmask;
    if (act[u]) {
      if (slot[u] < qcap)
        dsmem_st_v4(dsmem_addr(S.q + nxt * qcap + slot[u], o), make_int4(e[u].x, e[u].y, e[u].z, 0));
      else
        A.spill[((size_t)o * 2u + nxt) * n + (slot[u] - qcap)] = v;
    }
    pushed += __popc(__ballot_sync(0xffffffffu, act[u]));
  }
  if (lane == 0 && pushed) atomicAdd(S.p3 + nd % 3u, pushed);
}

// The edges of up to 32 rows (one per lane) at level L.  With `single` only
// lane 0 holds a row and the warp walks it directly; otherwise the edges of
// all rows are spread evenly over the lanes (prefix of the degrees, each slot
// finds its row by a binary search over the lanes).
template <int MB>
__device__ __forceinline__ void mc_rows(const McArgs &A, const McSmem &S, unsigned cs, unsigned L, int beg, int end,
                                        bool single) {
  const unsigned lane = threadIdx.x & 31u;
  if (single) {
    const int b = __shfl_sync(0xffffffffu, beg, 0), en = __shfl_sync(0xffffffffu, end, 0);
    for (int base = b; base < en; base += 32 * kMcU) {
      int4 e[kMcU];
      bool act[kMcU];
#pragma unroll
      for (int u = 0; u < kMcU; ++u) {
        const int idx = base + 32 * u + (int)lane;
        act[u] = idx < en;
        e[u] = act[u] ? __ldg(A.adj + idx) : make_int4(0, 0, 0, 0);
      }
      mc_round<MB>(A, S, cs, L, e, act);
    }
    return;
  }
  int incl = end - beg;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += t;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  for (int base = 0; base < total; base += 32 * kMcU) {
    int4 e[kMcU];
    bool act[kMcU];
#pragma unroll
    for (int u = 0; u < kMcU; ++u) {
      const int idx = base + 32 * u + (int)lane;
      act[u] = idx < total;
      int lo = 0;  // row = first lane whose inclusive prefix exceeds idx
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int pv = __shfl_sync(0xffffffffu, incl, lo + step - 1);
        if (pv <= idx) lo += step;
      }
      const int own = lo > 31 ? 31 : lo;
      const int o_end = __shfl_sync(0xffffffffu, end, own);
      const int o_incl = __shfl_sync(0xffffffffu, incl, own);
      e[u] = act[u] ? __ldg(A.adj + o_end - (o_incl - idx)) : make_int4(0, 0, 0, 0);
    }
    mc_round<MB>(A, S, cs, L, e, act);
  }
}

// Expands this CTA's queue of level L (cnt entries).  A warp takes ipw
// consecutive entries, ipw a power of two chosen so that small levels are
// spread over all warps.
template <int MB>
__device__ __forceinline__ void mc_expand(const McArgs &A, const McSmem &S, unsigned r, unsigned cs, unsigned L,
                                          unsigned cnt) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const unsigned cur = L & 1u, n = (unsigned)A.n, qcap = (unsigned)A.qcap;
  unsigned ipw = 1;
  while (ipw < 32u && ipw * nwarps < cnt) ipw <<= 1;
  for (unsigned base = warp * ipw; base < cnt; base += nwarps * ipw) {
    const unsigned idx = base + lane;
    int beg = 0, end = 0;
    if (lane < ipw && idx < cnt) {
      if (idx < qcap) {
        const int4 e = S.q[cur * qcap + idx];
        beg = e.y;
        end = e.z;
      } else {
        const unsigned v = __ldcg(A.spill + ((size_t)r * 2u + cur) * n + (idx - qcap));
        beg = __ldg(A.rowptr + v);
        end = __ldg(A.rowptr + v + 1);
      }
    }
    mc_rows<MB>(A, S, cs, L, beg, end, ipw == 1u);
  }
}

// MB: bytes of mind per node (4, or 2 for graphs whose 4-byte mind does not fit)
template <int MB>
__global__ void __launch_bounds__(kMcThreads, 1) k_maxmin_cluster(McArgs A) {
  extern __shared__ __align__(16) unsigned char mc_smem[];
  __shared__ unsigned s_t3[3], s_p3[3];
  __shared__ unsigned long long s_wbest[kMcThreads / 32];
  using MindT = typename std::conditional<MB == 4, unsigned, unsigned short>::type;
  constexpr unsigned kInfM = MB == 4 ? kMcInf : kMcInf16;
  McSmem S;
  MindT *mind = reinterpret_cast<MindT *>(mc_smem);
  S.mind = mind;
  S.q = reinterpret_cast<int4 *>(mc_smem + (size_t)MB * A.slots);
  S.cnts = reinterpret_cast<unsigned *>(S.q + 2 * (size_t)A.qcap);
  S.t3 = s_t3;
  S.p3 = s_p3;
  unsigned long long *bests = reinterpret_cast<unsigned long long *>(S.cnts + 32);  // [16] published maxima

  const unsigned cs = (unsigned)A.cshift, C = 1u << cs, cmask = C - 1u;
  const unsigned r = cluster_rank();
  const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const unsigned n = (unsigned)A.n;
  const unsigned own = n > r ? ((n - 1u - r) >> cs) + 1u : 0u;  // nodes r, r + C, ... below n

  // the level counters of the next search, reset before the cluster barrier
  // that precedes it: from that barrier on another CTA may push into this
  // one's queue (level 0 publishes a total of 1: the pivot)
  auto reset_search = [&]() {
    if (tid < (unsigned)kMcMaxCluster) S.cnts[tid] = (tid == 0) ? 1u : 0u;
    if (tid == 0) {
      s_t3[0] = s_t3[1] = s_t3[2] = 0;
      s_p3[0] = s_p3[1] = s_p3[2] = 0;
    }
  };
  unsigned p = (unsigned)A.start;
  int j0 = 0;
  if (A.init_mind && __ldcg(A.init_gaveup) == 0u) {
    // the search from start ran on the whole GPU (it reaches every node, and
    // a grid of all SMs does that faster than one cluster): take its mind
    // and its maximum, which is pivot 1 (uniform: every CTA reads the same key)
    const unsigned long long key0 = __ldcg(A.init_best);
    const unsigned top = (unsigned)(key0 >> 32);
    if (top == kMcInf) goto done;  // unreachable nodes: already recorded by that search
    if (MB == 2 && top >= kMcInf16) {  // deeper than a 2-byte mind holds: the grid kernel takes over
      if (r == 0 && tid == 0) *A.fallback = 1u;
      goto done;
    }
    for (unsigned s = tid; s < own; s += blockDim.x) mind[s] = (MindT)__ldcg(A.init_mind + r + (s << cs));
    p = ~(unsigned)key0;
    j0 = 1;
  } else {
    for (unsigned s = tid; s < own; s += blockDim.x) mind[s] = (MindT)kInfM;
  }
  reset_search();
  cluster_sync();  // every CTA of the cluster runs before any DSMEM access

  for (int j = j0; j < A.k; ++j) {
    if (r == 0 && tid == 0) A.pivots[j] = (int32_t)p;
    const bool last = (j == A.k - 1);
    if (last && j > 0) break;  // the final pivot needs no search

    // level 0: the queue of p's owner holds p.  Only the owner expands level 0,
    // and every CTA finished reading mind (the last argmax) before the barrier
    // that ended the previous search, so no cluster barrier is needed here
    if (tid == 0 && r == (p & cmask)) {
      mind[p >> cs] = 0;
      S.q[0] = make_int4((int)p, __ldg(A.rowptr + p), __ldg(A.rowptr + p + 1), 0);
      s_t3[0] = 1;
    }
    __syncthreads();

    for (unsigned L = 0;; ++L) {
      unsigned tot = lane < C ? S.cnts[(L & 1u) * 16u + lane] : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
      if (tot == 0) break;  // same published counts in every CTA: uniform
      if (MB == 2 && L + 1u >= kMcInf16) {  // a 2-byte mind cannot hold the next level (uniform):
        if (r == 0 && tid == 0) *A.fallback = 1u;  // the grid kernel queued after this one takes over
        goto done;
      }
      const unsigned cnt = s_t3[L % 3u];
      if (tid == 0) {
        s_t3[(L + 2u) % 3u] = 0;  // read during level L-1; raised again from level L+1 on
        s_p3[(L + 2u) % 3u] = 0;
      }
      mc_expand<MB>(A, S, r, cs, L, cnt);
      __syncthreads();  // own push count is final
      if (tid < C) dsmem_st_u32(dsmem_addr(S.cnts + ((L + 1u) & 1u) * 16u + r, tid), s_p3[(L + 1u) % 3u]);
      cluster_sync();
    }

    // argmax of mind over the cluster, ties to the lowest node id: a thread
    // takes 16 bytes of slots at a time, keeps the first chunk whose largest
    // value (a packed maximum) beats what it saw, and then the first slot of
    // that chunk holding it (chunks ascending, so that is its lowest node id);
    // a chunk that runs past the last owned slot is taken slot by slot
    unsigned long long key = 0;
    {
      constexpr unsigned kPer = 16u / MB;  // slots per 16-byte load (slots is a multiple of 8)
      const uint4 *chunks = reinterpret_cast<const uint4 *>(mind);
      auto slot_val = [&](const uint4 &w, unsigned e) -> unsigned {
        const unsigned wd = e / (4u / MB) == 0 ? w.x : e / (4u / MB) == 1 ? w.y : e / (4u / MB) == 2 ? w.z : w.w;
        return MB == 4 ? wd : (wd >> (16u * (e & 1u))) & 0xFFFFu;
      };
      unsigned bv = 0, bc = 0;
      bool any = false;
      for (unsigned c = tid; c * kPer < own; c += blockDim.x) {
        const uint4 w = chunks[c];
        unsigned v;
        if ((c + 1u) * kPer <= own) {
          if (MB == 2) {
            const unsigned m = __vmaxu2(__vmaxu2(w.x, w.y), __vmaxu2(w.z, w.w));
            v = max(m & 0xFFFFu, m >> 16);
          } else {
            v = max(max(w.x, w.y), max(w.z, w.w));
          }
        } else {
          v = 0;
          for (unsigned e = 0; c * kPer + e < own; ++e) v = max(v, slot_val(w, e));
        }
        if (!any || v > bv) {
          bv = v;
          bc = c;
          any = true;
        }
      }
      if (any) {
        const uint4 w = chunks[bc];
        unsigned e = 0;
        while (bc * kPer + e < own && slot_val(w, e) != bv) ++e;  // the value is in the chunk
        key = ((unsigned long long)bv << 32) | (unsigned long long)(~(r + ((bc * kPer + e) << cs)));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, key, o);
      key = t > key ? t : key;
    }
    if (lane == 0) s_wbest[warp] = key;
    __syncthreads();
    if (warp == 0) {
      key = lane < nwarps ? s_wbest[lane] : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, key, o);
        key = t > key ? t : key;
      }
      if (lane < C) dsmem_st_u64(dsmem_addr(bests + r, lane), key);
    }
    reset_search();  // the level loop is over in every CTA (it ended at a cluster barrier)
    cluster_sync();
    key = 0;
    for (unsigned x = 0; x < C; ++x) key = bests[x] > key ? bests[x] : key;
    if ((unsigned)(key >> 32) == kInfM) {  // some node was never reached
      if (r == 0 && tid == 0) dev_fail(A.status, SSM_E_DISCONNECTED);
      break;
    }
    if (last) break;
    p = ~(unsigned)key;
  }
done:
  cluster_sync();  // no CTA leaves while another may still read its shared memory
}

// ------------------------------------------------------------------- host
struct McShape {
  int C = 0;
  int mb = 4;  // bytes of mind per node
  int slots = 0;
  int qcap = 0;
  size_t smem = 0;
};

static size_t mc_smem_bytes(int slots, int qcap, int mb) {
  return (size_t)slots * mb + (size_t)2 * qcap * sizeof(int4) + 32 * 4 + kMcMaxCluster * 8;
}

static const void *mc_kernel(int mb) {
  return mb == 4 ? (const void *)k_maxmin_cluster<4> : (const void *)k_maxmin_cluster<2>;
}

// Cluster shape for n nodes on the current device (16 CTAs before 8, 4-byte
// mind before 2-byte), or C == 0 if no cluster of up to 16 CTAs holds mind in
// shared memory.
static McShape mc_shape(int32_t n) {
  McShape sh;
  int dev = 0, smem_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return sh;
  if (cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return sh;
  const size_t budget = (size_t)smem_max - 2 * 1024;  // static shared memory of the kernel
  for (int C : {16, 8}) {
    for (int mb : {4, 2}) {
      const void *kern = mc_kernel(mb);
      // a multiple of 8 slots keeps the queue after mind 16-byte aligned
      const int slots = (int)((((int64_t)n + C - 1) / C + 7) / 8 * 8);
      const size_t fixed = mc_smem_bytes(slots, 0, mb);
      if (fixed >= budget) continue;
      const int qcap = (int)std::min<size_t>(kMcQcapMax, (budget - fixed) / (2 * sizeof(int4)));
      if (qcap < kMcQcapMin) continue;
      const size_t smem = mc_smem_bytes(slots, qcap, mb);
      if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        (void)cudaGetLastError();
        continue;
      }
      if (allow_dynamic_smem(kern) != cudaSuccess) {
        (void)cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)C);
      cfg.blockDim = dim3(kMcThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        continue;
      }
      if (clusters < 1) continue;
      sh.C = C;
      sh.mb = mb;
      sh.slots = slots;
      sh.qcap = qcap;
      sh.smem = smem;
      return sh;
    }
  }
  return sh;
}

bool maxmin_cluster_candidate(int32_t n) {
  // mind of 2 bytes per node over at most 16 CTAs, with room for the queues
  return (int64_t)n * 2 <= (int64_t)kMcMaxCluster * 190 * 1024;
}

size_t maxmin_cluster_spill_entries(int32_t n) {
  return maxmin_cluster_candidate(n) ? (size_t)kMcMaxCluster * 2 * (size_t)n : 0;
}

// what the last pivot selection on this host thread chose (ssm_last_pivot_config)
static thread_local int32_t g_last_pivot_config[2] = {-1, 0};

void note_pivot_config(int32_t cluster, int32_t mind_bytes) {
  g_last_pivot_config[0] = cluster;
  g_last_pivot_config[1] = mind_bytes;
}

int maxmin_cluster_mind_bytes(int32_t n) {
  if (!maxmin_cluster_candidate(n)) return 0;
  const McShape sh = mc_shape(n);
  return sh.C ? sh.mb : 0;
}

int launch_maxmin_cluster(int32_t n, const int32_t *rowptr, const int4 *adj, int32_t k, int32_t start,
                          int32_t *pivots, int32_t *status, unsigned *spill, unsigned *fallback,
                          const unsigned *init_mind, const unsigned long long *init_best,
                          const unsigned *init_gaveup, cudaStream_t s, int *mind_bytes) {
  *mind_bytes = 0;
  if (!maxmin_cluster_candidate(n)) return SSM_OK;
  const McShape sh = mc_shape(n);
  if (sh.C == 0) return SSM_OK;
  McArgs A;
  A.n = n; A.rowptr = rowptr; A.adj = adj; A.k = k; A.start = start; A.pivots = pivots; A.status = status;
  A.spill = spill;
  A.fallback = fallback;
  A.init_mind = init_mind;
  A.init_best = init_best;
  A.init_gaveup = init_gaveup;
  A.cshift = sh.C == 16 ? 4 : 3;
  A.slots = sh.slots;
  A.qcap = sh.qcap;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)sh.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)sh.C);
  cfg.blockDim = dim3(kMcThreads);
  cfg.dynamicSmemBytes = sh.smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (sh.mb == 2) SSM_TRY_CUDA(cudaMemsetAsync(fallback, 0, sizeof(unsigned), s));
  note_launch();
  if (sh.mb == 4)
    SSM_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_maxmin_cluster<4>, A));
  else
    SSM_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_maxmin_cluster<2>, A));
  *mind_bytes = sh.mb;
  note_pivot_config(sh.C, sh.mb);
  return SSM_OK;
}

}  // namespace ssm

SSM_API void ssm_last_pivot_config(int32_t *out) {
  out[0] = ssm::g_last_pivot_config[0];
  out[1] = ssm::g_last_pivot_config[1];
}
