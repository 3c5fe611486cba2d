// Breadth-first searches on the device:
//   * ssm_select_pivots: max/min-sp pivot sampling (Section 4.1), one pruned
//     level-synchronous BFS per new pivot inside one cooperative persistent
//     kernel; small frontiers are expanded by one block without device-wide
//     barriers, large ones by the whole grid;
//   * ssm_pivot_bfs:     all k pivot distances d_ip (Algorithm 1 line 2): one
//     block per source with the visited set as a bitmap in shared memory
//     (k_bfs_cta), or, for graphs whose bitmap does not fit, one multi-source
//     BFS over per-node bitsets with one bit per source (k_msbfs).
// Frontier appends are compacted with warp ballots; every device-wide wait is
// bounded (SSM_E_TIMEOUT).
#include <algorithm>

#include "bfs.cuh"

namespace ssm {

constexpr int kBfsThreads = 512;
constexpr unsigned kInf = 0xFFFFFFFFu;

// --------------------------------------------------------------------------
// one BFS level expanded by one block
// --------------------------------------------------------------------------
constexpr int kFlatChunk = 2048;  // frontier nodes whose degree prefix sits in shared memory
constexpr int kFlatU = 8;         // adjacency loads in flight per thread

struct FlatSmem {
  unsigned pref[kFlatChunk + 1];  // exclusive prefix of the chunk's degrees
  int rb[kFlatChunk];             // row begin of each chunk node
  unsigned warp_tot[32];
  unsigned total;
};

// exclusive prefix of v over the block (blockDim.x <= 1024); the block total lands in S.total
__device__ __forceinline__ unsigned block_scan_excl(unsigned v, FlatSmem &S) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = (blockDim.x + 31u) >> 5;
  unsigned incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += t;
  }
  if (lane == 31) S.warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned w = lane < nw ? S.warp_tot[lane] : 0u;
    unsigned wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= (unsigned)o) wi += t;
    }
    if (lane < nw) S.warp_tot[lane] = wi - w;
    if (lane == 31) S.total = wi;
  }
  __syncthreads();
  return incl - v + S.warp_tot[warp];
}

// One BFS level by one block.  fr(i) gives the row range of frontier node i
// (i < cc).  The frontier is taken in chunks of kFlatChunk nodes: a prefix of
// their degrees goes to shared memory, then all edge slots of the chunk are
// spread evenly over the block's threads, kFlatU independent 16-byte
// adjacency loads in flight per thread (one latency per kFlatU slots, not one
// per 32-slot round of a warp).  gather(e) claims neighbour e.x and returns
// whether it is new; emit(e, claimed) runs for every slot with the whole
// warp converged (appends use warp ballots).  Every thread of the block must
// call this with the same cc.
template <class Fr, class Gather, class Emit>
__device__ void block_expand_level(Fr &&fr, unsigned cc, const int4 *__restrict__ adj, FlatSmem &S, Gather &&gather,
                                   Emit &&emit) {
  const unsigned tid = threadIdx.x, nth = blockDim.x;
  for (unsigned c0 = 0; c0 < cc; c0 += kFlatChunk) {
    const unsigned cn = min((unsigned)kFlatChunk, cc - c0);
    const unsigned per = (cn + nth - 1) / nth;  // <= kFlatChunk / 32
    unsigned mine = 0;
    for (unsigned j = 0; j < per; ++j) {
      const unsigned i = tid * per + j;
      if (i < cn) {
        const int2 r = fr(c0 + i);
        S.rb[i] = r.x;
        mine += (unsigned)(r.y - r.x);
      }
    }
    unsigned off = block_scan_excl(mine, S);
    for (unsigned j = 0; j < per; ++j) {
      const unsigned i = tid * per + j;
      if (i < cn) {
        S.pref[i] = off;
        off += (unsigned)(fr(c0 + i).y - S.rb[i]);
      }
    }
    if (tid == 0) S.pref[cn] = S.total;
    __syncthreads();
    const unsigned E = S.pref[cn];
    for (unsigned base = 0; base < E; base += nth * kFlatU) {
      int4 e[kFlatU];
      bool act[kFlatU];
#pragma unroll
      for (int u = 0; u < kFlatU; ++u) {
        const unsigned t = base + (unsigned)u * nth + tid;
        act[u] = t < E;
        e[u] = make_int4(0, 0, 0, 0);
        if (act[u]) {
          unsigned lo = 0;  // largest i with pref[i] <= t
#pragma unroll
          for (unsigned step = kFlatChunk / 2; step > 0; step >>= 1)
            if (lo + step <= cn && S.pref[lo + step] <= t) lo += step;
          e[u] = __ldg(adj + S.rb[lo] + (int)(t - S.pref[lo]));
        }
      }
#pragma unroll
      for (int u = 0; u < kFlatU; ++u) act[u] = act[u] && gather(e[u]);
#pragma unroll
      for (int u = 0; u < kFlatU; ++u) emit(e[u], act[u]);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// max/min sp
// --------------------------------------------------------------------------
constexpr int kSoloMax = 2048;       // frontiers up to this size are expanded by block 0 alone
constexpr int kFirstSearchLevels = 16;  // depth up to which a cluster run's first search stays on the grid
constexpr int kSoloLevels = 4096;    // block 0 hands back to the grid at least this often

struct MaxMinArgs {
  int32_t n;
  const int32_t *rowptr;
  const int32_t *colidx;
  int32_t k;
  int32_t start;
  int32_t *pivots;
  int32_t *status;
  const int4 *adj;  // [2m] edge-expanded adjacency (v, rowptr[v], rowptr[v+1], 0)
  unsigned *mind;  // [n] hop distance to the closest chosen pivot
  unsigned *q0, *q1;  // [n] frontier queues (alternate by level parity)
  unsigned *qcnt;     // [3] queue lengths, rotated by level
  unsigned *level;    // level reached by a solo phase of block 0
  unsigned long long *best;  // [2] packed (mind << 32 | ~node) maxima, by pivot parity
  BarrierState *bar;
  const unsigned *run_if;  // non-null: run only if *run_if != 0 (the cluster kernel gave the search up)
  // the first search of a cluster run (k_first_search): at most max_levels
  // levels, else *gave_up (a deep graph is searched faster by the cluster itself)
  int32_t max_levels;
  unsigned *gave_up;
  unsigned *fb;     // [kFirstSearchLevels + 1][fbw] frontier bitmaps, one per level (zeroed by the caller)
  size_t fbw;       // words per bitmap (whole 128-byte rows)
  unsigned *lcnt;   // [kFirstSearchLevels + 2] nodes first reached at each level (zeroed by the caller)
  unsigned *nlong;  // rows above kFirstLong entries, listed in q0 (zeroed by the caller)
};

// Block 0 alone expands levels L, L+1, ... while the frontier has at most
// kSoloMax nodes: row ranges of the frontier stay in shared memory and the
// levels are separated by __syncthreads instead of device-wide barriers.
// Every new frontier is also written to the global queue, so the grid can
// take over when it grows.  Returns with qcnt and *level describing the
// frontier it stopped at.
__device__ void maxmin_solo(const MaxMinArgs &A, unsigned L, unsigned c, int2 (*sq)[kSoloMax], unsigned *s_cnt,
                            FlatSmem &S) {
  const unsigned *qin0 = (L & 1) ? A.q1 : A.q0;
  for (unsigned e = threadIdx.x; e < c; e += blockDim.x) {
    const unsigned u = __ldcg(qin0 + e);
    sq[0][e] = make_int2(__ldg(A.rowptr + u), __ldg(A.rowptr + u + 1));
  }
  if (threadIdx.x == 0) {
    s_cnt[0] = c;
    s_cnt[1] = 0;
  }
  __syncthreads();
  int cur = 0;
  for (int steps = 0; steps < kSoloLevels; ++steps) {
    const unsigned cc = s_cnt[cur];
    if (cc == 0 || cc > (unsigned)kSoloMax) break;
    const int nxt = cur ^ 1;
    unsigned *qout = ((L + 1) & 1) ? A.q1 : A.q0;
    const unsigned nd = L + 1;
    const int2 *fr = sq[cur];
    block_expand_level(
        [&](unsigned i) { return fr[i]; }, cc, A.adj, S,
        [&](int4 ed) { return atomicMin(A.mind + ed.x, nd) > nd; },
        [&](int4 ed, bool push) {
          const unsigned pos = warp_slot(push, s_cnt + nxt);
          if (push) {
            qout[pos] = (unsigned)ed.x;
            if (pos < (unsigned)kSoloMax) sq[nxt][pos] = make_int2(ed.y, ed.z);
          }
        });
    if (threadIdx.x == 0) s_cnt[cur] = 0;
    __syncthreads();
    cur = nxt;
    ++L;
  }
  if (threadIdx.x == 0) {
    A.qcnt[L % 3] = s_cnt[cur];
    A.qcnt[(L + 1) % 3] = 0;
    A.qcnt[(L + 2) % 3] = 0;
    *A.level = L;
  }
}

// Pruned BFS from the newest pivot p: node v is expanded at level L+1 only
// if L+1 < mind[v].  Since mind (a minimum of distance functions) changes by
// at most 1 along an edge, every node whose distance to p is below its old
// mind is reached along a shortest path of such nodes, so the result is
// exactly mind = min(mind, d(p, .)).
__global__ void __launch_bounds__(kBfsThreads) k_maxmin(MaxMinArgs A) {
  extern __shared__ __align__(16) unsigned char mm_smem[];
  int2 (*sq)[kSoloMax] = reinterpret_cast<int2 (*)[kSoloMax]>(mm_smem);
  FlatSmem &S = *reinterpret_cast<FlatSmem *>(mm_smem + sizeof(int2) * 2 * kSoloMax);
  __shared__ unsigned s_cnt[2];
  const unsigned nthreads = gridDim.x * blockDim.x;
  const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gwarp = gtid >> 5, nwarps = nthreads >> 5;
  const unsigned n = (unsigned)A.n;
  if (A.run_if && __ldcg(A.run_if) == 0u) return;  // every block, before any barrier

  for (unsigned v = gtid; v < n; v += nthreads) A.mind[v] = kInf;
  if (!grid_barrier(A.bar, A.status)) return;

  unsigned p = (unsigned)A.start;
  for (int j = 0; j < A.k; ++j) {
    if (gtid == 0) {
      A.pivots[j] = (int32_t)p;
      A.mind[p] = 0;
      A.q0[0] = p;
      A.qcnt[0] = 1;
      A.qcnt[1] = 0;
      A.qcnt[2] = 0;
    }
    const bool last = (j == A.k - 1);
    if (last && j > 0) break;  // the final pivot needs no search
    // level 0 is the pivot alone: block 0 seeded it and expands it (and the
    // levels after it while they stay small) on its own, so the other blocks
    // need not see the seed and go straight to the barrier after that phase
    if (blockIdx.x == 0) {
      __syncthreads();
      maxmin_solo(A, 0, 1, sq, s_cnt, S);
    }
    if (!grid_barrier(A.bar, A.status)) return;

    for (unsigned L = __ldcg(A.level);;) {
      const unsigned c = __ldcg(A.qcnt + L % 3);
      if (c == 0) break;
      if (c <= (unsigned)kSoloMax) {
        if (blockIdx.x == 0) maxmin_solo(A, L, c, sq, s_cnt, S);
        if (!grid_barrier(A.bar, A.status)) return;
        L = __ldcg(A.level);
        continue;
      }
      if (gtid == 0) A.qcnt[(L + 2) % 3] = 0;
      const unsigned *qin = (L & 1) ? A.q1 : A.q0;
      unsigned *qout = (L & 1) ? A.q0 : A.q1;
      unsigned *cout = A.qcnt + (L + 1) % 3;
      const unsigned nd = L + 1;
      for (unsigned base = gwarp * 32u; base < c; base += nwarps * 32u) {
        const unsigned e = base + lane;
        int beg = 0, end = 0;
        if (e < c) {
          const unsigned u = __ldcg(qin + e);
          beg = __ldg(A.rowptr + u);
          end = __ldg(A.rowptr + u + 1);
        }
        warp_for_each_neighbor(beg, end, A.colidx, [&](int, bool act, int v) {
          bool push = false;
          if (act && nd < __ldcg(A.mind + v)) {
            const unsigned old = atomicMin(A.mind + v, nd);
            push = old > nd;
          }
          warp_append(push, (unsigned)v, qout, cout);
        });
      }
      if (!grid_barrier(A.bar, A.status)) return;
      ++L;
    }

    // argmax of mind, ties to the lowest node id
    unsigned long long key = 0;
    for (unsigned v = gtid; v < n; v += nthreads) {
      const unsigned long long kk = ((unsigned long long)__ldcg(A.mind + v) << 32) | (unsigned long long)(~v);
      key = kk > key ? kk : key;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, key, o);
      key = t > key ? t : key;
    }
    if (lane == 0) atomicMax(A.best + (j & 1), key);
    if (!grid_barrier(A.bar, A.status)) return;
    key = __ldcg(A.best + (j & 1));
    if (gtid == 0) A.best[(j + 1) & 1] = 0;
    if ((unsigned)(key >> 32) == kInf) {  // some node was never reached
      if (gtid == 0) dev_fail(A.status, SSM_E_DISCONNECTED);
      return;
    }
    if (last) break;
    p = ~(unsigned)key;
  }
}

// The first search of a cluster run (from start, over every node, at most
// kFirstSearchLevels levels) as a BFS pulled level by level: every node not
// reached yet scans its row for a neighbour in level L's frontier and stops
// at the first one, so a level costs about one edge per new node where a
// pushed expansion touches every edge of the frontier (small-world graphs:
// levels of up to most of the graph).  The frontier of level L is a bitmap of
// its own, written (by atomics, in L2) during level L - 1 and read from level
// L on, so it can be read through L1.  Rows above kFirstLong entries are
// scanned by a whole warp after the short rows of the level.  Writes mind
// (= d(start, .)), pivots[0] = start and best[0] (the packed maximum), or sets
// *gave_up when the search needs more levels, or when its first kFirstProbe
// levels reached less than 1/64 of the nodes (a large diameter: the cluster
// kernel, whose levels cost less, then searches from start itself).
constexpr int kFirstLong = 64;
constexpr unsigned kFirstProbe = 6;
__global__ void __launch_bounds__(kBfsThreads) k_first_search(MaxMinArgs A) {
  const unsigned nthreads = gridDim.x * blockDim.x;
  const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gwarp = gtid >> 5, nwarps = nthreads >> 5;
  const unsigned n = (unsigned)A.n, start = (unsigned)A.start;
  for (unsigned base = gwarp * 32u; base < n; base += nwarps * 32u) {  // uniform per warp
    const unsigned v = base + lane;
    if (v < n) A.mind[v] = v == start ? 0u : kInf;
    warp_append(v < n && __ldg(A.rowptr + v + 1) - __ldg(A.rowptr + v) > kFirstLong, v, A.q0, A.nlong);
  }
  if (gtid == 0) {
    A.pivots[0] = (int32_t)start;
    atomicOr(A.fb + (start >> 5), 1u << (start & 31u));
    A.lcnt[0] = 1u;
  }
  if (!grid_barrier(A.bar, A.status)) return;
  const unsigned nlong = __ldcg(A.nlong);
  for (unsigned L = 0;; ++L) {
    if (__ldcg(A.lcnt + L) == 0u) break;  // the same count in every thread: uniform
    unsigned reached = 0;
    if (L == kFirstProbe)
      for (unsigned l = 0; l <= L; ++l) reached += __ldcg(A.lcnt + l);
    if (L >= (unsigned)A.max_levels || (L == kFirstProbe && 64ull * reached < (unsigned long long)n)) {
      if (gtid == 0) *A.gave_up = 1u;
      return;
    }
    const unsigned *fbc = A.fb + (size_t)L * A.fbw;
    unsigned *fbn = A.fb + (size_t)(L + 1u) * A.fbw;
    unsigned found = 0;
    for (unsigned base = gwarp * 32u; base < n; base += nwarps * 32u) {
      const unsigned v = base + lane;
      bool hit = false;
      if (v < n && __ldcg(A.mind + v) == kInf) {
        const int rb = __ldg(A.rowptr + v), re = __ldg(A.rowptr + v + 1);
        if (re - rb <= kFirstLong)
          for (int e = rb; e < re && !hit; e += 4) {
            unsigned u[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) u[q] = e + q < re ? (unsigned)__ldg(A.colidx + e + q) : kInf;
#pragma unroll
            for (int q = 0; q < 4; ++q) hit |= u[q] != kInf && ((fbc[u[q] >> 5] >> (u[q] & 31u)) & 1u);
          }
        if (hit) A.mind[v] = L + 1u;
      }
      const unsigned bits = __ballot_sync(0xffffffffu, hit);
      if (lane == 0 && bits) {
        atomicOr(fbn + (base >> 5), bits);
        found += __popc(bits);
      }
    }
    // the long rows, a warp each, 32 entries at a time
    for (unsigned li = gwarp; li < nlong; li += nwarps) {
      const unsigned v = __ldcg(A.q0 + li);
      if (__ldcg(A.mind + v) != kInf) continue;  // warp-uniform
      const int rb = __ldg(A.rowptr + v), re = __ldg(A.rowptr + v + 1);
      bool hit = false;
      for (int e = rb; e < re && !hit; e += 32) {
        const int t = e + (int)lane;
        const unsigned u = t < re ? (unsigned)__ldg(A.colidx + t) : kInf;
        hit = __any_sync(0xffffffffu, u != kInf && ((fbc[u >> 5] >> (u & 31u)) & 1u));
      }
      if (hit && lane == 0) {
        A.mind[v] = L + 1u;
        atomicOr(fbn + (v >> 5), 1u << (v & 31u));
        ++found;
      }
    }
    found = __reduce_add_sync(0xffffffffu, found);
    if (lane == 0 && found) atomicAdd(A.lcnt + L + 1u, found);
    if (!grid_barrier(A.bar, A.status)) return;
  }
  // argmax of mind, ties to the lowest node id
  unsigned long long key = 0;
  for (unsigned v = gtid; v < n; v += nthreads) {
    const unsigned long long kk = ((unsigned long long)__ldcg(A.mind + v) << 32) | (unsigned long long)(~v);
    key = kk > key ? kk : key;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, key, o);
    key = t > key ? t : key;
  }
  if (lane == 0) atomicMax(A.best, key);
  if (!grid_barrier(A.bar, A.status)) return;
  if (gtid == 0 && (unsigned)(__ldcg(A.best) >> 32) == kInf) dev_fail(A.status, SSM_E_DISCONNECTED);
}

// adj[t] = (colidx[t], rowptr[colidx[t]], rowptr[colidx[t] + 1], 0)
__global__ void k_expand_adj(int64_t m2, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                             int4 *__restrict__ adj) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m2; t += (int64_t)gridDim.x * blockDim.x) {
    const int v = __ldg(colidx + t);
    adj[t] = make_int4(v, __ldg(rowptr + v), __ldg(rowptr + v + 1), 0);
  }
}

static int expand_adj(int64_t m2, const int32_t *rowptr, const int32_t *colidx, int4 *adj, cudaStream_t s) {
  if (m2 <= 0) return SSM_OK;
  const int blocks = (int)std::min<int64_t>((m2 + 255) / 256, (int64_t)num_sms() * 8);
  note_launch(), k_expand_adj<<<blocks, 256, 0, s>>>(m2, rowptr, colidx, adj);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

static void carve_maxmin(Carver &c, MaxMinArgs &A, unsigned **spill, int32_t n, int64_t m2) {
  A.adj = c.take<int4>((size_t)(m2 > 0 ? m2 : 1));
  A.mind = c.take<unsigned>(n);
  A.q0 = c.take<unsigned>(n);
  A.q1 = c.take<unsigned>(n);
  A.qcnt = c.take<unsigned>(4);
  A.level = c.take<unsigned>(1);
  A.best = c.take<unsigned long long>(2);
  A.bar = c.take<BarrierState>(1);
  *spill = c.take<unsigned>(std::max<size_t>(1, maxmin_cluster_spill_entries(n)));
  A.run_if = c.take<unsigned>(1);
  A.gave_up = c.take<unsigned>(1);
  A.fbw = (((size_t)n + 1023) / 1024) * 32;
  A.fb = c.take<unsigned>(A.fbw * (kFirstSearchLevels + 1));
  A.lcnt = c.take<unsigned>(kFirstSearchLevels + 2);
  A.nlong = c.take<unsigned>(1);
}

// the cooperative grid kernel, after resetting its counters and barrier
static int launch_maxmin_grid(MaxMinArgs A, cudaStream_t s) {
  SSM_TRY_CUDA(cudaMemsetAsync(A.qcnt, 0, 4 * sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(A.best, 0, 2 * sizeof(unsigned long long), s));
  if (int rc_ = reset_barrier(A.bar, s)) return rc_;
  const size_t smem = sizeof(int2) * 2 * kSoloMax + sizeof(FlatSmem);
  SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_maxmin));
  const int blocks = cooperative_blocks((const void *)k_maxmin, kBfsThreads, smem, 1);
  if (blocks < 1) return fail(SSM_E_CUDA, "max/min pivots: kernel cannot be resident");
  void *args[] = {&A};
  note_launch();
  SSM_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)k_maxmin, dim3(blocks), dim3(kBfsThreads), args, smem, s));
  return SSM_OK;
}

// the first search of a cluster run (k_first_search), after zeroing its state
static int launch_first_search(MaxMinArgs A, cudaStream_t s) {
  SSM_TRY_CUDA(cudaMemsetAsync(A.best, 0, sizeof(unsigned long long), s));
  SSM_TRY_CUDA(cudaMemsetAsync(A.fb, 0, A.fbw * (kFirstSearchLevels + 1) * sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(A.lcnt, 0, (kFirstSearchLevels + 2) * sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(A.nlong, 0, sizeof(unsigned), s));
  if (int rc_ = reset_barrier(A.bar, s)) return rc_;
  const int blocks = cooperative_blocks((const void *)k_first_search, kBfsThreads, 0, 2);
  if (blocks < 1) return fail(SSM_E_CUDA, "max/min pivots: first search cannot be resident");
  void *args[] = {&A};
  note_launch();
  SSM_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)k_first_search, dim3(blocks), dim3(kBfsThreads), args, 0, s));
  return SSM_OK;
}

// Graphs whose mind fits a cluster: the first search (from start, over every
// node) pulled on the whole grid, the other k - 1 searches (pruned, mostly small)
// in the cluster; with a 2-byte mind the full grid selection is queued behind
// them and runs only if the cluster handed over (a search deeper than 65534
// levels).  Other graphs: the grid kernel alone.
int launch_maxmin(int32_t n, int64_t m2, const int32_t *rowptr, const int32_t *colidx, int32_t k, int32_t start,
                  int32_t *pivots, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  Carver c(ws, ws_bytes);
  MaxMinArgs A;
  A.n = n; A.rowptr = rowptr; A.colidx = colidx; A.k = k; A.start = start;
  A.pivots = pivots; A.status = status;
  unsigned *spill = nullptr;
  carve_maxmin(c, A, &spill, n, m2);
  if (!c.ok) return fail(SSM_E_NOMEM, "max/min pivots: workspace %zu bytes, need %zu", ws_bytes, c.size());
  int rc = expand_adj(m2, rowptr, colidx, const_cast<int4 *>(A.adj), s);
  if (rc) return rc;
  unsigned *fallback = const_cast<unsigned *>(A.run_if);
  A.run_if = nullptr;
  A.max_levels = 0;
  if (k >= 2 && maxmin_cluster_mind_bytes(n) > 0) {
    // the first search on the grid while it stays within kFirstSearchLevels
    // levels (small-world graphs: few levels of up to all nodes); deeper
    // graphs leave it to the cluster, whose levels cost less
    MaxMinArgs first = A;
    first.k = 1;
    first.max_levels = kFirstSearchLevels;
    SSM_TRY_CUDA(cudaMemsetAsync(A.gave_up, 0, sizeof(unsigned), s));
    if ((rc = launch_first_search(first, s))) return rc;
    int mind_bytes = 0;
    rc = launch_maxmin_cluster(n, rowptr, A.adj, k, start, pivots, status, spill, fallback, A.mind, A.best,
                               A.gave_up, s, &mind_bytes);
    if (rc || mind_bytes == 4) return rc;
    if (mind_bytes == 2) A.run_if = fallback;
  }
  if (!A.run_if) note_pivot_config(0, 4);
  return launch_maxmin_grid(A, s);
}
size_t maxmin_workspace(int32_t n, int64_t m2) {
  Carver c(nullptr, 0);
  MaxMinArgs A;
  unsigned *spill;
  carve_maxmin(c, A, &spill, n, m2);
  return c.size();
}

// --------------------------------------------------------------------------
// one source per block: visited bitmap in shared memory
// --------------------------------------------------------------------------
#ifndef SSM_CTA_STEP
#define SSM_CTA_STEP 4
#endif
#ifndef SSM_CTA_LANE_ROW
#define SSM_CTA_LANE_ROW 32
#endif
#ifndef SSM_CTA_QMAX
#define SSM_CTA_QMAX 4096
#endif
#ifndef SSM_ADJ2_MAX_MB
#define SSM_ADJ2_MAX_MB 48
#endif
constexpr int kCtaThreads = 512;
constexpr int kCtaStep = SSM_CTA_STEP;         // edges whose loads a lane has in flight at once
constexpr int kCtaLaneRow = SSM_CTA_LANE_ROW;  // rows up to this length: one lane; longer: the warp
constexpr int kCtaQMax = SSM_CTA_QMAX;         // frontier entries per level kept in shared memory (at most)
#ifndef SSM_CTA_FEW_MIN_NODES
#define SSM_CTA_FEW_MIN_NODES 131072
#endif
constexpr int kCtaFewMinNodes = SSM_CTA_FEW_MIN_NODES;  // smaller graphs always take four blocks per SM
constexpr size_t kCtaBitmapMax = 200 * 1024;   // bytes of shared memory for the visited bitmap
constexpr size_t kAdj2MaxBytes = (size_t)SSM_ADJ2_MAX_MB << 20;  // packed adjacency kept only while it fits well inside L2
constexpr int kAdj2NodeBits = 21;              // packed adjacency: node id below 2^21 ...
constexpr unsigned kAdj2DegEsc = 2047u;        // ... and min(deg, 2047) above it (2047: read rowptr)

struct CtaBfsArgs {
  int32_t n;
  const int32_t *rowptr;
  const int32_t *colidx;
  int32_t nsrc;
  const int32_t *sources;
  uint16_t *dist;  // [nsrc][n]
  int32_t *status;
  const int2 *adj; // [2m] packed adjacency (v | min(deg v, 2047) << 21, rowptr[v])
  int2 *queues;    // [slots][2][n] frontier entries (row start, degree) past the shared part
  int32_t qsm;     // entries per level kept in shared memory (a multiple of 32)
  const unsigned *run_if;  // run only if this device word is nonzero (the pulled BFS gave up)
};

// Each block owns sources blockIdx.x, blockIdx.x + gridDim.x, ...; per source
// a level-synchronous BFS whose visited set is a bitmap in shared memory
// (claimed with shared atomicOr).  The frontier holds (row start, degree) of
// its nodes -- read from the packed adjacency when a node is claimed, so the
// next level needs no rowptr lookup -- in shared memory for its first qsm
// entries, in global memory past them.  Levels are separated by one
// __syncthreads (three rotating frontier counters: level L reads counter
// L mod 3, appends to L + 1 mod 3, and thread 0 clears L + 2 mod 3, which
// nobody reads again before the barrier).  A lane walks the row of its own
// frontier node with the loads of kCtaStep edges in flight (the warp takes
// as many steps as its longest row needs); rows longer than kCtaLaneRow are
// walked by the whole warp, one row at a time.  Each step claims its nodes,
// compacts the appends with warp ballots and reserves their slots with one
// shared-memory atomic, so a round costs about one global-memory latency.
template <bool ADJ, int MINB>
__global__ void __launch_bounds__(kCtaThreads, MINB) k_bfs_cta(CtaBfsArgs A) {
  extern __shared__ __align__(16) unsigned cta_smem[];
  __shared__ unsigned s_cnt[3];
  const unsigned n = (unsigned)A.n, nwords = (n + 31u) / 32u;
  unsigned *vis = cta_smem;
  int2 *sq = reinterpret_cast<int2 *>(cta_smem + ((nwords + 3u) & ~3u));  // [2][qsm]
  const unsigned qsm = (unsigned)A.qsm;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  if (__ldcg(A.run_if) == 0u) return;
  int2 *const qg = A.queues + (size_t)blockIdx.x * 2 * n;
  for (int si = blockIdx.x; si < A.nsrc; si += gridDim.x) {
    for (unsigned w = threadIdx.x; w < nwords; w += blockDim.x) vis[w] = 0u;
    __syncthreads();
    uint16_t *row = A.dist + (size_t)si * n;
    if (threadIdx.x == 0) {
      unsigned s = (unsigned)__ldg(A.sources + si);
      if (s >= n) {  // a source id outside the graph: recorded; node 0 keeps the search in bounds
        dev_fail(A.status, SSM_E_ARG);
        s = 0;
      }
      vis[s >> 5] |= 1u << (s & 31u);
      const int rb = __ldg(A.rowptr + s);
      const int2 e0 = make_int2(rb, __ldg(A.rowptr + s + 1) - rb);
      if (qsm > 0) sq[0] = e0; else qg[0] = e0;
      row[s] = 0;
      s_cnt[0] = 1;
      s_cnt[1] = 0;
      s_cnt[2] = 0;
    }
    __syncthreads();
    unsigned total = 0;  // nodes reached (thread 0)
    int c0 = 0;          // counter of this level
    for (unsigned L = 0;; ++L) {
      const unsigned cc = s_cnt[c0];
      if (cc == 0) break;
      if (L + 1 > 65534u) {
        if (threadIdx.x == 0) dev_fail(A.status, SSM_E_DIST_OVERFLOW);
        break;
      }
      const int c1 = c0 == 2 ? 0 : c0 + 1, c2 = c1 == 2 ? 0 : c1 + 1;
      if (threadIdx.x == 0) {
        total += cc;
        s_cnt[c2] = 0;
      }
      const unsigned bin = L & 1u, bout = bin ^ 1u;
      const int2 *sin = sq + bin * qsm, *gin = qg + (size_t)bin * n;
      int2 *sout = sq + bout * qsm, *gout = qg + (size_t)bout * n;
      unsigned *cnt_next = s_cnt + c1;
      const uint16_t nd = (uint16_t)(L + 1);
      // claim the nodes of up to kCtaStep edges per lane (edge u valid where
      // ok[u]) and append the new ones to the next frontier
      auto step = [&](const int (&idx)[kCtaStep], const bool (&ok)[kCtaStep]) {
        int2 ed[kCtaStep];
        bool push[kCtaStep];
#pragma unroll
        for (int u = 0; u < kCtaStep; ++u) ed[u] = ok[u] ? __ldg(A.adj + idx[u]) : make_int2(0, 0);
        unsigned tot = 0;
#pragma unroll
        for (int u = 0; u < kCtaStep; ++u) {
          push[u] = false;
          if (ok[u]) {
            const unsigned v = (unsigned)ed[u].x & ((1u << kAdj2NodeBits) - 1u);
            const unsigned bit = 1u << (v & 31u);
            unsigned *wp = vis + (v >> 5);
            push[u] = !(*wp & bit) && !(atomicOr(wp, bit) & bit);
          }
          tot += __popc(__ballot_sync(0xffffffffu, push[u]));
        }
        if (tot == 0) return;
        unsigned pos = 0;
        if (lane == 0) pos = atomicAdd(cnt_next, tot);
        pos = __shfl_sync(0xffffffffu, pos, 0);
#pragma unroll
        for (int u = 0; u < kCtaStep; ++u) {
          const unsigned mk = __ballot_sync(0xffffffffu, push[u]);
          if (push[u]) {
            const unsigned v = (unsigned)ed[u].x & ((1u << kAdj2NodeBits) - 1u);
            unsigned dg = (unsigned)ed[u].x >> kAdj2NodeBits;
            if (dg == kAdj2DegEsc) dg = (unsigned)(__ldg(A.rowptr + v + 1) - ed[u].y);
            row[v] = nd;
            const unsigned q = pos + __popc(mk & lt);
            const int2 ent = make_int2(ed[u].y, (int)dg);
            if (q < qsm) sout[q] = ent; else gout[q] = ent;
          }
          pos += __popc(mk);
        }
      };
      for (unsigned base = warp * 32u; base < cc; base += nwarps * 32u) {
        const unsigned e = base + lane;
        const int2 r = e < cc ? (e < qsm ? sin[e] : __ldcg(gin + e)) : make_int2(0, 0);
        if (ADJ) {
          const bool mine = r.y <= kCtaLaneRow;
          const int steps = __reduce_max_sync(0xffffffffu, mine ? r.y : 0);
          for (int j = 0; j < steps; j += kCtaStep) {
            int idx[kCtaStep];
            bool ok[kCtaStep];
#pragma unroll
            for (int u = 0; u < kCtaStep; ++u) {
              ok[u] = mine && j + u < r.y;
              idx[u] = r.x + j + u;
            }
            step(idx, ok);
          }
          // rows longer than kCtaLaneRow: the whole warp walks each in turn
          unsigned longm = __ballot_sync(0xffffffffu, !mine);
          while (longm) {
            const int o = __ffs(longm) - 1;
            longm &= longm - 1u;
            const int rb = __shfl_sync(0xffffffffu, r.x, o), dg = __shfl_sync(0xffffffffu, r.y, o);
            for (int t = 0; t < dg; t += 32 * kCtaStep) {
              int idx[kCtaStep];
              bool ok[kCtaStep];
#pragma unroll
              for (int u = 0; u < kCtaStep; ++u) {
                const int t1 = t + 32 * u + (int)lane;
                ok[u] = t1 < dg;
                idx[u] = rb + t1;
              }
              step(idx, ok);
            }
          }
        } else {
          warp_for_each_neighbor_batched<4>(
              r.x, r.x + r.y, A.colidx,
              [&](int, int, int v) {
                const unsigned bit = 1u << ((unsigned)v & 31u);
                unsigned *wp = vis + ((unsigned)v >> 5);
                return !(*wp & bit) && !(atomicOr(wp, bit) & bit);
              },
              [&](int, int, int v, bool push) {
                const unsigned q = warp_slot(push, cnt_next);
                if (push) {
                  row[v] = nd;
                  const int rb = __ldg(A.rowptr + v);
                  const int2 ent = make_int2(rb, __ldg(A.rowptr + v + 1) - rb);
                  if (q < qsm) sout[q] = ent; else gout[q] = ent;
                }
              });
        }
      }
      __syncthreads();
      c0 = c1;
    }
    if (threadIdx.x == 0 && total != n) dev_fail(A.status, SSM_E_DISCONNECTED);
    __syncthreads();
  }
}

// packed adjacency: adj[t] = (v | min(deg v, 2047) << 21, rowptr[v]) for v = colidx[t]
__global__ void k_pack_adj(int64_t m2, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                           int2 *__restrict__ adj) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m2; t += (int64_t)gridDim.x * blockDim.x) {
    const int v = __ldg(colidx + t);
    const int rb = __ldg(rowptr + v);
    const unsigned dg = min((unsigned)(__ldg(rowptr + v + 1) - rb), kAdj2DegEsc);
    adj[t] = make_int2((int)((unsigned)v | (dg << kAdj2NodeBits)), rb);
  }
}

static bool cta_bfs_fits(int32_t n) { return (size_t)((n + 31) / 32) * 4 <= kCtaBitmapMax; }

struct CtaBfsShape {
  bool many;  // four blocks per SM (32 registers a thread), else two (64)
  int slots, qsm;
  size_t smem;
};

static const void *cta_bfs_kernel(bool packed, bool many) {
  if (packed) return many ? (const void *)k_bfs_cta<true, 4> : (const void *)k_bfs_cta<true, 2>;
  return many ? (const void *)k_bfs_cta<false, 4> : (const void *)k_bfs_cta<false, 2>;
}

// Blocks of 512 threads: on a large graph whose sources fit two per SM, two
// per SM, with the shared memory an SM can give each beyond the bitmap holding
// the first qsm frontier entries of both levels; otherwise four per SM, with
// the bitmap alone (measured: a shared-memory frontier at four blocks per SM
// leaves less L1 for the adjacency reads and was slower on rgg256k, and two
// fat blocks per SM cost concurrent requests of mid-size graphs 7 % of the
// serving capacity).  Without a device (workspace queries on a host) one slot
// per SM is assumed.
static CtaBfsShape cta_bfs_shape(int32_t n, int32_t nsrc) {
  CtaBfsShape S;
  const int sms = num_sms();
  S.many = nsrc > 2 * sms || n < kCtaFewMinNodes;
  const int want = S.many ? 4 : 2;
  const size_t bitmap = (size_t)(((n + 31) / 32 + 3) & ~3) * 4;
  int dev = 0, per_sm_smem = 0, per_block_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_block_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    per_sm_smem = 0;
    per_block_max = 0;
  }
  const int64_t budget = std::min<int64_t>(per_block_max, (int64_t)per_sm_smem / want - 1024) - 64;
  int64_t q = (!S.many && budget > (int64_t)bitmap) ? (budget - (int64_t)bitmap) / (2 * (int64_t)sizeof(int2)) : 0;
  q = std::min<int64_t>(q, kCtaQMax) & ~31ll;
  S.qsm = (int)std::max<int64_t>(0, q);
  S.smem = bitmap + 2 * (size_t)S.qsm * sizeof(int2);
  int per_sm = 0;
  const void *kern = cta_bfs_kernel(true, S.many);
  if (allow_dynamic_smem(kern) != cudaSuccess || allow_dynamic_smem(cta_bfs_kernel(false, S.many)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCtaThreads, S.smem) != cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  S.slots = std::max(1, std::min(nsrc, sms * std::min(per_sm, want)));
  return S;
}

// --------------------------------------------------------------------------
// multi-source bitset BFS
// --------------------------------------------------------------------------
struct MsBfsArgs {
  int32_t n;
  const int32_t *rowptr;
  const int32_t *colidx;
  int32_t k;
  int32_t W;  // 32-bit words per node = ceil(k/32)
  const int32_t *sources;
  uint16_t *dist;  // [k][n]
  int32_t *status;
  unsigned *seen;  // [n*W] sources that have reached each node
  unsigned *F[3];  // [n*W] frontier bits of levels L, L+1, L+2 (rotated)
  unsigned *Q[3];  // [n*W] queue of (node*W + word) entries with nonzero frontier bits
  unsigned *qcnt;  // [4] queue lengths, rotated by level
  unsigned long long *ndisc;  // total (source, node) discoveries
  BarrierState *bar;
};

// Level L expands every queued (u, w) entry: the sources in frontier word
// F_L[u][w] are pushed to each neighbour v.  New bits are claimed with one
// atomicOr on seen[v][w] (so each (source, node) pair is discovered exactly
// once, at its BFS level), merged into F_{L+1}[v][w], and the first claimant
// of a word appends (v, w) to the next queue.  Entries of F_{L-1} are cleared
// through their queue so the three frontier arrays can rotate.
__global__ void __launch_bounds__(kBfsThreads) k_msbfs(MsBfsArgs A) {
  const unsigned nthreads = gridDim.x * blockDim.x;
  const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gwarp = gtid >> 5, nwarps = nthreads >> 5;
  const unsigned n = (unsigned)A.n, W = (unsigned)A.W, k = (unsigned)A.k;
  unsigned long long found = 0;

  // level 0: the sources themselves (warp-uniform loop so appends stay converged)
  for (unsigned base = gwarp * 32u; base < k; base += nwarps * 32u) {
    const unsigned a = base + lane;
    bool push = false;
    unsigned idx = 0;
    if (a < k && (unsigned)__ldg(A.sources + a) >= n) dev_fail(A.status, SSM_E_ARG);  // not seeded
    if (a < k && (unsigned)__ldg(A.sources + a) < n) {
      const unsigned v = (unsigned)__ldg(A.sources + a);
      const unsigned w = a >> 5, bit = 1u << (a & 31u);
      idx = v * W + w;
      const unsigned old = atomicOr(A.seen + idx, bit);
      if (!(old & bit)) {
        A.dist[(size_t)a * n + v] = 0;
        ++found;
        push = atomicOr(A.F[0] + idx, bit) == 0u;
      }
    }
    warp_append(push, idx, A.Q[0], A.qcnt + 0);
  }
  if (!grid_barrier(A.bar, A.status)) return;

  for (unsigned L = 0;; ++L) {
    const unsigned c = __ldcg(A.qcnt + (L & 3u));
    if (c == 0) break;
    if (L + 1 > 65534u) {
      if (gtid == 0) dev_fail(A.status, SSM_E_DIST_OVERFLOW);
      break;
    }
    if (gtid == 0) A.qcnt[(L + 2) & 3u] = 0;
    // clear F_{L-1} (its array becomes F_{L+2})
    {
      const unsigned cprev = __ldcg(A.qcnt + ((L + 3) & 3u));
      const unsigned *qprev = A.Q[(L + 2) % 3];
      unsigned *fprev = A.F[(L + 2) % 3];
      for (unsigned e = gtid; e < cprev; e += nthreads) fprev[__ldcg(qprev + e)] = 0u;
    }
    const unsigned *qin = A.Q[L % 3];
    const unsigned *fin = A.F[L % 3];
    unsigned *fout = A.F[(L + 1) % 3];
    unsigned *qout = A.Q[(L + 1) % 3];
    unsigned *cout = A.qcnt + ((L + 1) & 3u);
    const uint16_t nd = (uint16_t)(L + 1);
    for (unsigned base = gwarp * 32u; base < c; base += nwarps * 32u) {
      const unsigned e = base + lane;
      int beg = 0, end = 0;
      unsigned w = 0, f = 0;
      if (e < c) {
        const unsigned idx = __ldcg(qin + e);
        const unsigned u = idx / W;
        w = idx - u * W;
        f = __ldcg(fin + idx);
        beg = __ldg(A.rowptr + u);
        end = __ldg(A.rowptr + u + 1);
      }
      warp_for_each_neighbor(beg, end, A.colidx, [&](int owner, bool act, int v) {
        const unsigned wo = __shfl_sync(0xffffffffu, w, owner);
        const unsigned fo = __shfl_sync(0xffffffffu, f, owner);
        const unsigned nidx = (unsigned)v * W + wo;
        bool push = false;
        if (act) {
          unsigned nb = fo & ~__ldcg(A.seen + nidx);
          if (nb) {
            nb &= ~atomicOr(A.seen + nidx, nb);
            if (nb) {
              push = atomicOr(fout + nidx, nb) == 0u;
              found += (unsigned)__popc(nb);
              uint16_t *col = A.dist + (size_t)(wo * 32u) * n + (unsigned)v;
              while (nb) {
                const unsigned b = (unsigned)__ffs(nb) - 1u;
                col[(size_t)b * n] = nd;
                nb &= nb - 1u;
              }
            }
          }
        }
        warp_append(push, nidx, qout, cout);
      });
    }
    if (!grid_barrier(A.bar, A.status)) return;
  }

  // every (source, node) pair must have been discovered
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(0xffffffffu, found, o);
  if (lane == 0 && found) atomicAdd(A.ndisc, found);
  if (!grid_barrier(A.bar, A.status)) return;
  if (gtid == 0 && __ldcg(A.ndisc) != (unsigned long long)k * n) {
    int32_t cur = __ldcg(A.status);
    if (cur == 0) dev_fail(A.status, SSM_E_DISCONNECTED);
  }
}

static void msbfs_carve(Carver &c, MsBfsArgs &A, int32_t n, int32_t k) {
  const size_t nw = (size_t)n * (size_t)((k + 31) / 32);
  A.seen = c.take<unsigned>(nw);
  for (int i = 0; i < 3; ++i) A.F[i] = c.take<unsigned>(nw);
  for (int i = 0; i < 3; ++i) A.Q[i] = c.take<unsigned>(nw);
  A.qcnt = c.take<unsigned>(4);
  A.ndisc = c.take<unsigned long long>(1);
  A.bar = c.take<BarrierState>(1);
}

size_t msbfs_workspace(int32_t n, int64_t m2, int32_t k) {
  Carver c(nullptr, 0);
  if (cta_bfs_fits(n)) {
    c.take<int2>((size_t)(m2 > 0 ? m2 : 1));
    c.take<int2>((size_t)cta_bfs_shape(n, k).slots * 2 * (size_t)n);
    c.take<unsigned>(1);
    c.take<char>(msbfs_pull_workspace(n));
    return c.size();
  }
  MsBfsArgs A;
  msbfs_carve(c, A, n, k);
  return c.size();
}

// dist[0 .. count) = 0xFFFF (unreached) when *run_if != 0
__global__ void k_fill_unreached_if(int64_t count, const unsigned *__restrict__ run_if, uint16_t *__restrict__ dist) {
  if (__ldcg(run_if) == 0u) return;
  uint4 *d4 = reinterpret_cast<uint4 *>(dist);
  const int64_t n16 = (reinterpret_cast<uintptr_t>(dist) & 15u) == 0 ? count / 8 : 0;  // 16-byte stores when aligned
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n16; t += (int64_t)gridDim.x * blockDim.x)
    d4[t] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
  for (int64_t t = n16 * 8 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    dist[t] = 0xFFFFu;
}

// Graphs whose visited bitmap fits shared memory: first the pulled bitset BFS
// (few levels, every level touches most edges); if it gives up on a large
// diameter, one block per source (k_bfs_cta), on a table first filled with
// "unreached".  Larger graphs: k_msbfs.
int launch_msbfs(int32_t n, int64_t m2, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                 const int32_t *sources, uint16_t *dist, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s,
                 const PullPassFn *after_pass, const unsigned **pull_gaveup) {
  Carver c(ws, ws_bytes);
  if (pull_gaveup) *pull_gaveup = nullptr;
  if (cta_bfs_fits(n)) {
    CtaBfsArgs B;
    B.n = n; B.rowptr = rowptr; B.colidx = colidx; B.nsrc = k; B.sources = sources; B.dist = dist;
    B.status = status;
    const CtaBfsShape S = cta_bfs_shape(n, k);
    int2 *adj = c.take<int2>((size_t)(m2 > 0 ? m2 : 1));
    B.adj = adj;
    B.queues = c.take<int2>((size_t)S.slots * 2 * (size_t)n);
    B.qsm = S.qsm;
    unsigned *gaveup = c.take<unsigned>(1);
    const size_t pw = msbfs_pull_workspace(n);
    void *pws = c.take<char>(pw);
    B.run_if = gaveup;
    if (!c.ok) return fail(SSM_E_NOMEM, "BFS: workspace %zu bytes, need %zu", ws_bytes, c.size());
    SSM_TRY_CUDA(cudaMemsetAsync(gaveup, 0, sizeof(unsigned), s));
    int rc = launch_msbfs_pull(n, rowptr, colidx, k, sources, dist, status, gaveup, pws, pw, s, after_pass);
    if (rc) return rc;
    if (pull_gaveup) *pull_gaveup = gaveup;
    // a complete pulled BFS wrote every entry (or handed every pass over)
    const int64_t cells = (int64_t)k * n;
    note_launch(), k_fill_unreached_if<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((cells / 8 + 255) / 256,
                                                                                          (int64_t)num_sms() * 8)),
                                         256, 0, s>>>(cells, gaveup, dist);
    // the packed adjacency saves a dependent rowptr load per level but doubles
    // adjacency traffic: use it only while it stays L2-resident
    const bool packed = (size_t)m2 * sizeof(int2) <= kAdj2MaxBytes && n < (1 << kAdj2NodeBits);
    if (packed && m2 > 0) {
      const int blocks = (int)std::min<int64_t>((m2 + 255) / 256, (int64_t)num_sms() * 8);
      note_launch(), k_pack_adj<<<blocks, 256, 0, s>>>(m2, rowptr, colidx, adj);
    }
    void *args[] = {&B};
    note_launch();
    SSM_TRY_CUDA(cudaLaunchKernel(cta_bfs_kernel(packed, S.many), dim3(S.slots), dim3(kCtaThreads), args, S.smem, s));
    return SSM_OK;
  }
  MsBfsArgs A;
  A.n = n; A.rowptr = rowptr; A.colidx = colidx; A.k = k; A.W = (k + 31) / 32;
  A.sources = sources; A.dist = dist; A.status = status;
  msbfs_carve(c, A, n, k);
  if (!c.ok) return fail(SSM_E_NOMEM, "multi-source BFS: workspace %zu bytes, need %zu", ws_bytes, c.size());
  const size_t nw = (size_t)n * (size_t)A.W;
  // seen, F[0..2] are contiguous carve-outs of equal size; clear each
  SSM_TRY_CUDA(cudaMemsetAsync(A.seen, 0, nw * sizeof(unsigned), s));
  for (int i = 0; i < 3; ++i) SSM_TRY_CUDA(cudaMemsetAsync(A.F[i], 0, nw * sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(A.qcnt, 0, 4 * sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(A.ndisc, 0, sizeof(unsigned long long), s));
  if (int rc_ = reset_barrier(A.bar, s)) return rc_;
  SSM_TRY_CUDA(cudaMemsetAsync(dist, 0xFF, (size_t)k * n * sizeof(uint16_t), s));
  const int blocks = cooperative_blocks((const void *)k_msbfs, kBfsThreads, 0, 2);
  if (blocks < 1) return fail(SSM_E_CUDA, "multi-source BFS: kernel cannot be resident");
  void *args[] = {&A};
  note_launch();
  SSM_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)k_msbfs, dim3(blocks), dim3(kBfsThreads), args, 0, s));
  return SSM_OK;
}

}  // namespace ssm

// ---------------------------------------------------------------- C ABI
SSM_API size_t ssm_select_pivots_workspace(int32_t n, int64_t m) {
  return (n > 0 && m >= 0) ? ssm::maxmin_workspace(n, 2 * m) : 0;
}

SSM_API int ssm_select_pivots(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                              int32_t start, int32_t *pivots, int32_t *status, void *ws, size_t ws_bytes,
                              cudaStream_t stream) {
  if (n < 1 || m < 0 || !rowptr || !colidx || !pivots || !status || !ws)
    return ssm::fail(SSM_E_ARG, "ssm_select_pivots: null pointer or bad size");
  if (k < 1 || k > n) return ssm::fail(SSM_E_ARG, "ssm_select_pivots: need 1 <= k <= n (k=%d, n=%d)", k, n);
  if (start < 0 || start >= n) return ssm::fail(SSM_E_ARG, "ssm_select_pivots: start %d outside 0..n-1", start);
  return ssm::launch_maxmin(n, 2 * m, rowptr, colidx, k, start, pivots, status, ws, ws_bytes, stream);
}

SSM_API size_t ssm_pivot_bfs_workspace(int32_t n, int64_t m, int32_t k) {
  return (n > 0 && m >= 0 && k > 0) ? ssm::msbfs_workspace(n, 2 * m, k) : 0;
}

SSM_API int ssm_pivot_bfs(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                          const int32_t *pivots, uint16_t *dip, int32_t *status, void *ws, size_t ws_bytes,
                          cudaStream_t stream) {
  if (n < 1 || m < 0 || !rowptr || !colidx || !pivots || !dip || !status || !ws)
    return ssm::fail(SSM_E_ARG, "ssm_pivot_bfs: null pointer or bad size");
  if (k < 1 || k > 65535) return ssm::fail(SSM_E_ARG, "ssm_pivot_bfs: need 1 <= k <= 65535 (k=%d)", k);
  if ((int64_t)n * ((k + 31) / 32) >= (int64_t)1 << 31)
    return ssm::fail(SSM_E_ARG, "ssm_pivot_bfs: n*ceil(k/32) must be below 2^31");
  return ssm::launch_msbfs(n, 2 * m, rowptr, colidx, k, pivots, dip, status, ws, ws_bytes, stream);
}
