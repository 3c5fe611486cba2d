// Multi-source BFS with one bit per source, pulled level by level (the
// "bottom-up" direction): at level L every node v that some sources have not
// reached yet ORs the frontier words of its neighbours,
//   new_v = (OR_{u in N(v)} F_L[u]) & ~seen_v,
// stopping its walk as soon as every missing source has turned up.  Each
// node's words are written by its own lane only, so no atomics are needed
// after the sources are seeded.  The new bits of every level are kept
// (F_0 = the sources, F_{L+1} = the bits found at level L), and after the
// pass k_pull_distances turns them into d_ip rows: a block takes 64 nodes,
// folds each node's levels into five bit planes of the distance (bit j of
// d(s, v) is bit s of plane j), and its warps write one source row segment
// of 32 consecutive nodes per store.
//
// This wins on graphs of small diameter (hubs, expanders), where a few levels
// each touch most edges and the per-source BFS would walk every edge once per
// source.  On large-diameter graphs every level re-reads the frontier words
// of all unfinished nodes, so a pass gives up when its first kPullProbeLevel
// levels reached less than 1/64 of all (source, node) pairs, or after
// kPullMaxLevels levels, and reports it; the caller then runs the per-source
// BFS.  Sources are taken in
// passes of 256 (eight 32-bit words per node).
//
// Beside F_L a bitmap per level marks the nodes whose F_L word is not zero
// (the frontier of level L); a node reads a neighbour's 32-byte frontier
// words only when its bit is set.  At the first levels the frontier is a
// small part of the graph and nearly every such read is saved; the bitmap
// (n / 8 bytes) stays in L1.
#include <algorithm>

#include "bfs.cuh"

namespace ssm {

constexpr int kPullThreads = 512;
constexpr int kPullSources = 256;  // sources per pass: 8 words per node
constexpr int kPullW4 = kPullSources / 128;  // uint4 chunks per node
constexpr unsigned kPullMaxLevels = 24;
static_assert(kPullSources == kPullPassSources && kPullMaxLevels + 1 == kPullPassLevels, "pass layout");
constexpr unsigned kPullProbeLevel = 6;  // after this level at least 1/64 of all pairs must be reached
constexpr int kPullLong = 64;  // longer rows are walked by the whole warp
#ifndef SSM_PULL_LONG_BATCH
#define SSM_PULL_LONG_BATCH 4
#endif
constexpr int kPullLongBatch = SSM_PULL_LONG_BATCH;  // neighbours per lane in flight while a warp walks a long row

struct PullArgs {
  int32_t n;
  const int32_t *rowptr;
  const int32_t *colidx;
  int32_t nsrc;     // sources in this pass (<= kPullSources)
  int32_t base;     // index of the pass's first source
  const int32_t *sources;
  uint16_t *dist;   // [all sources][n]
  int32_t *status;
  uint4 *seen;      // [n][kPullW4] sources that reached the node
  uint4 *F;         // [kPullMaxLevels + 1][n][kPullW4] new bits of every level
  unsigned *fb;     // [kPullMaxLevels + 1][fbw] bit v of level L: F_L[v] is not zero (zeroed by the caller)
  size_t fbw;       // words per level bitmap (a multiple of 32: 128-byte rows)
  const int32_t *long_rows;  // nodes of degree above kPullLong
  const unsigned *nlong;     // how many (device)
  unsigned *nlev;   // levels with new bits (written when the pass completes)
  unsigned *flag;   // [6]: new bits seen at level L, nodes left unfinished (both by L mod 3)
  unsigned long long *found;  // (source, node) pairs reached up to the probe level
  unsigned *gaveup; // set when a pass needed more than kPullMaxLevels levels
  BarrierState *bar;
};

__device__ __forceinline__ unsigned src_mask(int nsrc, int w) {  // valid source bits of word w
  const int lo = w * 32;
  if (lo >= nsrc) return 0u;
  return nsrc - lo >= 32 ? 0xFFFFFFFFu : (1u << (nsrc - lo)) - 1u;
}

__device__ __forceinline__ unsigned word(const uint4 q, int j) {
  return j == 0 ? q.x : j == 1 ? q.y : j == 2 ? q.z : q.w;
}

__global__ void __launch_bounds__(kPullThreads, 2) k_msbfs_pull(PullArgs A) {
  const unsigned nthreads = gridDim.x * blockDim.x;
  const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gwarp = gtid >> 5, nwarps = nthreads >> 5;
  const unsigned n = (unsigned)A.n;

  if (__ldcg(A.gaveup)) return;  // an earlier pass already gave up
  const unsigned nlong = __ldcg(A.nlong);
  // level 0: the sources (seen and F_0 were cleared by the caller)
  for (int a = (int)gtid; a < A.nsrc; a += (int)nthreads) {
    const unsigned v = (unsigned)__ldg(A.sources + A.base + a);
    if (v >= n) {  // a source id outside the graph: recorded, not seeded
      dev_fail(A.status, SSM_E_ARG);
      continue;
    }
    const unsigned bit = 1u << (a & 31);
    unsigned *s = reinterpret_cast<unsigned *>(A.seen + (size_t)v * kPullW4) + (a >> 5);
    unsigned *f = reinterpret_cast<unsigned *>(A.F + (size_t)v * kPullW4) + (a >> 5);
    atomicOr(s, bit);
    atomicOr(f, bit);
    atomicOr(A.fb + (v >> 5), 1u << (v & 31u));
  }
  if (gtid == 0) {
    for (int i = 0; i < 6; ++i) A.flag[i] = 0u;
    *A.found = 0ull;
  }
  if (!grid_barrier(A.bar, A.status)) return;

  uint4 valid[kPullW4];
#pragma unroll
  for (int c = 0; c < kPullW4; ++c)
    valid[c] = make_uint4(src_mask(A.nsrc, 4 * c), src_mask(A.nsrc, 4 * c + 1), src_mask(A.nsrc, 4 * c + 2),
                          src_mask(A.nsrc, 4 * c + 3));

  for (unsigned L = 0;; ++L) {
    if (L >= kPullMaxLevels) {
      if (gtid == 0) atomicExch(A.gaveup, 1u);
      return;
    }
    const uint4 *fcur = A.F + (size_t)L * n * kPullW4;
    uint4 *fnext = A.F + (size_t)(L + 1u) * n * kPullW4;
    // level L's bitmap was written (in L2, by atomics) during level L - 1 and is
    // read only from this level on, so no cache holds an older copy of it
    const unsigned *fbcur = A.fb + (size_t)L * A.fbw;
    unsigned *fbnext = A.fb + (size_t)(L + 1u) * A.fbw;
    // the flags of level L+1 were last read right after the barrier of level
    // L-2, which every thread has passed since
    if (gtid == 0) {
      A.flag[(L + 1u) % 3u] = 0u;
      A.flag[3 + (L + 1u) % 3u] = 0u;
    }
    bool any_new = false, unfinished = false;
    unsigned pairs = 0;  // new (source, node) pairs of this lane (counted up to the probe level)
    for (unsigned base = gwarp * 32u; base < n; base += nwarps * 32u) {
      const unsigned v = base + lane;
      const bool live = v < n;
      uint4 miss[kPullW4], acc[kPullW4];
      bool open = false;
#pragma unroll
      for (int c = 0; c < kPullW4; ++c) {
        const uint4 s = live ? A.seen[(size_t)v * kPullW4 + c] : valid[c];
        miss[c] = make_uint4(~s.x & valid[c].x, ~s.y & valid[c].y, ~s.z & valid[c].z, ~s.w & valid[c].w);
        acc[c] = make_uint4(0u, 0u, 0u, 0u);
        open |= (miss[c].x | miss[c].y | miss[c].z | miss[c].w) != 0u;
      }
      int rb = 0, re = 0;
      if (open) {
        rb = __ldg(A.rowptr + v);
        re = __ldg(A.rowptr + v + 1);
      }
      // rows longer than kPullLong wait for the second phase of the level
      const bool deferred = open && re - rb > kPullLong;
      if (open && re - rb <= kPullLong) {
        // four neighbours in flight, stop once every missing source turned up
        for (int t = rb; t < re; t += 4) {
          unsigned u[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) u[e] = t + e < re ? (unsigned)__ldg(A.colidx + t + e) : 0xFFFFFFFFu;
          // neighbours outside level L's frontier add nothing
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (u[e] != 0xFFFFFFFFu && ((fbcur[u[e] >> 5] >> (u[e] & 31u)) & 1u) == 0u) u[e] = 0xFFFFFFFFu;
          bool done = true;
#pragma unroll
          for (int c = 0; c < kPullW4; ++c) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (u[e] == 0xFFFFFFFFu) continue;
              const uint4 f = __ldcg(fcur + (size_t)u[e] * kPullW4 + c);
              acc[c].x |= f.x;
              acc[c].y |= f.y;
              acc[c].z |= f.z;
              acc[c].w |= f.w;
            }
            done &= ((acc[c].x & miss[c].x) == miss[c].x) && ((acc[c].y & miss[c].y) == miss[c].y) &&
                    ((acc[c].z & miss[c].z) == miss[c].z) && ((acc[c].w & miss[c].w) == miss[c].w);
          }
          if (done) break;
        }
      }
      uint4 nw[kPullW4];
      bool got = false, left = false;
#pragma unroll
      for (int c = 0; c < kPullW4; ++c) {
        nw[c] = make_uint4(acc[c].x & miss[c].x, acc[c].y & miss[c].y, acc[c].z & miss[c].z, acc[c].w & miss[c].w);
        got |= (nw[c].x | nw[c].y | nw[c].z | nw[c].w) != 0u;
        left |= (nw[c].x ^ miss[c].x) | (nw[c].y ^ miss[c].y) | (nw[c].z ^ miss[c].z) | (nw[c].w ^ miss[c].w);
      }
      // this warp's 32 nodes in level L + 1's bitmap (a long row adds its bit later)
      const unsigned fbits = __ballot_sync(0xffffffffu, live && !deferred && got);
      if (lane == 0 && fbits != 0u) atomicOr(fbnext + (base >> 5), fbits);
      if (live && !deferred) {
#pragma unroll
        for (int c = 0; c < kPullW4; ++c) {
          fnext[(size_t)v * kPullW4 + c] = nw[c];
          if (got) {
            uint4 s = A.seen[(size_t)v * kPullW4 + c];
            s.x |= nw[c].x;
            s.y |= nw[c].y;
            s.z |= nw[c].z;
            s.w |= nw[c].w;
            A.seen[(size_t)v * kPullW4 + c] = s;
          }
        }
      }
      if (!deferred) {
        any_new |= got;
        unfinished |= left;
        if (L < kPullProbeLevel)
#pragma unroll
          for (int c = 0; c < kPullW4; ++c)
            pairs += __popc(nw[c].x) + __popc(nw[c].y) + __popc(nw[c].z) + __popc(nw[c].w);
      }
    }
    // second phase: the open long rows (hubs), one per warp across the grid,
    // kPullLongBatch entries per lane in flight, stopping once the node has
    // every missing source
    for (unsigned li = gwarp; li < nlong; li += nwarps) {
      const unsigned v = (unsigned)__ldg(A.long_rows + li);
      uint4 hmiss[kPullW4], part[kPullW4];
      bool open = false;
#pragma unroll
      for (int c = 0; c < kPullW4; ++c) {
        const uint4 sv = A.seen[(size_t)v * kPullW4 + c];
        hmiss[c] = make_uint4(~sv.x & valid[c].x, ~sv.y & valid[c].y, ~sv.z & valid[c].z, ~sv.w & valid[c].w);
        part[c] = make_uint4(0u, 0u, 0u, 0u);
        open |= (hmiss[c].x | hmiss[c].y | hmiss[c].z | hmiss[c].w) != 0u;
      }
      if (!open) continue;  // warp-uniform; the first phase wrote its empty frontier word
      const int hb = __ldg(A.rowptr + v), he = __ldg(A.rowptr + v + 1);
      for (int t0 = hb + (int)lane; t0 - (int)lane < he; t0 += 32 * kPullLongBatch) {
        unsigned u[kPullLongBatch];
#pragma unroll
        for (int e = 0; e < kPullLongBatch; ++e)
          u[e] = t0 + 32 * e < he ? (unsigned)__ldg(A.colidx + t0 + 32 * e) : 0xFFFFFFFFu;
#pragma unroll
        for (int e = 0; e < kPullLongBatch; ++e)
          if (u[e] != 0xFFFFFFFFu && ((fbcur[u[e] >> 5] >> (u[e] & 31u)) & 1u) == 0u) u[e] = 0xFFFFFFFFu;
#pragma unroll
        for (int c = 0; c < kPullW4; ++c)
#pragma unroll
          for (int e = 0; e < kPullLongBatch; ++e) {
            if (u[e] == 0xFFFFFFFFu) continue;
            const uint4 f = __ldcg(fcur + (size_t)u[e] * kPullW4 + c);
            part[c].x |= f.x;
            part[c].y |= f.y;
            part[c].z |= f.z;
            part[c].w |= f.w;
          }
        bool done = true;
#pragma unroll
        for (int c = 0; c < kPullW4; ++c) {
          part[c].x = __reduce_or_sync(0xffffffffu, part[c].x);
          part[c].y = __reduce_or_sync(0xffffffffu, part[c].y);
          part[c].z = __reduce_or_sync(0xffffffffu, part[c].z);
          part[c].w = __reduce_or_sync(0xffffffffu, part[c].w);
          done &= ((part[c].x & hmiss[c].x) == hmiss[c].x) && ((part[c].y & hmiss[c].y) == hmiss[c].y) &&
                  ((part[c].z & hmiss[c].z) == hmiss[c].z) && ((part[c].w & hmiss[c].w) == hmiss[c].w);
        }
        if (done) break;  // warp-uniform: every lane holds the reduced words
      }
      bool got = false, left = false;
      unsigned np = 0;
#pragma unroll
      for (int c = 0; c < kPullW4; ++c) {
        const uint4 nw = make_uint4(part[c].x & hmiss[c].x, part[c].y & hmiss[c].y, part[c].z & hmiss[c].z,
                                    part[c].w & hmiss[c].w);
        got |= (nw.x | nw.y | nw.z | nw.w) != 0u;
        left |= (nw.x ^ hmiss[c].x) | (nw.y ^ hmiss[c].y) | (nw.z ^ hmiss[c].z) | (nw.w ^ hmiss[c].w);
        np += __popc(nw.x) + __popc(nw.y) + __popc(nw.z) + __popc(nw.w);
        if (lane == 0) {
          fnext[(size_t)v * kPullW4 + c] = nw;
          if ((nw.x | nw.y | nw.z | nw.w) != 0u) {
            uint4 sv = A.seen[(size_t)v * kPullW4 + c];
            sv.x |= nw.x;
            sv.y |= nw.y;
            sv.z |= nw.z;
            sv.w |= nw.w;
            A.seen[(size_t)v * kPullW4 + c] = sv;
          }
        }
      }
      if (lane == 0) {
        any_new |= got;
        unfinished |= left;
        if (L < kPullProbeLevel) pairs += np;
        if (got) atomicOr(fbnext + (v >> 5), 1u << (v & 31u));
      }
    }
    if (__any_sync(0xffffffffu, any_new) && lane == 0) atomicOr(A.flag + L % 3u, 1u);
    if (__any_sync(0xffffffffu, unfinished) && lane == 0) atomicOr(A.flag + 3 + L % 3u, 1u);
    if (L < kPullProbeLevel) {
      pairs = __reduce_add_sync(0xffffffffu, pairs);
      if (lane == 0 && pairs) atomicAdd(A.found, (unsigned long long)pairs);
    }
    if (!grid_barrier(A.bar, A.status)) return;
    // a graph whose BFS balls grow slowly (large diameter) is left to the
    // per-source BFS early
    if (L + 1u == kPullProbeLevel && __ldcg(A.flag + L % 3u) != 0u &&
        __ldcg(A.found) * 64ull < (unsigned long long)A.n * (unsigned long long)A.nsrc) {
      if (gtid == 0) atomicExch(A.gaveup, 1u);
      return;
    }
    if (__ldcg(A.flag + L % 3u) == 0u) {
      // nothing new at this level: the pass is complete; unreached pairs mean
      // the graph is disconnected
      if (gtid == 0) {
        if (__ldcg(A.flag + 3 + L % 3u) != 0u) dev_fail(A.status, SSM_E_DISCONNECTED);
        *A.nlev = L + 1u;  // F_0 .. F_L hold every distance
      }
      return;
    }
  }
}

// d_ip rows from the level history (see the top of the file).  Block: 64
// nodes; planes[w][j][v] = OR of F_L[v] word w over the levels L with bit j
// set, so bit s & 31 of planes[s >> 5][j][v] is bit j of d(s, v).
constexpr int kPullTile = 64;
constexpr int kPullDistBits = 5;  // distances up to kPullMaxLevels < 32
__global__ void __launch_bounds__(256) k_pull_distances(PullArgs A) {
  __shared__ unsigned planes[kPullSources / 32][kPullDistBits][kPullTile];
  __shared__ unsigned reached[kPullSources / 32][kPullTile];
  if (__ldcg(A.gaveup)) return;
  // nlev is zeroed before each pass; a pass that stopped early (a barrier
  // wait ran out) leaves it 0 and the rows read as unreached
  const unsigned nlev = min(__ldcg(A.nlev), kPullMaxLevels + 1u);
  const int n = A.n;
  const int v0 = blockIdx.x * kPullTile;
  for (int t = threadIdx.x; t < (kPullSources / 32) * kPullTile; t += blockDim.x) {
    // consecutive threads take consecutive words of one node (coalesced reads)
    const int w = t % (kPullSources / 32), v = t / (kPullSources / 32);
    unsigned pl[kPullDistBits] = {0u, 0u, 0u, 0u, 0u}, any = 0u;
    if (v0 + v < n)
      for (unsigned L = 0; L < nlev; ++L) {
        const unsigned f =
            __ldcg(reinterpret_cast<const unsigned *>(A.F + ((size_t)L * n + (size_t)(v0 + v)) * kPullW4) + w);
        any |= f;
#pragma unroll
        for (int j = 0; j < kPullDistBits; ++j)
          if ((L >> j) & 1u) pl[j] |= f;
      }
#pragma unroll
    for (int j = 0; j < kPullDistBits; ++j) planes[w][j][v] = pl[j];
    reached[w][v] = any;
  }
  __syncthreads();
  // warp: one source at a time, the tile's 64 nodes in one store per lane (two
  // consecutive distances in a 32-bit word when the rows are 4-byte aligned)
  static_assert(kPullTile == 64, "two nodes per lane");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const bool pairs = (n % 2 == 0) && (reinterpret_cast<uintptr_t>(A.dist) & 3u) == 0;
  for (int sidx = warp; sidx < A.nsrc; sidx += nwarp) {
    const int w = sidx >> 5;
    const unsigned bit = 1u << (sidx & 31);
    uint16_t *row = A.dist + (size_t)(A.base + sidx) * n;
    unsigned dd[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int v = 2 * lane + h;
      unsigned d = 0;
#pragma unroll
      for (int j = 0; j < kPullDistBits; ++j) d |= ((planes[w][j][v] & bit) ? 1u : 0u) << j;
      dd[h] = (reached[w][v] & bit) ? d : 0xFFFFu;
    }
    const int v = v0 + 2 * lane;
    if (pairs && v + 1 < n) {
      *reinterpret_cast<unsigned *>(row + v) = dd[0] | (dd[1] << 16);
    } else {
      if (v < n) row[v] = (uint16_t)dd[0];
      if (v + 1 < n) row[v + 1] = (uint16_t)dd[1];
    }
  }
}

// the nodes of degree above kPullLong, in any order (the pass is order-free)
__global__ void k_pull_long_rows(int32_t n, const int32_t *__restrict__ rowptr, int32_t *__restrict__ out,
                                 unsigned *__restrict__ count) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (__ldg(rowptr + v + 1) - __ldg(rowptr + v) > kPullLong) out[atomicAdd(count, 1u)] = v;
}

// words of one level's frontier bitmap, rounded to whole 128-byte rows
static size_t pull_bitmap_words(int32_t n) { return (((size_t)n + 1023) / 1024) * 32; }

size_t msbfs_pull_workspace(int32_t n) {
  Carver c(nullptr, 0);
  c.take<uint4>((size_t)n * kPullW4);
  c.take<uint4>((size_t)n * kPullW4 * (kPullMaxLevels + 1));
  c.take<unsigned>(pull_bitmap_words(n) * (kPullMaxLevels + 1));
  c.take<int32_t>((size_t)n);
  c.take<unsigned>(1);
  c.take<unsigned>(1);
  c.take<unsigned>(6);
  c.take<unsigned long long>(1);
  c.take<BarrierState>(1);
  return c.size();
}

int launch_msbfs_pull(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k, const int32_t *sources,
                      uint16_t *dist, int32_t *status, unsigned *gaveup, void *ws, size_t ws_bytes, cudaStream_t s,
                      const PullPassFn *after_pass) {
  Carver c(ws, ws_bytes);
  PullArgs A;
  A.n = n; A.rowptr = rowptr; A.colidx = colidx; A.sources = sources; A.dist = dist; A.status = status;
  A.seen = c.take<uint4>((size_t)n * kPullW4);
  A.F = c.take<uint4>((size_t)n * kPullW4 * (kPullMaxLevels + 1));
  A.fbw = pull_bitmap_words(n);
  A.fb = c.take<unsigned>(A.fbw * (kPullMaxLevels + 1));
  int32_t *long_rows = c.take<int32_t>((size_t)n);
  unsigned *nlong = c.take<unsigned>(1);
  A.nlev = c.take<unsigned>(1);
  A.flag = c.take<unsigned>(6);
  A.found = c.take<unsigned long long>(1);
  A.bar = c.take<BarrierState>(1);
  A.gaveup = gaveup;
  if (!c.ok) return fail(SSM_E_NOMEM, "multi-source BFS: workspace %zu bytes, need %zu", ws_bytes, c.size());
  const int blocks = cooperative_blocks((const void *)k_msbfs_pull, kPullThreads, 0, 2);
  if (blocks < 1) return fail(SSM_E_CUDA, "multi-source BFS: kernel cannot be resident");
  // the long rows (listed on the device; the BFS reads their number there)
  SSM_TRY_CUDA(cudaMemsetAsync(nlong, 0, sizeof(unsigned), s));
  note_launch(), k_pull_long_rows<<<std::max(1, std::min((n + 255) / 256, num_sms() * 8)), 256, 0, s>>>(
      n, rowptr, long_rows, nlong);
  SSM_TRY_CUDA(cudaGetLastError());
  A.long_rows = long_rows;
  A.nlong = nlong;
  for (int base = 0; base < k; base += kPullSources) {
    A.base = base;
    A.nsrc = std::min(kPullSources, k - base);
    SSM_TRY_CUDA(cudaMemsetAsync(A.seen, 0, (size_t)n * kPullW4 * sizeof(uint4), s));
    SSM_TRY_CUDA(cudaMemsetAsync(A.F, 0, (size_t)n * kPullW4 * sizeof(uint4), s));
    SSM_TRY_CUDA(cudaMemsetAsync(A.fb, 0, A.fbw * (kPullMaxLevels + 1) * sizeof(unsigned), s));
    SSM_TRY_CUDA(cudaMemsetAsync(A.nlev, 0, sizeof(unsigned), s));
    if (int rc_ = reset_barrier(A.bar, s)) return rc_;
    void *args[] = {&A};
    note_launch();
    SSM_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)k_msbfs_pull, dim3(blocks), dim3(kPullThreads), args, 0, s));
    if (after_pass) {
      static_assert(kPullPassWords * 4 == kPullW4 * 16, "pass words per node");
      const PullPass P = {reinterpret_cast<const unsigned *>(A.F), A.nlev, gaveup, A.base, A.nsrc, base / kPullSources};
      if (int rc_ = (*after_pass)(P)) return rc_;
      continue;
    }
    note_launch(), k_pull_distances<<<(unsigned)((n + kPullTile - 1) / kPullTile), 256, 0, s>>>(A);
    SSM_TRY_CUDA(cudaGetLastError());
  }
  return SSM_OK;
}

}  // namespace ssm
