// Graph construction (Section 1: a simple undirected graph G = (V, E)):
// edge list -> CSR with both directions, rows sorted ascending, self-loops and
// repeated edges dropped, followed by a connectivity check (union-find).
//
//   count degrees (atomics) -> exclusive scan -> scatter both directions
//   -> sort every row (warp bitonic in registers for rows <= 128, block
//      bitonic in shared memory up to kSmemSortCap, block bitonic in global
//      memory beyond) -> flag first occurrences (entry-parallel) -> scan flags
//      -> compact.
#include <algorithm>

#include "bfs.cuh"
#include "scan.cuh"

namespace ssm {

constexpr int kSmemSortCap = 8192;  // ints sorted in shared memory by one block
constexpr int kSortBlock = 512;
constexpr int32_t kPad = 0x7fffffff;

__global__ void k_count_degrees(int64_t m, const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                                int32_t n, int *__restrict__ deg, int32_t *__restrict__ status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n) {
      dev_fail(status, SSM_E_GRAPH);
      continue;
    }
    if (u == v) continue;
    atomicAdd(deg + u, 1);
    atomicAdd(deg + v, 1);
  }
}

__global__ void k_scatter(int64_t m, const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int32_t n,
                          const int *__restrict__ off, int *__restrict__ cursor, int32_t *__restrict__ tmp) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n || u == v) continue;
    tmp[off[u] + atomicAdd(cursor + u, 1)] = v;
    tmp[off[v] + atomicAdd(cursor + v, 1)] = u;
  }
}

// Bitonic sorting network in the variant whose comparators all point
// upwards: for block size b, first compare i with its mirror i ^ (b-1), then
// half-cleaners i ^ j for j = b/4 .. 1.  Virtual +inf padding at positions
// >= len never has to move, so comparisons touching it can be skipped.

// rows of length <= 32: one warp per row, values in registers
// Bitonic sort of 32 E keys held by a warp, key e 32 + lane in x[e] of that
// lane: partners 32 or more apart sit in the same lane, closer ones in
// another lane of the same slot (a shuffle)
template <int E>
__device__ __forceinline__ void warp_bitonic(int32_t (&x)[E]) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int bs = 2; bs <= 32 * E; bs <<= 1) {
#pragma unroll
    for (int j = bs >> 1; j >= 1; j >>= 1) {
      if (j >= 32) {
        const int je = j >> 5;
#pragma unroll
        for (int e = 0; e < E; ++e)
          if ((e & je) == 0) {
            const bool asc = (((e * 32) & bs) == 0);
            const int32_t a = x[e], c = x[e | je];
            x[e] = asc ? min(a, c) : max(a, c);
            x[e | je] = asc ? max(a, c) : min(a, c);
          }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const unsigned idx = (unsigned)e * 32u + lane;
          const bool asc = (idx & (unsigned)bs) == 0u;
          const int32_t y = __shfl_xor_sync(0xffffffffu, x[e], j);
          x[e] = (((idx & (unsigned)j) == 0u) == asc) ? min(x[e], y) : max(x[e], y);
        }
      }
    }
  }
}

// rows of up to kWarpSortMax entries: one warp each, keys in registers (1 or
// 4 per lane); longer rows are listed for k_sort_big_rows
constexpr int kWarpSortMax = 128;
__global__ void k_sort_small_rows(int32_t n, const int *__restrict__ off, int32_t *__restrict__ tmp,
                                  unsigned *__restrict__ big_rows, unsigned *__restrict__ big_count) {
  const unsigned lane = threadIdx.x & 31u;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = warp; row < n; row += nwarps) {
    const int b = off[row], len = off[row + 1] - b;
    if (len > kWarpSortMax) {
      if (lane == 0) big_rows[atomicAdd(big_count, 1u)] = (unsigned)row;
      continue;
    }
    if (len > 32) {
      int32_t x[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = e * 32 + (int)lane;
        x[e] = i < len ? tmp[b + i] : kPad;
      }
      warp_bitonic<4>(x);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = e * 32 + (int)lane;
        if (i < len) tmp[b + i] = x[e];
      }
      continue;
    }
    int32_t x[1] = {(int)lane < len ? tmp[b + lane] : kPad};
    warp_bitonic<1>(x);
    if ((int)lane < len) tmp[b + lane] = x[0];
  }
}

template <class Get, class Put>
__device__ void block_bitonic(int len, Get get, Put put) {
  int P = 1;
  while (P < len) P <<= 1;
  for (int bs = 2; bs <= P; bs <<= 1) {
    for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
      // pair index i -> (lo, hi) in the mirror stage
      const int blk = i / (bs >> 1), r = i % (bs >> 1);
      const int lo = blk * bs + r, hi = blk * bs + bs - 1 - r;
      if (hi < len) {
        const int32_t a = get(lo), c = get(hi);
        if (a > c) { put(lo, c); put(hi, a); }
      }
    }
    __syncthreads();
    for (int j = bs >> 2; j >= 1; j >>= 1) {
      for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
        const int lo = (i / j) * 2 * j + (i % j), hi = lo + j;
        if (hi < len) {
          const int32_t a = get(lo), c = get(hi);
          if (a > c) { put(lo, c); put(hi, a); }
        }
      }
      __syncthreads();
    }
  }
}

// rows longer than kWarpSortMax: one block per row
__global__ void __launch_bounds__(kSortBlock) k_sort_big_rows(const int *__restrict__ off, int32_t *__restrict__ tmp,
                                                               const unsigned *__restrict__ big_rows,
                                                               const unsigned *__restrict__ big_count) {
  __shared__ int32_t sbuf[kSmemSortCap];
  const unsigned cnt = *big_count;
  for (unsigned t = blockIdx.x; t < cnt; t += gridDim.x) {
    const unsigned row = big_rows[t];
    const int b = off[row], len = off[row + 1] - b;
    int32_t *g = tmp + b;
    if (len <= kSmemSortCap) {
      for (int i = threadIdx.x; i < len; i += blockDim.x) sbuf[i] = g[i];
      __syncthreads();
      block_bitonic(len, [&](int i) { return sbuf[i]; }, [&](int i, int32_t v) { sbuf[i] = v; });
      for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = sbuf[i];
    } else {
      block_bitonic(len, [&](int i) { return __ldcg(g + i); }, [&](int i, int32_t v) { __stcg(g + i, v); });
    }
    __syncthreads();
  }
}

// flag[t] = 1 for the first occurrence of a value within its (sorted) row
// flag[t] = 1 for the first occurrence of a value in its (sorted) row: every
// entry against the one before it, then (k_flag_row_starts) every row's first
// entry, so hub rows do not queue in one thread
__global__ void k_flag_unique(const int *__restrict__ total, const int32_t *__restrict__ tmp, int *__restrict__ flag) {
  const int64_t tot = *total;  // off[n]: the directed entries before dedupe
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    flag[t] = (t == 0 || tmp[t] != tmp[t - 1]) ? 1 : 0;
}

__global__ void k_flag_row_starts(int32_t n, const int *__restrict__ off, int *__restrict__ flag) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    const int b = off[row];
    if (off[row + 1] > b) flag[b] = 1;
  }
}

__global__ void k_compact(int32_t n, int64_t total, const int *__restrict__ off, const int32_t *__restrict__ tmp,
                          const int *__restrict__ flag, const int *__restrict__ pos, int32_t *__restrict__ rowptr,
                          int32_t *__restrict__ colidx) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride)
    if (flag[t]) colidx[pos[t]] = tmp[t];
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row <= n; row += stride)
    rowptr[row] = pos[off[row]];
}

// ---- connectivity by union-find (no per-level latency) with neighbour
// sampling (Sutton, Ben-Nun and Barak, "Optimizing parallel graph
// connectivity computation via subgraph sampling", 2018): every node first
// links with its first two neighbours, the forest is compressed, the most
// frequent root among kUfSamples evenly spaced nodes is taken for the large
// component's, and only the nodes outside it link their remaining edges (an
// edge between that component and another one is also in the row of its
// other endpoint, which does not skip it).  A link hangs the root with the
// larger id under the one with the smaller id by compare-and-swap; the graph
// is connected iff exactly one node is its own root.
__device__ __forceinline__ int uf_find(int *parent, int x) {
  int p = __ldcg(parent + x);
  while (p != x) {
    const int gp = __ldcg(parent + p);
    if (gp != p) atomicCAS(parent + x, p, gp);  // path halving (only ever shortens)
    x = p;
    p = __ldcg(parent + x);
  }
  return x;
}

__global__ void k_uf_init(int32_t n, int *__restrict__ parent) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = (int)i;
}

// x and y in one tree; self-loops and repeated edges are harmless
__device__ __forceinline__ void uf_link(int *parent, int x, int y) {
  int a = uf_find(parent, x), b = uf_find(parent, y);
  while (a != b) {
    if (a > b) { const int t2 = a; a = b; b = t2; }
    const int old = atomicCAS(parent + b, b, a);  // b is a root: hang it under a
    if (old == b) break;
    a = uf_find(parent, a);
    b = uf_find(parent, old);
  }
}

// every node links with its neighbour number r (rows are sorted, so the
// smallest ids first)
__global__ void k_uf_sample(int32_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, int r,
                            int *parent) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int e = __ldg(rowptr + v) + r;
    if (e < __ldg(rowptr + v + 1)) uf_link(parent, (int)v, __ldg(colidx + e));
  }
}

// parent[v] = root of v (no links run meanwhile, so the roots hold still)
__global__ void k_uf_compress(int32_t n, int *parent) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    parent[v] = uf_find(parent, (int)v);
}

// one block of kUfSamples threads: the most frequent root among the
// compressed parents of kUfSamples evenly spaced nodes (ties: the smaller id)
constexpr int kUfSamples = 256;
__global__ void __launch_bounds__(kUfSamples) k_uf_guess(int32_t n, const int *__restrict__ parent,
                                                         unsigned *__restrict__ big) {
  __shared__ int root[kUfSamples];
  __shared__ unsigned long long best[kUfSamples / 32];
  const int t = threadIdx.x;
  root[t] = __ldcg(parent + (int)((int64_t)t * n / kUfSamples));
  __syncthreads();
  unsigned cnt = 0;
  for (int j = 0; j < kUfSamples; ++j) cnt += root[j] == root[t];
  // largest count, then smallest root
  unsigned long long key = ((unsigned long long)cnt << 32) | (unsigned)(0x7FFFFFFF - root[t]);
  for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
  if ((t & 31) == 0) best[t >> 5] = key;
  __syncthreads();
  if (t == 0) {
    for (int w = 1; w < kUfSamples / 32; ++w) key = max(key, best[w]);
    *big = (unsigned)(0x7FFFFFFF - (int)(key & 0xFFFFFFFFu));
  }
}

// nodes outside the guessed large component link their remaining edges
__global__ void k_uf_finish(int32_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                            const unsigned *__restrict__ big, int *parent) {
  const int c = (int)__ldg(big);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (__ldcg(parent + v) == c) continue;
    const int e1 = __ldg(rowptr + v + 1);
    for (int e = __ldg(rowptr + v) + 2; e < e1; ++e) uf_link(parent, (int)v, __ldg(colidx + e));
  }
}

__global__ void k_uf_roots(int32_t n, const int *__restrict__ parent, unsigned *__restrict__ roots) {
  unsigned c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += (__ldcg(parent + i) == (int)i);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(roots, c);
}

struct BuildWs {
  int *deg, *off, *cursor, *flag, *pos, *tiles;
  int32_t *tmp;
  unsigned *big_rows, *big_count;
  int32_t *status;
  int *parent;
  unsigned *roots;
};

static size_t carve_build(Carver &c, BuildWs &w, int32_t n, int64_t m_in) {
  const int64_t e2 = 2 * m_in;
  w.deg = c.take<int>(n);
  w.off = c.take<int>((size_t)n + 1);
  w.cursor = c.take<int>(n);
  w.tmp = c.take<int32_t>((size_t)(e2 > 0 ? e2 : 1));
  w.flag = c.take<int>((size_t)(e2 > 0 ? e2 : 1));
  w.pos = c.take<int>((size_t)e2 + 1);
  int64_t tiles = scan_tiles(e2 > n ? e2 : n);
  w.tiles = c.take<int>((size_t)(tiles > 0 ? tiles : 1));
  w.big_rows = c.take<unsigned>(n);
  w.big_count = c.take<unsigned>(1);
  w.status = c.take<int32_t>(2);
  w.parent = c.take<int>(n);
  w.roots = c.take<unsigned>(4);  // components, then the two row classes
  return c.size();
}

}  // namespace ssm

SSM_API size_t ssm_build_graph_workspace(int32_t n, int64_t m_in) {
  if (n < 1 || m_in < 0) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::BuildWs w;
  return ssm::carve_build(c, w, n, m_in);
}

SSM_API int ssm_build_graph(int32_t n, int64_t m_in, const int32_t *src, const int32_t *dst, int32_t *rowptr,
                            int32_t *colidx, int64_t *m_out, int32_t *row_classes, void *ws, size_t ws_bytes,
                            cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || m_in < 0 || !rowptr || !colidx || !m_out || !ws || (m_in > 0 && (!src || !dst)))
    return fail(SSM_E_ARG, "ssm_build_graph: null pointer or bad size (n=%d, m_in=%lld)", n, (long long)m_in);
  if (2 * m_in >= ((int64_t)1 << 31)) return fail(SSM_E_ARG, "ssm_build_graph: 2*m_in must be below 2^31");
  Carver c(ws, ws_bytes);
  BuildWs w;
  carve_build(c, w, n, m_in);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_build_graph: workspace %zu bytes, need %zu", ws_bytes, c.size());
  const int sms = num_sms();
  const int eblocks = (int)std::min<int64_t>((m_in + 255) / 256 + 1, (int64_t)sms * 16);
  const int nblocks = (int)std::min<int64_t>(((int64_t)n + 255) / 256 + 1, (int64_t)sms * 16);
  SSM_TRY_CUDA(cudaMemsetAsync(w.deg, 0, (size_t)n * sizeof(int), s));
  SSM_TRY_CUDA(cudaMemsetAsync(w.cursor, 0, (size_t)n * sizeof(int), s));
  SSM_TRY_CUDA(cudaMemsetAsync(w.big_count, 0, sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(w.status, 0, 2 * sizeof(int32_t), s));
  note_launch(), k_count_degrees<<<eblocks, 256, 0, s>>>(m_in, src, dst, n, w.deg, w.status);
  int rc = exclusive_scan(w.deg, w.off, n, w.tiles, s);
  if (rc) return rc;
  note_launch(), k_scatter<<<eblocks, 256, 0, s>>>(m_in, src, dst, n, w.off, w.cursor, w.tmp);
  note_launch(), k_sort_small_rows<<<nblocks, 256, 0, s>>>(n, w.off, w.tmp, w.big_rows, w.big_count);
  note_launch(), k_sort_big_rows<<<sms * 2, kSortBlock, 0, s>>>(w.off, w.tmp, w.big_rows, w.big_count);
  note_launch(), k_flag_unique<<<2 * eblocks, 256, 0, s>>>(w.off + n, w.tmp, w.flag);
  note_launch(), k_flag_row_starts<<<nblocks, 256, 0, s>>>(n, w.off, w.flag);
  // total directed entries before dedupe = off[n]; read it to size the scan
  int total = 0;
  SSM_TRY_CUDA(cudaMemcpyAsync(&total, w.off + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  int32_t hstatus = 0;
  SSM_TRY_CUDA(cudaMemcpyAsync(&hstatus, w.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SSM_TRY_CUDA(cudaStreamSynchronize(s));
  if (hstatus) return fail(hstatus, "ssm_build_graph: %s", ssm_status_string(hstatus));
  rc = exclusive_scan(w.flag, w.pos, total, w.tiles, s);
  if (rc) return rc;
  note_launch(), k_compact<<<std::max(eblocks, nblocks), 256, 0, s>>>(n, total, w.off, w.tmp, w.flag, w.pos, rowptr, colidx);
  SSM_TRY_CUDA(cudaGetLastError());
  int32_t uniq = 0;
  SSM_TRY_CUDA(cudaMemcpyAsync(&uniq, rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SSM_TRY_CUDA(cudaStreamSynchronize(s));
  *m_out = uniq / 2;
  // connectivity: union-find over the final CSR (roots[3]: the large component's root)
  SSM_TRY_CUDA(cudaMemsetAsync(w.roots, 0, 4 * sizeof(unsigned), s));
  note_launch(), k_uf_init<<<nblocks, 256, 0, s>>>(n, w.parent);
  for (int r = 0; r < 2; ++r) note_launch(), k_uf_sample<<<nblocks, 256, 0, s>>>(n, rowptr, colidx, r, w.parent);
  note_launch(), k_uf_compress<<<nblocks, 256, 0, s>>>(n, w.parent);
  note_launch(), k_uf_guess<<<1, kUfSamples, 0, s>>>(n, w.parent, w.roots + 3);
  note_launch(), k_uf_finish<<<nblocks, 256, 0, s>>>(n, rowptr, colidx, w.roots + 3, w.parent);
  note_launch(), k_uf_roots<<<nblocks, 256, 0, s>>>(n, w.parent, w.roots);
  // the sweep's row classes, read back with the component count
  if (row_classes) note_launch(), k_row_classes<<<nblocks, 256, 0, s>>>(n, rowptr, w.roots + 1);
  unsigned hr[3] = {0, 0, 0};
  SSM_TRY_CUDA(cudaMemcpyAsync(hr, w.roots, sizeof hr, cudaMemcpyDeviceToHost, s));
  SSM_TRY_CUDA(cudaStreamSynchronize(s));
  const unsigned roots = hr[0];
  if (row_classes) {
    row_classes[0] = (int32_t)hr[1];
    row_classes[1] = (int32_t)hr[2];
  }
  if (roots != 1) return fail(SSM_E_DISCONNECTED, "ssm_build_graph: %u connected components", roots);
  return SSM_OK;
}
