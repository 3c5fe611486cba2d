// Regions R(p) and the per-pivot cumulative distance counts behind the
// adapted weights w'_ip = s / d_ip^2 (Section 3, after Eq. 4):
//   region[i] = lowest pivot index a minimising d_ia,
//   ecc_a     = max_{i in R(a)} d_ia,
//   cnt[cnt_off[a] + t] = |{ i in R(a) : d_ia <= t }|.
// The sweep then reads s = cnt[cnt_off[a] + min(floor(d_ia/2), ecc_a)]
// instead of a stored k x n weight table.
#include <mutex>

#include "common.cuh"

namespace ssm {

constexpr int kAggThreads = 256;

// one thread per node: nearest pivot (ties to the lowest index) and the
// per-pivot maximum distance over its region; dmax (may be null) receives
// the largest entry of the whole table
__global__ void __launch_bounds__(kAggThreads) k_region_ecc(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                                                            int32_t *__restrict__ region, unsigned *__restrict__ ecc,
                                                            unsigned *__restrict__ dmax) {
  unsigned worst = 0u;
  // the loop runs over whole warps so that lanes past n can join the warp-wide
  // aggregation below
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
    const int64_t i = i0 + (threadIdx.x & 31);
    const bool live = i < n;
    unsigned best = 0xFFFFFFFFu;
    int32_t arg = 0;
    if (live) {
      const uint16_t *col = dip + i;
      // eight pivots' distances in flight, compared in pivot order (ties to the lowest a)
      for (int32_t a0 = 0; a0 < k; a0 += 8) {
        unsigned dq[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) dq[q] = a0 + q < k ? (unsigned)__ldg(col + (size_t)(a0 + q) * n) : 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (dq[q] < best) {
            best = dq[q];
            arg = a0 + q;
          }
          if (a0 + q < k) worst = max(worst, dq[q]);
        }
      }
      if (region) region[i] = arg;
    }
    // one atomic per distinct region among the warp's nodes
    const unsigned peers = __match_any_sync(0xffffffffu, live ? arg : -1);
    const unsigned bval = live ? best : 0u;
    unsigned m = 0u;
    for (int src = 0; src < 32; ++src) {  // the maximum over this lane's group
      const unsigned t = __shfl_sync(0xffffffffu, bval, src);
      if ((peers >> src) & 1u) m = max(m, t);
    }
    if (live && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicMax(ecc + arg, m);
  }
  if (dmax) {
    for (int o = 16; o > 0; o >>= 1) worst = max(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0 && worst) atomicMax(dmax, worst);
  }
}

__global__ void k_table_len(int32_t k, const unsigned *__restrict__ ecc, long long *__restrict__ len) {
  __shared__ long long part[32];
  long long s = 0;
  for (int a = threadIdx.x; a < k; a += blockDim.x) s += (long long)ecc[a] + 1;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += part[w];
    *len = t;
  }
}

// one block: cnt_off = exclusive scan of (ecc + 1); flags a length mismatch
__global__ void k_cnt_off(int32_t k, const unsigned *__restrict__ ecc, int32_t *__restrict__ cnt_off,
                          long long expect, int32_t *__restrict__ status) {
  if (threadIdx.x != 0) return;
  long long acc = 0;
  for (int a = 0; a < k; ++a) {
    cnt_off[a] = (int32_t)acc;
    acc += (long long)ecc[a] + 1;
  }
  cnt_off[k] = (int32_t)acc;
  if (acc != expect) dev_fail(status, SSM_E_ARG);
}

__global__ void __launch_bounds__(kAggThreads) k_histogram(int32_t n, const uint16_t *__restrict__ dip,
                                                           const int32_t *__restrict__ region,
                                                           const int32_t *__restrict__ cnt_off, int64_t cnt_len,
                                                           unsigned *__restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
    const int64_t i = i0 + (threadIdx.x & 31);
    int64_t slot = -1;
    if (i < n) {
      const int32_t a = region[i];
      slot = (int64_t)cnt_off[a] + __ldg(dip + (size_t)a * n + i);
      if (slot >= cnt_len) slot = -1;
    }
    // one atomic per distinct slot among the warp's nodes
    const unsigned peers = __match_any_sync(0xffffffffu, (unsigned long long)slot);
    if (slot >= 0 && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(cnt + slot, (unsigned)__popc(peers));
  }
}

// one warp per pivot: inclusive prefix over t of the histogram row
__global__ void k_row_prefix(int32_t k, const int32_t *__restrict__ cnt_off, int64_t cnt_len,
                             unsigned *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = warp; a < k; a += nwarps) {
    const int64_t b = cnt_off[a], e = cnt_off[a + 1] < cnt_len ? cnt_off[a + 1] : cnt_len;
    unsigned carry = 0;
    for (int64_t base = b; base < e; base += 32) {
      const int64_t t = base + lane;
      unsigned v = t < e ? cnt[t] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      v += carry;
      if (t < e) cnt[t] = v;
      carry = __shfl_sync(0xffffffffu, v, 31);
    }
  }
}

// ---------------------------------------------------------------- the paper's tie rule
// Regions as Section 3 builds them: incrementally while the distances are
// computed, a tie going to the partition that is smallest at that moment.
// Nodes join in the order a multi-source search settles them (increasing distance L to the
// nearest pivot, then increasing id); a node with several nearest pivots
// joins the one whose region is smallest at that moment (lowest index on
// equal sizes).  The prepass finds each node's L and its nearest pivots
// (up to kTieCand of them, ascending); one block then walks the levels in
// order, 1024 node ids at a time: a chunk without ties adds its nodes in
// parallel (the order of unique assignments does not matter), a chunk with
// ties is walked in id order by one thread, which keeps the region sizes in
// shared memory.
constexpr int kTieCand = 4;
constexpr int kTieMaxK = 8192;

__global__ void __launch_bounds__(kAggThreads) k_tie_prepass(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                                                             uint16_t *__restrict__ L, int4 *__restrict__ cand,
                                                             int32_t *__restrict__ ncand, unsigned *__restrict__ lmax) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
    const int64_t i = i0 + (threadIdx.x & 31);
    unsigned m = 0u;
    if (i < n) {
      const uint16_t *col = dip + i;
      int c[kTieCand] = {0, 0, 0, 0};
      int cnt = 0;
      m = 0xFFFFFFFFu;
      for (int32_t a0 = 0; a0 < k; a0 += 8) {
        unsigned dq[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) dq[q] = a0 + q < k ? (unsigned)__ldg(col + (size_t)(a0 + q) * n) : 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (dq[q] < m) {
            m = dq[q];
            cnt = 0;
          }
          if (dq[q] == m && a0 + q < k) {
            if (cnt < kTieCand) c[cnt] = a0 + q;
            ++cnt;
          }
        }
      }
      L[i] = (uint16_t)m;
      ncand[i] = cnt;
      cand[i] = make_int4(c[0], c[1], c[2], c[3]);
    }
    m = __reduce_max_sync(0xffffffffu, i < n ? m : 0u);
    if ((threadIdx.x & 31) == 0) atomicMax(lmax, m);
  }
}

__global__ void __launch_bounds__(1024) k_regions_smallest(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                                                           const uint16_t *__restrict__ L,
                                                           const int4 *__restrict__ cand,
                                                           const int32_t *__restrict__ ncand,
                                                           const unsigned *__restrict__ lmax_p,
                                                           int32_t *__restrict__ region) {
  extern __shared__ unsigned tsize[];  // [k] current region sizes
  __shared__ unsigned s_in[32], s_tied[32];
  __shared__ int s_any;
  for (int a = threadIdx.x; a < k; a += blockDim.x) tsize[a] = 0u;
  const unsigned lmax = *lmax_p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (unsigned l = 0; l <= lmax; ++l) {
    for (int c = 0; c < n; c += blockDim.x) {
      const int v = c + (int)threadIdx.x;
      const bool in = v < n && (unsigned)L[v] == l;
      const int nc = in ? ncand[v] : 0;
      const unsigned bin = __ballot_sync(0xffffffffu, in), btied = __ballot_sync(0xffffffffu, in && nc > 1);
      if (threadIdx.x == 0) s_any = 0;
      __syncthreads();
      if (lane == 0) {
        s_in[warp] = bin;
        s_tied[warp] = btied;
        if (btied) s_any = 1;
      }
      __syncthreads();
      if (!s_any) {
        if (in) {
          const int a = cand[v].x;
          atomicAdd(tsize + a, 1u);
          region[v] = a;
        }
      } else if (threadIdx.x == 0) {
        // nodes of this level in id order; ties to the smallest region
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
          for (unsigned mi = s_in[w]; mi; mi &= mi - 1u) {
            const int b = __ffs(mi) - 1, node = c + 32 * w + b;
            const int4 cv = cand[node];
            int best = cv.x;
            if ((s_tied[w] >> b) & 1u) {
              const int cnt = ncand[node];
              if (cnt <= kTieCand) {
                const int cs[kTieCand] = {cv.x, cv.y, cv.z, cv.w};
                for (int q = 1; q < cnt; ++q)
                  if (tsize[cs[q]] < tsize[best]) best = cs[q];
              } else {
                best = -1;
                for (int a = 0; a < k; ++a)
                  if ((unsigned)__ldg(dip + (size_t)a * n + node) == l && (best < 0 || tsize[a] < tsize[best])) best = a;
              }
            }
            tsize[best] += 1u;
            region[node] = best;
          }
      }
      __syncthreads();
    }
  }
}

// ecc_a = max over the nodes of the given region a of d_ia
__global__ void __launch_bounds__(kAggThreads) k_ecc_given(int32_t n, const uint16_t *__restrict__ dip,
                                                           const int32_t *__restrict__ region, int32_t k,
                                                           unsigned *__restrict__ ecc, int32_t *__restrict__ status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
    const int64_t i = i0 + (threadIdx.x & 31);
    int a = -1;
    unsigned d = 0u;
    if (i < n) {
      a = region[i];
      if ((unsigned)a >= (unsigned)k) {
        dev_fail(status, SSM_E_ARG);
        a = -1;
      } else {
        d = __ldg(dip + (size_t)a * n + i);
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, a);
    unsigned mx = 0u;
    for (int src = 0; src < 32; ++src) {
      const unsigned t = __shfl_sync(0xffffffffu, d, src);
      if ((peers >> src) & 1u) mx = max(mx, t);
    }
    if (a >= 0 && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicMax(ecc + a, mx);
  }
}

static int grid_for(int64_t items, int threads) {
  int64_t b = (items + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms() * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// The same as k_region_ecc with four consecutive nodes per thread (one 8-byte
// load per pivot, so a warp reads 256 contiguous bytes of a row), for n a
// multiple of 4 and k <= kAggSmemPivots: the per-region maxima go through a
// shared-memory copy of ecc (one shared atomicMax per node, then one global
// atomicMax per pivot and block)
constexpr int kAggSmemPivots = 4096;
__global__ void __launch_bounds__(kAggThreads) k_region_ecc4(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                                                             int32_t *__restrict__ region, unsigned *__restrict__ ecc,
                                                             unsigned *__restrict__ dmax) {
  __shared__ unsigned s_ecc[kAggSmemPivots];
  for (int a = threadIdx.x; a < k; a += blockDim.x) s_ecc[a] = 0u;
  __syncthreads();
  unsigned worst = 0u;
  const int64_t n4 = n / 4;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += (int64_t)gridDim.x * blockDim.x) {
    const uint2 *col = reinterpret_cast<const uint2 *>(dip) + g;  // nodes 4g .. 4g + 3 of every row
    unsigned best[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
    int32_t arg[4] = {0, 0, 0, 0};
    // eight pivots' words in flight, compared in pivot order (ties to the lowest a)
    for (int32_t a0 = 0; a0 < k; a0 += 8) {
      uint2 w[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) w[q] = a0 + q < k ? __ldg(col + (size_t)(a0 + q) * n4) : make_uint2(0u, 0u);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (a0 + q >= k) break;
        const unsigned d[4] = {w[q].x & 0xFFFFu, w[q].x >> 16, w[q].y & 0xFFFFu, w[q].y >> 16};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          if (d[h] < best[h]) {
            best[h] = d[h];
            arg[h] = a0 + q;
          }
          worst = max(worst, d[h]);
        }
      }
    }
    if (region) reinterpret_cast<int4 *>(region)[g] = make_int4(arg[0], arg[1], arg[2], arg[3]);
#pragma unroll
    for (int h = 0; h < 4; ++h) atomicMax(s_ecc + arg[h], best[h]);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < k; a += blockDim.x)
    if (s_ecc[a]) atomicMax(ecc + a, s_ecc[a]);
  if (dmax) {
    for (int o = 16; o > 0; o >>= 1) worst = max(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0 && worst) atomicMax(dmax, worst);
  }
}

// regions and eccentricities (and the largest entry into dmax when given)
static void launch_region_ecc(int32_t n, int32_t k, const uint16_t *dip, int32_t *region, unsigned *ecc,
                              unsigned *dmax, cudaStream_t s) {
  const bool vec = n % 4 == 0 && k <= kAggSmemPivots && (reinterpret_cast<uintptr_t>(dip) & 7u) == 0 &&
                   (!region || (reinterpret_cast<uintptr_t>(region) & 15u) == 0);
  if (vec)
    note_launch(), k_region_ecc4<<<grid_for(n / 4, kAggThreads), kAggThreads, 0, s>>>(n, k, dip, region, ecc, dmax);
  else
    note_launch(), k_region_ecc<<<grid_for(n, kAggThreads), kAggThreads, 0, s>>>(n, k, dip, region, ecc, dmax);
}

}  // namespace ssm

SSM_API size_t ssm_aggregate_workspace(int32_t k) {
  ssm::Carver c(nullptr, 0);
  c.take<unsigned>(k > 0 ? k : 1);
  c.take<long long>(2);
  return c.size();
}

SSM_API int ssm_aggregate_size(int32_t n, int32_t k, const uint16_t *dip, int64_t *cnt_len, int32_t *dip_max,
                               void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || k < 1 || !dip || !cnt_len || !ws) return fail(SSM_E_ARG, "ssm_aggregate_size: bad argument");
  Carver c(ws, ws_bytes);
  unsigned *ecc = c.take<unsigned>(k);
  long long *len = c.take<long long>(2);  // the length, then the largest entry
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_aggregate_size: workspace %zu bytes, need %zu", ws_bytes, c.size());
  SSM_TRY_CUDA(cudaMemsetAsync(ecc, 0, (size_t)k * sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(len, 0, 2 * sizeof(long long), s));
  launch_region_ecc(n, k, dip, nullptr, ecc, (unsigned *)(len + 1), s);
  note_launch(), k_table_len<<<1, 256, 0, s>>>(k, ecc, len);
  long long h[2] = {0, 0};
  SSM_TRY_CUDA(cudaMemcpyAsync(h, len, sizeof h, cudaMemcpyDeviceToHost, s));
  SSM_TRY_CUDA(cudaStreamSynchronize(s));
  *cnt_len = h[0];
  if (dip_max) *dip_max = (int32_t)(unsigned)(h[1] & 0xFFFFFFFFll);
  return SSM_OK;
}

SSM_API int ssm_aggregate(int32_t n, int32_t k, const uint16_t *dip, int32_t *region, int32_t *cnt_off, uint32_t *cnt,
                          int64_t cnt_len, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || k < 1 || !dip || !region || !cnt_off || !cnt || !status || !ws || cnt_len < k)
    return fail(SSM_E_ARG, "ssm_aggregate: bad argument");
  if (cnt_len >= ((int64_t)1 << 31)) return fail(SSM_E_ARG, "ssm_aggregate: table length must be below 2^31");
  Carver c(ws, ws_bytes);
  unsigned *ecc = c.take<unsigned>(k);
  c.take<long long>(1);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_aggregate: workspace %zu bytes, need %zu", ws_bytes, c.size());
  SSM_TRY_CUDA(cudaMemsetAsync(ecc, 0, (size_t)k * sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(cnt, 0, (size_t)cnt_len * sizeof(uint32_t), s));
  launch_region_ecc(n, k, dip, region, ecc, nullptr, s);
  note_launch(), k_cnt_off<<<1, 32, 0, s>>>(k, ecc, cnt_off, (long long)cnt_len, status);
  note_launch(), k_histogram<<<grid_for(n, kAggThreads), kAggThreads, 0, s>>>(n, dip, region, cnt_off, cnt_len, cnt);
  note_launch(), k_row_prefix<<<grid_for((int64_t)k * 32, 256), 256, 0, s>>>(k, cnt_off, cnt_len, cnt);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

// ---------------------------------------------------------------- without allocation
// Scratch of ssm_aggregate_noalloc: one eccentricity per pivot and the table
// length, in a fixed device array (every GPU that loads the library holds one
// copy until the process exits).  Host code must not use the array's name as
// a device address; it asks the runtime for the address once per device.
namespace ssm {
constexpr int kNoAllocMaxPivots = 4096;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned g_agg_scratch[kNoAllocMaxPivots + 4];
static std::mutex g_agg_mutex;
static void *g_agg_addr[kNoAllocMaxDevices];

// device address of g_agg_scratch on the current device (looked up on the
// first call for that device, with that device current)
static int agg_scratch(unsigned **out) {
  int dev = 0;
  SSM_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SSM_E_ARG, "ssm_aggregate_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_agg_mutex);
  if (!g_agg_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_agg_scratch);
    if (e != cudaSuccess) return cuda_status(e, "ssm_aggregate_noalloc: cudaGetSymbolAddress");
    g_agg_addr[dev] = p;
  }
  *out = static_cast<unsigned *>(g_agg_addr[dev]);
  return SSM_OK;
}
}  // namespace ssm

SSM_API int ssm_aggregate_noalloc(int32_t n, int32_t k, const uint16_t *dip, int32_t *region, int32_t *cnt_off,
                                  uint32_t *cnt, int64_t cnt_cap, int64_t *cnt_len, int32_t *status,
                                  cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !dip || !region || !cnt_off || !cnt_len || !status || cnt_cap < 0 || (cnt_cap > 0 && !cnt))
    return fail(SSM_E_ARG, "ssm_aggregate_noalloc: null pointer or bad size");
  if (k < 1 || k > kNoAllocMaxPivots)
    return fail(SSM_E_ARG, "ssm_aggregate_noalloc: k = %d, this entry point handles 1 <= k <= %d pivots", k,
                kNoAllocMaxPivots);
  unsigned *ecc = nullptr;
  int rc = agg_scratch(&ecc);
  if (rc) return rc;
  long long *len = reinterpret_cast<long long *>(ecc + kNoAllocMaxPivots);
  SSM_TRY_CUDA(cudaMemsetAsync(ecc, 0, (size_t)k * sizeof(unsigned), s));
  launch_region_ecc(n, k, dip, region, ecc, nullptr, s);
  note_launch(), k_table_len<<<1, 256, 0, s>>>(k, ecc, len);
  long long h = 0;
  SSM_TRY_CUDA(cudaMemcpyAsync(&h, len, sizeof h, cudaMemcpyDeviceToHost, s));
  SSM_TRY_CUDA(cudaStreamSynchronize(s));
  *cnt_len = h;
  if (h > cnt_cap)
    return fail(SSM_E_NOMEM, "ssm_aggregate_noalloc: the count table needs %lld entries, cnt holds %lld", h,
                (long long)cnt_cap);
  if (h >= ((int64_t)1 << 31)) return fail(SSM_E_ARG, "ssm_aggregate_noalloc: table length must be below 2^31");
  SSM_TRY_CUDA(cudaMemsetAsync(cnt, 0, (size_t)h * sizeof(uint32_t), s));
  note_launch(), k_cnt_off<<<1, 32, 0, s>>>(k, ecc, cnt_off, h, status);
  note_launch(), k_histogram<<<grid_for(n, kAggThreads), kAggThreads, 0, s>>>(n, dip, region, cnt_off, h, cnt);
  note_launch(), k_row_prefix<<<grid_for((int64_t)k * 32, 256), 256, 0, s>>>(k, cnt_off, h, cnt);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

SSM_API size_t ssm_regions_smallest_workspace(int32_t n) {
  if (n < 1) return 0;
  ssm::Carver c(nullptr, 0);
  c.take<uint16_t>((size_t)n);
  c.take<int4>((size_t)n);
  c.take<int32_t>((size_t)n);
  c.take<unsigned>(1);
  return c.size();
}

SSM_API int ssm_regions_smallest(int32_t n, int32_t k, const uint16_t *dip, int32_t *region, int32_t *status, void *ws,
                                 size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !dip || !region || !status || !ws) return fail(SSM_E_ARG, "ssm_regions_smallest: bad argument");
  if (k < 1 || k > kTieMaxK) return fail(SSM_E_ARG, "ssm_regions_smallest: need 1 <= k <= %d", kTieMaxK);
  Carver c(ws, ws_bytes);
  uint16_t *L = c.take<uint16_t>((size_t)n);
  int4 *cand = c.take<int4>((size_t)n);
  int32_t *ncand = c.take<int32_t>((size_t)n);
  unsigned *lmax = c.take<unsigned>(1);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_regions_smallest: workspace %zu bytes, need %zu", ws_bytes, c.size());
  SSM_TRY_CUDA(cudaMemsetAsync(lmax, 0, sizeof(unsigned), s));
  note_launch(), k_tie_prepass<<<grid_for(n, kAggThreads), kAggThreads, 0, s>>>(n, k, dip, L, cand, ncand, lmax);
  SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_regions_smallest));
  note_launch(), k_regions_smallest<<<1, 1024, (size_t)k * sizeof(unsigned), s>>>(n, k, dip, L, cand, ncand, lmax, region);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

SSM_API int ssm_aggregate_regions(int32_t n, int32_t k, const uint16_t *dip, const int32_t *region, int32_t *cnt_off,
                                  uint32_t *cnt, int64_t cnt_cap, int64_t *cnt_len, int32_t *status, void *ws,
                                  size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || k < 1 || !dip || !region || !cnt_off || !cnt_len || !status || !ws || cnt_cap < 0 || (cnt_cap > 0 && !cnt))
    return fail(SSM_E_ARG, "ssm_aggregate_regions: bad argument");
  Carver c(ws, ws_bytes);
  unsigned *ecc = c.take<unsigned>(k);
  long long *len = c.take<long long>(1);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_aggregate_regions: workspace %zu bytes, need %zu", ws_bytes, c.size());
  SSM_TRY_CUDA(cudaMemsetAsync(ecc, 0, (size_t)k * sizeof(unsigned), s));
  note_launch(), k_ecc_given<<<grid_for(n, kAggThreads), kAggThreads, 0, s>>>(n, dip, region, k, ecc, status);
  note_launch(), k_table_len<<<1, 256, 0, s>>>(k, ecc, len);
  long long h = 0;
  SSM_TRY_CUDA(cudaMemcpyAsync(&h, len, sizeof h, cudaMemcpyDeviceToHost, s));
  SSM_TRY_CUDA(cudaStreamSynchronize(s));
  *cnt_len = h;
  if (h > cnt_cap)
    return fail(SSM_E_NOMEM, "ssm_aggregate_regions: the count table needs %lld entries, cnt holds %lld", h,
                (long long)cnt_cap);
  if (h >= ((int64_t)1 << 31)) return fail(SSM_E_ARG, "ssm_aggregate_regions: table length must be below 2^31");
  SSM_TRY_CUDA(cudaMemsetAsync(cnt, 0, (size_t)h * sizeof(uint32_t), s));
  note_launch(), k_cnt_off<<<1, 32, 0, s>>>(k, ecc, cnt_off, h, status);
  note_launch(), k_histogram<<<grid_for(n, kAggThreads), kAggThreads, 0, s>>>(n, dip, region, cnt_off, h, cnt);
  note_launch(), k_row_prefix<<<grid_for((int64_t)k * 32, 256), 256, 0, s>>>(k, cnt_off, h, cnt);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
