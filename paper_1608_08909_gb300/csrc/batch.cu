// Many small graphs in one launch: the Jacobi sweeps of Eq. 4 (Algorithm 1
// lines 5-10) for a whole batch of independent layouts.
//
// One block owns one graph at a time (graphs are handed out largest first
// from an atomic counter) and runs all of its iterations: the graph's
// positions X^t and X^{t+1} live in shared memory (two buffers of n float2),
// so a block needs no grid-wide barrier between iterations -- a
// __syncthreads() separates them -- and neighbour and pivot positions are
// shared-memory reads.  Per iteration a warp takes 64-node tiles of the graph
// (a lane owns two consecutive nodes, whose d_ia for one pivot arrive in one
// 32-bit word of a tiled copy of d_ip, streamed from HBM with the next
// pivots' words in flight), sums the pivot terms in packed FP32x2 with the
// clamped s table (the single-graph sweep's clamped mode: q = d^2 r^2,
// u = q^-1/2, B = s u = w d / r, W = B u r^2 = w), then walks the two nodes'
// CSR rows for the neighbour terms (ascending column order) and writes the
// new positions into the other buffer.  In the last iteration each tile adds
// (sum |x^{t+1} - x^t|^2, sum |x^t|^2) in FP64, and the block reduces the
// tiles in order for the graph's relative change.
//
// ssm_batch_iterate wraps, for the whole batch, a setup kernel (per-graph s
// tables and tiled d_ip), the counter reset and the sweep kernel in one CUDA
// graph and launches it once.  The block size is tuned on the batch itself
// unless the caller fixes it: each candidate runs a few iterations on a
// scratch copy of the positions, timed with CUDA events.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace ssm {

constexpr int kBatchMaxN = 12288;     // nodes per graph: X^t and X^{t+1} in shared memory
constexpr int kBatchMaxK = 1024;
constexpr int kBatchPrefetch = 8;
constexpr float kBatchR2Floor = 1e-24f;

struct BatchDev {
  int32_t n, k, cnt_len, ppt;  // ppt: node pairs per tile of the tiled d_ip copy (32 or 64)
  int64_t node_off, row_off, col_off, piv_off, dip_off, cnt_off_off, cnt_base;
  int64_t dtile_off, stab_off;
};

struct BatchArgs {
  int32_t G, iters;
  const BatchDev *desc;
  const int32_t *order;  // graphs, largest first
  const int32_t *rowptr, *colidx, *pivots, *cnt_off;
  const uint32_t *cnt;
  const uint16_t *dip;
  unsigned *dtile;
  float *stab;
  float2 *pos;
  double *rel_change;
  unsigned *ctr;
  int32_t *status;
};

__device__ __forceinline__ unsigned bword(uint2 w, int j) { return j == 0 ? w.x : w.y; }
__device__ __forceinline__ unsigned bword(unsigned w, int) { return w; }

__device__ __forceinline__ float b_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// per graph (block b: graph b, or order[b] with use_order): the clamped s
// table (s by d at 2 off_a + a: 0 below 2, cnt[min(d/2, ecc)] up to d =
// 2 ecc + 2, larger d clamped there; with do_stab) and d_ip re-laid in tiles
// of P = ppt node pairs: word (t k + a) P + q holds d(a, 2(t P + q)) |
// d(a, 2(t P + q) + 1) << 16 (0 past the last node) -- a lane owning
// 2 P / 32 consecutive nodes reads its P / 32 words of a pivot together
__global__ void k_batch_setup(BatchArgs A, int use_order, int do_stab) {
  const int gi = use_order ? __ldg(A.order + blockIdx.x) : (int)blockIdx.x;
  const BatchDev D = A.desc[gi];
  const int32_t *off = A.cnt_off + D.cnt_off_off;
  if (do_stab)
    for (int a = 0; a < D.k; ++a) {
      const int o = __ldg(off + a), ecc = __ldg(off + a + 1) - o - 1;
      for (int d = threadIdx.x; d <= 2 * ecc + 2; d += blockDim.x)
        A.stab[D.stab_off + 2 * o + a + d] = d >= 2 ? (float)__ldg(A.cnt + D.cnt_base + o + min(d >> 1, ecc)) : 0.f;
    }
  const int P = D.ppt;
  const int tiles = (D.n + 2 * P - 1) / (2 * P), total = tiles * D.k * P;  // below 2^31: n <= 12288, k <= 1024
  const uint16_t *dip = A.dip + D.dip_off;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    const int q = w % P, ta = w / P;
    const int a = ta % D.k;
    const int i = 2 * ((ta / D.k) * P + q);
    const uint16_t *row = dip + (size_t)a * D.n;
    const unsigned lo = i < D.n ? (unsigned)__ldg(row + i) : 0u;
    const unsigned hi = i + 1 < D.n ? (unsigned)__ldg(row + i + 1) : 0u;
    A.dtile[D.dtile_off + w] = lo | (hi << 16);
  }
}

// words of a graph's tiled copy, room for either tile shape (128-node tiles)
static int64_t batch_words(int32_t n, int32_t k) { return (int64_t)((n + 127) / 128) * k * 64; }

// shared memory: X[2][nmax] float2, pivot node[kmax], pivot table (base, clamp)[kmax],
// tile partials [2][tmax], then (TAB_SMEM) the graph's s table [smax].
// NPL: nodes per lane (2: 64-node tiles, one 32-bit word of two distances per
// lane and pivot; 4: 128-node tiles, two words); the update is the
// single-graph sweep's form about x_i: x_i + (sum_a (B - W)(x_i - x_p) +
// sum_j (x_j - x_i)(1 - 1/r)) / (deg(i) + sum_a W)
template <int THREADS, bool TAB_SMEM, int NPL>
__global__ void __launch_bounds__(THREADS, 1) k_sweep_batch(BatchArgs A, int32_t nmax, int32_t kmax) {
  constexpr int PPL = NPL / 2;    // node pairs per lane
  constexpr int TN = 32 * NPL;    // nodes per tile
  using DW = typename std::conditional<PPL == 2, uint2, unsigned>::type;
  extern __shared__ __align__(16) unsigned char bsm[];
  float2 *X0 = reinterpret_cast<float2 *>(bsm);
  float2 *X1 = X0 + nmax;
  int32_t *pnode = reinterpret_cast<int32_t *>(X1 + nmax);
  uint2 *pidx = reinterpret_cast<uint2 *>(pnode + ((kmax + 1) & ~1));
  double *tpart = reinterpret_cast<double *>(pidx + kmax);
  float *stab_s = reinterpret_cast<float *>(tpart + 2 * ((nmax + 63) / 64));
  __shared__ int s_g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = THREADS / 32;

  for (;;) {
    if (threadIdx.x == 0) s_g = (int)atomicAdd(A.ctr, 1u);
    __syncthreads();
    const int gslot = s_g;
    __syncthreads();
    if (gslot >= A.G) break;
    const int gi = __ldg(A.order + gslot);
    const BatchDev D = A.desc[gi];
    const int n = D.n, k = D.k;
    const int tiles = (n + TN - 1) / TN;
    float2 *pos = A.pos + D.node_off;
    for (int i = threadIdx.x; i < n; i += THREADS) X0[i] = pos[i];
    const int tab_len = 2 * D.cnt_len + k;
    if (TAB_SMEM)
      for (int t = threadIdx.x; t < tab_len; t += THREADS) stab_s[t] = __ldg(A.stab + D.stab_off + t);
    // s of distance d for pivot a sits at stab[base_a + min(d, D_a)], base_a = the
    // graph's table start + 2 off_a + a, D_a = 2 ecc_a + 2; min(d, D_a) is taken
    // on 2^23 + d as a float, whose low bits are the integer
    for (int a = threadIdx.x; a < k; a += THREADS) {
      int p = __ldg(A.pivots + D.piv_off + a);
      if ((unsigned)p >= (unsigned)n) {
        dev_fail(A.status, SSM_E_GRAPH);
        p = 0;
      }
      pnode[a] = p;
      const int o = __ldg(A.cnt_off + D.cnt_off_off + a), e = __ldg(A.cnt_off + D.cnt_off_off + a + 1);
      pidx[a] = make_uint2((unsigned)((TAB_SMEM ? 0 : D.stab_off) + 2 * (int64_t)o + a), 0x4B000000u | (2u * (unsigned)(e - o)));
    }
    __syncthreads();
    const int32_t *rowptr = A.rowptr + D.row_off;
    const int32_t *colidx = A.colidx + D.col_off;
    const DW *dt = reinterpret_cast<const DW *>(A.dtile + D.dtile_off);
    const float *stab = TAB_SMEM ? stab_s : A.stab;

    for (int it = 0; it < A.iters; ++it) {
      const float2 *Xc = (it & 1) ? X1 : X0;
      float2 *Xn = (it & 1) ? X0 : X1;
      const bool last = it + 1 == A.iters;
      for (int tile = warp; tile < tiles; tile += kWarps) {
        const int i0 = tile * TN + NPL * lane;
        float2 xs[NPL], xi2[PPL], yi2[PPL], ax2[PPL], ay2[PPL], den2[PPL];
#pragma unroll
        for (int q = 0; q < NPL; ++q) xs[q] = i0 + q < n ? Xc[i0 + q] : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < PPL; ++j) {
          xi2[j] = make_float2(xs[2 * j].x, xs[2 * j + 1].x);
          yi2[j] = make_float2(xs[2 * j].y, xs[2 * j + 1].y);
          ax2[j] = ay2[j] = den2[j] = make_float2(0.f, 0.f);
        }
        const DW *tp = dt + (size_t)tile * (size_t)k * 32u + lane;
        const float2 kTiny2 = make_float2(kBatchR2Floor, kBatchR2Floor), kTinyQ2 = make_float2(1e-36f, 1e-36f);
        const float2 kMagic2 = make_float2(-8388608.f, -8388608.f), kMinus2 = make_float2(-1.f, -1.f);
        auto term = [&](int a, DW pw) {
          const float2 P = Xc[pnode[a]];
          const uint2 I = pidx[a];
          const float cap = __uint_as_float(I.y);
          const float2 px2 = make_float2(-P.x, -P.x), py2 = make_float2(-P.y, -P.y);
#pragma unroll
          for (int j = 0; j < PPL; ++j) {
            const unsigned pk = bword(pw, j);
            float2 f2;
            f2.x = __uint_as_float(__byte_perm(pk, 0x4B00u, 0x5410u));
            f2.y = __uint_as_float(__byte_perm(pk, 0x4B00u, 0x5432u));
            float2 s2;
            const unsigned ix = I.x + (__float_as_uint(fminf(f2.x, cap)) - 0x4B000000u);
            const unsigned iy = I.x + (__float_as_uint(fminf(f2.y, cap)) - 0x4B000000u);
            s2.x = TAB_SMEM ? stab[ix] : __ldg(stab + ix);
            s2.y = TAB_SMEM ? stab[iy] : __ldg(stab + iy);
            const float2 d2 = __fadd2_rn(f2, kMagic2);
            const float2 dx2 = __fadd2_rn(xi2[j], px2);
            const float2 dy2 = __fadd2_rn(yi2[j], py2);
            // r^2 + 1e-24 (r == 0 adds w x_p only); + 1e-36 keeps q > 0 at d = 0
            const float2 r2 = __ffma2_rn(dx2, dx2, __ffma2_rn(dy2, dy2, kTiny2));
            const float2 q2 = __ffma2_rn(__fmul2_rn(d2, d2), r2, kTinyQ2);
            float2 u2;
            u2.x = b_rsqrt(q2.x);
            u2.y = b_rsqrt(q2.y);
            const float2 B2 = __fmul2_rn(s2, u2);
            const float2 W2 = __fmul2_rn(__fmul2_rn(B2, u2), r2);
            const float2 c2 = __ffma2_rn(W2, kMinus2, B2);  // B - W
            ax2[j] = __ffma2_rn(c2, dx2, ax2[j]);
            ay2[j] = __ffma2_rn(c2, dy2, ay2[j]);
            den2[j] = __fadd2_rn(den2[j], W2);
          }
        };
        DW buf[kBatchPrefetch];
        int a0 = 0;
        if (k >= 2 * kBatchPrefetch) {
#pragma unroll
          for (int t = 0; t < kBatchPrefetch; ++t) buf[t] = __ldg(tp + (unsigned)t * 32u);
          for (; a0 + 2 * kBatchPrefetch <= k; a0 += kBatchPrefetch) {
#pragma unroll
            for (int t = 0; t < kBatchPrefetch; ++t) {
              const DW pw = buf[t];
              buf[t] = __ldg(tp + (unsigned)(a0 + kBatchPrefetch + t) * 32u);
              term(a0 + t, pw);
            }
          }
#pragma unroll
          for (int t = 0; t < kBatchPrefetch; ++t) term(a0 + t, buf[t]);
          a0 += kBatchPrefetch;
        }
        for (; a0 < k; ++a0) term(a0, __ldg(tp + (unsigned)a0 * 32u));

        // neighbour terms (w = 1, d = 1) less deg(i) x_i, in ascending column
        // order, X^t from shared memory; then the update about x_i
        float cn = 0.f, cd = 0.f;
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
          const int i = i0 + q;
          const int j = q >> 1;
          const bool hi = (q & 1) != 0;
          if (i >= n) continue;
          const float dq = hi ? den2[j].y : den2[j].x;
          if (!(dq == dq)) dev_fail(A.status, SSM_E_NUMERIC);
          const float2 x = xs[q];
          const int rb = __ldg(rowptr + i), re = __ldg(rowptr + i + 1);
          float sx = 0.f, sy = 0.f;
          for (int t = rb; t < re; ++t) {
            const unsigned c = (unsigned)__ldg(colidx + t);
            if (c >= (unsigned)n) {
              dev_fail(A.status, SSM_E_GRAPH);
              continue;
            }
            const float2 qv = Xc[c];
            const float ex = qv.x - x.x, ey = qv.y - x.y;
            const float rr = fmaf(ex, ex, ey * ey);
            const float f = rr > 0.f ? 1.f - b_rsqrt(rr) : 0.f;
            sx = fmaf(ex, f, sx);
            sy = fmaf(ey, f, sy);
          }
          const float dn = dq + (float)(re - rb);
          const float nx = hi ? ax2[j].y : ax2[j].x, ny = hi ? ay2[j].y : ay2[j].x;
          const float ex = dn > 0.f ? (nx + sx) / dn : 0.f, ey = dn > 0.f ? (ny + sy) / dn : 0.f;
          Xn[i] = make_float2(x.x + ex, x.y + ey);
          cn = fmaf(ex, ex, fmaf(ey, ey, cn));
          cd = fmaf(x.x, x.x, fmaf(x.y, x.y, cd));
        }
        if (last) {
          double tn = (double)cn, td = (double)cd;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            tn += __shfl_xor_sync(0xffffffffu, tn, o);
            td += __shfl_xor_sync(0xffffffffu, td, o);
          }
          if (lane == 0) {
            tpart[2 * tile] = tn;
            tpart[2 * tile + 1] = td;
          }
        }
      }
      __syncthreads();
    }
    const float2 *Xf = (A.iters & 1) ? X1 : X0;
    for (int i = threadIdx.x; i < n; i += THREADS) pos[i] = Xf[i];
    if (threadIdx.x == 0) {
      double num = 0.0, den = 0.0;
      for (int t = 0; t < tiles; ++t) {
        num += tpart[2 * t];
        den += tpart[2 * t + 1];
      }
      A.rel_change[gi] = den > 0.0 ? sqrt(num) / sqrt(den) : 0.0;
    }
    __syncthreads();
  }
}

static size_t batch_smem(int nmax, int kmax, int smax) {
  const int tmax = (nmax + 63) / 64;
  return 2 * (size_t)nmax * sizeof(float2) + (size_t)((kmax + 1) & ~1) * sizeof(int32_t) + (size_t)kmax * sizeof(uint2) +
         2 * (size_t)tmax * sizeof(double) + (size_t)smax * sizeof(float);
}

struct BatchWs {
  BatchDev *desc;
  int32_t *order;
  unsigned *dtile;
  float *stab;
  float2 *scratch;
  unsigned *ctr;
};

static size_t carve_batch(Carver &c, BatchWs &w, int32_t G, int64_t words, int64_t stab_len, int64_t nodes) {
  w.desc = c.take<BatchDev>((size_t)std::max(G, 1));
  w.order = c.take<int32_t>((size_t)std::max(G, 1));
  w.dtile = c.take<unsigned>((size_t)std::max<int64_t>(words, 1));
  w.stab = c.take<float>((size_t)std::max<int64_t>(stab_len, 1));
  w.scratch = c.take<float2>((size_t)std::max<int64_t>(nodes, 1));
  w.ctr = c.take<unsigned>(4);
  return c.size();
}

static void batch_sizes(int32_t G, const ssm_batch_graph *g, int64_t &words, int64_t &stab_len, int64_t &nodes) {
  words = stab_len = nodes = 0;
  for (int32_t i = 0; i < G; ++i) {
    words += batch_words(g[i].n, g[i].k);
    stab_len += 2 * (int64_t)g[i].cnt_len + g[i].k;
    nodes += g[i].n;
  }
}

typedef void (*BatchKernel)(BatchArgs, int32_t, int32_t);
template <int NPL>
static BatchKernel batch_kernel_npl(int threads, bool tab_smem) {
  switch (threads) {
    case 128: return tab_smem ? k_sweep_batch<128, true, NPL> : k_sweep_batch<128, false, NPL>;
    case 256: return tab_smem ? k_sweep_batch<256, true, NPL> : k_sweep_batch<256, false, NPL>;
    case 512: return tab_smem ? k_sweep_batch<512, true, NPL> : k_sweep_batch<512, false, NPL>;
    default: return nullptr;
  }
}
static BatchKernel batch_kernel(int threads, bool tab_smem = false, int npl = 2) {
  return npl == 4 ? batch_kernel_npl<4>(threads, tab_smem) : npl == 2 ? batch_kernel_npl<2>(threads, tab_smem) : nullptr;
}

// the s tables go to shared memory when the largest one fits beside the positions
static int batch_table_floats(int nmax, int kmax, int smax) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return batch_smem(nmax, kmax, smax) + 64 <= (size_t)optin ? smax : 0;
}

// grid of the persistent kernel for a block size (attribute and occupancy
// queries stay outside stream capture)
static int batch_grid(int threads, int npl, int nmax, int kmax, int smax, int G, int *blocks) {
  BatchKernel kern = batch_kernel(threads, smax > 0, npl);
  const size_t smem = batch_smem(nmax, kmax, smax);
  SSM_TRY_CUDA(allow_dynamic_smem((const void *)kern));
  int per_sm = 0;
  SSM_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)kern, threads, smem));
  if (per_sm < 1) return fail(SSM_E_ARG, "ssm_batch_iterate: %zu bytes of shared memory do not fit", smem);
  *blocks = std::max(1, std::min(per_sm * num_sms(), G));
  return SSM_OK;
}

static int launch_batch_sweep(const BatchArgs &A, int threads, int npl, int blocks, int nmax, int kmax, int smax,
                              cudaStream_t s) {
  SSM_TRY_CUDA(cudaMemsetAsync(A.ctr, 0, sizeof(unsigned), s));
  note_launch(), batch_kernel(threads, smax > 0, npl)<<<blocks, threads, batch_smem(nmax, kmax, smax), s>>>(A, nmax, kmax);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

}  // namespace ssm

SSM_API size_t ssm_batch_iterate_workspace(int32_t G, const ssm_batch_graph *graphs) {
  if (G < 1 || !graphs) return 0;
  int64_t words, stab_len, nodes;
  ssm::batch_sizes(G, graphs, words, stab_len, nodes);
  ssm::Carver c(nullptr, 0);
  ssm::BatchWs w;
  return ssm::carve_batch(c, w, G, words, stab_len, nodes);
}

SSM_API int ssm_batch_iterate(int32_t G, const ssm_batch_graph *graphs, const int32_t *rowptr, const int32_t *colidx,
                              const int32_t *pivots, const uint16_t *dip, const int32_t *cnt_off, const uint32_t *cnt,
                              float *pos, int32_t iters, double *rel_change, int32_t threads, int32_t nodes_per_lane,
                              int32_t *shape_used, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (G < 1 || !graphs || !rowptr || !colidx || !pivots || !dip || !cnt_off || !cnt || !pos || !rel_change ||
      !status || !ws)
    return fail(SSM_E_ARG, "ssm_batch_iterate: null pointer or G < 1");
  if (iters < 1) return fail(SSM_E_ARG, "ssm_batch_iterate: iters must be >= 1");
  if (threads != 0 && !batch_kernel(threads)) return fail(SSM_E_ARG, "ssm_batch_iterate: threads must be 0, 128, 256 or 512");
  if (nodes_per_lane != 0 && nodes_per_lane != 2 && nodes_per_lane != 4)
    return fail(SSM_E_ARG, "ssm_batch_iterate: nodes_per_lane must be 0, 2 or 4");
  int nmax = 1, kmax = 1;
  std::vector<BatchDev> dv((size_t)G);
  int64_t words = 0, stab_len = 0, tmax_len = 0;
  for (int32_t i = 0; i < G; ++i) {
    const ssm_batch_graph &g = graphs[i];
    if (g.n < 1 || g.n > kBatchMaxN) return fail(SSM_E_ARG, "ssm_batch_iterate: graph %d has n = %d (1..%d)", i, g.n, kBatchMaxN);
    if (g.k < 1 || g.k > g.n || g.k > kBatchMaxK) return fail(SSM_E_ARG, "ssm_batch_iterate: graph %d has k = %d", i, g.k);
    if (g.cnt_len < g.k) return fail(SSM_E_ARG, "ssm_batch_iterate: graph %d has cnt_len < k", i);
    if (stab_len + 2 * (int64_t)g.cnt_len + g.k >= ((int64_t)1 << 31))
      return fail(SSM_E_ARG, "ssm_batch_iterate: count tables of the batch too long");
    BatchDev &d = dv[(size_t)i];
    d.n = g.n; d.k = g.k; d.cnt_len = g.cnt_len; d.ppt = 32;
    d.node_off = g.node_off; d.row_off = g.row_off; d.col_off = g.col_off; d.piv_off = g.piv_off;
    d.dip_off = g.dip_off; d.cnt_off_off = g.cnt_off_off; d.cnt_base = g.cnt_base;
    d.dtile_off = words; d.stab_off = stab_len;
    words += batch_words(g.n, g.k);
    stab_len += 2 * (int64_t)g.cnt_len + g.k;
    nmax = std::max(nmax, g.n);
    kmax = std::max(kmax, g.k);
    tmax_len = std::max<int64_t>(tmax_len, 2 * (int64_t)g.cnt_len + g.k);
  }
  (void)nmax; (void)kmax; (void)tmax_len;
  // size classes: a kernel's shared memory is sized for its largest graph,
  // so small graphs run in their own launch with many blocks per SM; each
  // class has its own order (largest work first), counter and block size
  constexpr int kClasses = 3;
  const int kClassMax[kClasses] = {1024, 4096, kBatchMaxN};
  std::vector<int32_t> order;
  order.reserve((size_t)G);
  struct Cls {
    int first, count, nmax, kmax, smax, threads, npl, blocks;
    int64_t work;
  } cls[kClasses];
  for (int ci = 0; ci < kClasses; ++ci) {
    Cls &C = cls[ci];
    C.first = (int)order.size();
    C.nmax = 1; C.kmax = 1; C.work = 0;
    int64_t tl = 0;
    for (int32_t i = 0; i < G; ++i) {
      const int lo = ci == 0 ? 0 : kClassMax[ci - 1];
      if (graphs[i].n <= lo || graphs[i].n > kClassMax[ci]) continue;
      order.push_back(i);
      C.nmax = std::max(C.nmax, graphs[i].n);
      C.kmax = std::max(C.kmax, graphs[i].k);
      tl = std::max<int64_t>(tl, 2 * (int64_t)graphs[i].cnt_len + graphs[i].k);
      C.work += (int64_t)graphs[i].n * graphs[i].k;
    }
    C.count = (int)order.size() - C.first;
    std::stable_sort(order.begin() + C.first, order.end(), [&](int32_t a, int32_t b) {
      return (int64_t)dv[(size_t)a].n * dv[(size_t)a].k > (int64_t)dv[(size_t)b].n * dv[(size_t)b].k;
    });
    C.smax = C.count ? batch_table_floats(C.nmax, C.kmax, (int)std::min<int64_t>(tl, 1 << 24)) : 0;
    C.threads = threads;
    C.npl = nodes_per_lane != 0 ? nodes_per_lane : (threads != 0 ? 2 : 0);
    C.blocks = 0;
  }
  // a tuned shape is kept per class fingerprint (largest n, largest k, table
  // floats, graph count, sum of n k) for the life of the process
  using ShapeKey = std::tuple<int, int, int, int, int, int64_t, int>;
  static std::map<ShapeKey, std::pair<int, int>> shape_cache;
  static std::mutex shape_mu;
  auto key_of = [&](int ci) {
    const Cls &C = cls[ci];
    return ShapeKey(ci, C.nmax, C.kmax, C.smax, C.count, C.work, nodes_per_lane);
  };
  bool tune = false;
  for (int ci = 0; ci < kClasses; ++ci) {
    Cls &C = cls[ci];
    if (!C.count || (C.threads != 0 && C.npl != 0)) continue;
    std::lock_guard<std::mutex> lk(shape_mu);
    const auto it = shape_cache.find(key_of(ci));
    if (it != shape_cache.end()) {
      C.threads = it->second.first;
      C.npl = it->second.second;
    } else {
      tune = true;
    }
  }
  int64_t nodes = 0;
  for (int32_t i = 0; i < G; ++i) nodes = std::max<int64_t>(nodes, graphs[i].node_off + graphs[i].n);
  Carver c(ws, ws_bytes);
  BatchWs w;
  carve_batch(c, w, G, words, stab_len, nodes);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_batch_iterate: workspace %zu bytes, need %zu", ws_bytes, c.size());
  SSM_TRY_CUDA(cudaMemcpyAsync(w.desc, dv.data(), dv.size() * sizeof(BatchDev), cudaMemcpyHostToDevice, s));
  SSM_TRY_CUDA(cudaMemcpyAsync(w.order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));

  BatchArgs A;
  A.G = G; A.iters = iters; A.desc = w.desc; A.order = w.order; A.rowptr = rowptr; A.colidx = colidx;
  A.pivots = pivots; A.cnt_off = cnt_off; A.cnt = cnt; A.dip = dip; A.dtile = w.dtile; A.stab = w.stab;
  A.pos = reinterpret_cast<float2 *>(pos); A.rel_change = rel_change; A.ctr = w.ctr; A.status = status;
  auto class_args = [&](const BatchArgs &base, int ci) {
    BatchArgs X = base;
    X.G = cls[ci].count;
    X.order = w.order + cls[ci].first;
    X.ctr = w.ctr + ci;
    return X;
  };

  // each class's graphs carry its tile shape (pairs per tile) in their descriptors
  auto set_class_ppt = [&](int ci, int npl) {
    for (int q = cls[ci].first; q < cls[ci].first + cls[ci].count; ++q) dv[(size_t)order[(size_t)q]].ppt = 16 * npl;
  };
  auto upload_desc = [&]() -> int {
    SSM_TRY_CUDA(cudaMemcpyAsync(w.desc, dv.data(), dv.size() * sizeof(BatchDev), cudaMemcpyHostToDevice, s));
    return SSM_OK;
  };
  // the tiled copies of one class (or of every graph) for the shapes in dv
  auto setup = [&](int ci, int do_stab) -> int {
    if (ci < 0) {
      note_launch(), k_batch_setup<<<G, 256, 0, s>>>(A, 0, do_stab);
    } else {
      note_launch(), k_batch_setup<<<cls[ci].count, 256, 0, s>>>(class_args(A, ci), 1, do_stab);
    }
    SSM_TRY_CUDA(cudaGetLastError());
    return SSM_OK;
  };

  if (tune) {
    // tune block size and nodes per lane of every class not fixed or cached:
    // a few iterations per candidate on a scratch copy of the positions
    BatchArgs T = A;
    T.pos = w.scratch;
    T.iters = std::min(iters, 4);
    cudaEvent_t e0, e1;
    SSM_TRY_CUDA(cudaEventCreate(&e0));
    SSM_TRY_CUDA(cudaEventCreate(&e1));
    int rc = SSM_OK;
    bool stab_done = false;
    for (int ci = 0; ci < kClasses && rc == SSM_OK; ++ci) {
      Cls &C = cls[ci];
      if (!C.count || (C.threads != 0 && C.npl != 0)) continue;
      const BatchArgs TC = class_args(T, ci);
      float best = 0.f;
      int bt = 0, bn = 0;
      for (int npl : {2, 4}) {
        if (C.npl != 0 && npl != C.npl) continue;
        set_class_ppt(ci, npl);
        if ((rc = upload_desc()) || (rc = setup(stab_done ? ci : -1, stab_done ? 0 : 1))) break;
        stab_done = true;
        for (int cand : {128, 256, 512}) {
          if (C.threads != 0 && cand != C.threads) continue;
          for (int rep = 0; rep < 2 && rc == SSM_OK; ++rep) {  // the first run of a candidate warms it up
            SSM_TRY_CUDA(cudaMemcpyAsync(w.scratch, pos, (size_t)nodes * sizeof(float2), cudaMemcpyDeviceToDevice, s));
            int blocks = 0;
            if ((rc = batch_grid(cand, npl, C.nmax, C.kmax, C.smax, C.count, &blocks))) break;
            SSM_TRY_CUDA(cudaEventRecord(e0, s));
            if ((rc = launch_batch_sweep(TC, cand, npl, blocks, C.nmax, C.kmax, C.smax, s))) break;
            SSM_TRY_CUDA(cudaEventRecord(e1, s));
            SSM_TRY_CUDA(cudaEventSynchronize(e1));
          }
          if (rc) break;
          float ms = 0.f;
          SSM_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (bt == 0 || ms < best) {
            best = ms;
            bt = cand;
            bn = npl;
          }
        }
        if (rc) break;
      }
      if (rc) break;
      C.threads = bt;
      C.npl = bn;
      std::lock_guard<std::mutex> lk(shape_mu);
      shape_cache[key_of(ci)] = std::make_pair(bt, bn);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
  }
  // the chosen shapes: descriptors, s tables and tiled copies of every graph
  for (int ci = 0; ci < kClasses; ++ci)
    if (cls[ci].count) set_class_ppt(ci, cls[ci].npl);
  if (int rc = upload_desc()) return rc;
  if (int rc = setup(-1, 1)) return rc;
  int heavy = 0;
  for (int ci = 0; ci < kClasses; ++ci)
    if (cls[ci].work > cls[heavy].work) heavy = ci;
  if (shape_used) {
    shape_used[0] = cls[heavy].threads;
    shape_used[1] = cls[heavy].npl;
  }
  for (int ci = 0; ci < kClasses; ++ci) {
    if (!cls[ci].count) continue;
    const int rc = batch_grid(cls[ci].threads, cls[ci].npl, cls[ci].nmax, cls[ci].kmax, cls[ci].smax, cls[ci].count,
                              &cls[ci].blocks);
    if (rc) return rc;
  }

  // the sweeps of the whole batch: one CUDA graph (per class a counter reset
  // and a persistent kernel, the classes on forked branches so that their
  // kernels can share the GPU), launched once; recorded on private streams
  // (the caller's may be the legacy default stream, which cannot be
  // captured), launched on the caller's
  cudaStream_t cs[kClasses + 1] = {};
  cudaEvent_t ev[kClasses + 1] = {};
  for (int q = 0; q <= kClasses; ++q) {
    SSM_TRY_CUDA(cudaStreamCreateWithFlags(&cs[q], cudaStreamNonBlocking));
    SSM_TRY_CUDA(cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming));
  }
  auto cleanup = [&]() {
    for (int q = 0; q <= kClasses; ++q) {
      cudaStreamDestroy(cs[q]);
      cudaEventDestroy(ev[q]);
    }
  };
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs[0], cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cleanup();
    SSM_TRY_CUDA(e);
  }
  int rc = SSM_OK;
  if ((e = cudaEventRecord(ev[kClasses], cs[0])) == cudaSuccess) {
    for (int ci = 0; ci < kClasses && rc == SSM_OK && e == cudaSuccess; ++ci) {
      if (!cls[ci].count) continue;
      if ((e = cudaStreamWaitEvent(cs[ci + 1], ev[kClasses], 0)) != cudaSuccess) break;
      rc = launch_batch_sweep(class_args(A, ci), cls[ci].threads, cls[ci].npl, cls[ci].blocks, cls[ci].nmax,
                              cls[ci].kmax, cls[ci].smax, cs[ci + 1]);
      if (rc == SSM_OK) e = cudaEventRecord(ev[ci], cs[ci + 1]);
      if (rc == SSM_OK && e == cudaSuccess) e = cudaStreamWaitEvent(cs[0], ev[ci], 0);
    }
  }
  cudaError_t e2 = cudaStreamEndCapture(cs[0], &graph);
  cleanup();
  if (rc || e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (rc) return rc;
    SSM_TRY_CUDA(e != cudaSuccess ? e : e2);
  }
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
  if (exec) cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  SSM_TRY_CUDA(e);
  return SSM_OK;
}
