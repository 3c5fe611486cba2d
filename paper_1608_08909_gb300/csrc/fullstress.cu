// Full stress majorization (Section 3, the localized update before Eq. 4):
//   x_i = sum_{j != i} w_ij (x_j + d_ij (x_i - x_j)/r_ij) / sum_{j != i} w_ij,
//   w_ij = d_ij^-2,  r = ||x_i - x_j||  (a term with r == 0 adds w_ij x_j),
// over an all-pairs hop-distance table D (row-major n x n uint16), and the
// sparse model's update of Eq. 4 in the paper's in-place order (Algorithm 1
// lines 6-10).  These are the quality references of the sparse model: the
// paper compares its layouts with full stress, and states that with k = n
// its model reduces to it.
//
// Orders:
//  * Jacobi (every node from X^t): one thread per node, the other nodes'
//    positions staged 256 at a time in shared memory, terms in ascending j;
//    D is read as D[j n + i] (symmetric), so a warp reads 32 consecutive
//    entries of one row.  FP64 rounds every operation explicitly in the
//    order the oracle uses (bit-identical); FP32 uses one rsqrt per term
//    (q = d^2 r^2, u = q^-1/2, B = u = w d / r, W = B u r^2 = w).
//  * Gauss-Seidel (nodes 0..n-1 in turn, each from the positions already
//    moved, FP64): inherently sequential over nodes, so one block of 1024
//    threads sums each node's terms in parallel (thread t takes every
//    1024th term in ascending order, then a fixed-order tree), writes the
//    node, and moves on after a block barrier.
// The relative change ||X^{t+1}-X^t||_F / ||X^t||_F of the last iteration is
// reduced in FP64 in a fixed order by one block.
#include <algorithm>

#include "common.cuh"

namespace ssm {

constexpr int kFullThreads = 256;
constexpr int kGsThreads = 1024;

__device__ __forceinline__ double fs_dist_rn(double dx, double dy) {
  return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

__device__ __forceinline__ float fs_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// one Jacobi iteration, FP64, in the oracle's operation order
__global__ void __launch_bounds__(kFullThreads) k_full_jacobi_f64(int32_t n, const uint16_t *__restrict__ D,
                                                                  const double2 *__restrict__ pin,
                                                                  double2 *__restrict__ pout,
                                                                  int32_t *__restrict__ status) {
  __shared__ double2 xj_s[kFullThreads];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  const double2 xi = live ? pin[i] : make_double2(0.0, 0.0);
  double nx = 0.0, ny = 0.0, den = 0.0;
  bool bad = false;
  for (int j0 = 0; j0 < n; j0 += kFullThreads) {
    __syncthreads();
    if (j0 + (int)threadIdx.x < n) xj_s[threadIdx.x] = pin[j0 + threadIdx.x];
    __syncthreads();
    const int jn = min(kFullThreads, n - j0);
    if (!live) continue;
    for (int t = 0; t < jn; ++t) {
      const int j = j0 + t;
      if (j == i) continue;
      const unsigned dv = __ldg(D + (size_t)j * n + i);
      if (dv == 0xFFFFu) {
        bad = true;
        continue;
      }
      const double d = (double)dv;
      const double w = __ddiv_rn(1.0, __dmul_rn(d, d));
      const double2 xj = xj_s[t];
      const double dx = __dsub_rn(xi.x, xj.x), dy = __dsub_rn(xi.y, xj.y);
      const double r = fs_dist_rn(dx, dy);
      if (r > 0.0) {
        nx = __dadd_rn(nx, __dmul_rn(w, __dadd_rn(xj.x, __ddiv_rn(__dmul_rn(d, dx), r))));
        ny = __dadd_rn(ny, __dmul_rn(w, __dadd_rn(xj.y, __ddiv_rn(__dmul_rn(d, dy), r))));
      } else {
        nx = __dadd_rn(nx, __dmul_rn(w, xj.x));
        ny = __dadd_rn(ny, __dmul_rn(w, xj.y));
      }
      den = __dadd_rn(den, w);
    }
  }
  if (!live) return;
  if (bad) dev_fail(status, SSM_E_DISCONNECTED);
  pout[i] = den > 0.0 ? make_double2(__ddiv_rn(nx, den), __ddiv_rn(ny, den)) : xi;
}

// one Jacobi iteration, FP32, one rsqrt per term
__global__ void __launch_bounds__(kFullThreads) k_full_jacobi_f32(int32_t n, const uint16_t *__restrict__ D,
                                                                  const float2 *__restrict__ pin,
                                                                  float2 *__restrict__ pout,
                                                                  int32_t *__restrict__ status) {
  __shared__ float2 xj_s[kFullThreads];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  const float2 xi = live ? pin[i] : make_float2(0.f, 0.f);
  // two-level sums: each chunk of 256 terms is summed from zero and then added
  // to the totals, so rounding grows with sqrt(256) + sqrt(n / 256) terms
  // instead of sqrt(n)
  float WX = 0.f, WY = 0.f, BX = 0.f, BY = 0.f, DEN = 0.f;
  bool bad = false;
  for (int j0 = 0; j0 < n; j0 += kFullThreads) {
    __syncthreads();
    if (j0 + (int)threadIdx.x < n) xj_s[threadIdx.x] = pin[j0 + threadIdx.x];
    __syncthreads();
    const int jn = min(kFullThreads, n - j0);
    if (!live) continue;
    float wx = 0.f, wy = 0.f, bx = 0.f, by = 0.f, den = 0.f;
#pragma unroll 4
    for (int t = 0; t < jn; ++t) {
      const int j = j0 + t;
      const unsigned dv = __ldg(D + (size_t)j * n + i);
      bad |= dv == 0xFFFFu && j != i;
      // j == i (d = 0) contributes nothing: W = B = 0 below
      const float d = j == i ? 0.f : (float)dv;
      const float2 xj = xj_s[t];
      const float dx = xi.x - xj.x, dy = xi.y - xj.y;
      // r^2 + 1e-24: coincident points (r == 0) add w x_j only; + 1e-36 keeps q > 0 at d = 0
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, 1e-24f));
      const float q = fmaf(d * d, r2, 1e-36f);
      const float u = fs_rsqrt(q);
      const float B = d > 0.f ? u : 0.f;  // w d / r
      const float W = B * u * r2;          // w = 1 / d^2
      wx = fmaf(W, xj.x, wx);
      wy = fmaf(W, xj.y, wy);
      bx = fmaf(B, dx, bx);
      by = fmaf(B, dy, by);
      den += W;
    }
    WX += wx;
    WY += wy;
    BX += bx;
    BY += by;
    DEN += den;
  }
  if (!live) return;
  if (bad) dev_fail(status, SSM_E_DISCONNECTED);
  pout[i] = DEN > 0.f ? make_float2((WX + BX) / DEN, (WY + BY) / DEN) : xi;
}

template <class T>
__device__ __forceinline__ T block_sum_fixed(T v, T *red) {
  // fixed-order tree: warp shuffles, then warp results in warp order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = (T)0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;  // valid in thread 0
}

// Gauss-Seidel sweeps of full stress, FP64, one block: pos is updated in place
__global__ void __launch_bounds__(kGsThreads) k_full_gs_f64(int32_t n, const uint16_t *__restrict__ D, double2 *pos,
                                                            int32_t iters, double2 *__restrict__ prev,
                                                            int32_t *__restrict__ status) {
  __shared__ double red[kGsThreads / 32];
  bool bad = false;
  for (int it = 0; it < iters; ++it) {
    if (it == iters - 1)
      for (int i = threadIdx.x; i < n; i += blockDim.x) prev[i] = pos[i];
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      const double2 xi = pos[i];
      double nx = 0.0, ny = 0.0, den = 0.0;
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        if (j == i) continue;
        const unsigned dv = __ldg(D + (size_t)j * n + i);
        if (dv == 0xFFFFu) {
          bad = true;
          continue;
        }
        const double d = (double)dv;
        const double w = __ddiv_rn(1.0, __dmul_rn(d, d));
        const double2 xj = pos[j];
        const double dx = __dsub_rn(xi.x, xj.x), dy = __dsub_rn(xi.y, xj.y);
        const double r = fs_dist_rn(dx, dy);
        if (r > 0.0) {
          nx = __dadd_rn(nx, __dmul_rn(w, __dadd_rn(xj.x, __ddiv_rn(__dmul_rn(d, dx), r))));
          ny = __dadd_rn(ny, __dmul_rn(w, __dadd_rn(xj.y, __ddiv_rn(__dmul_rn(d, dy), r))));
        } else {
          nx = __dadd_rn(nx, __dmul_rn(w, xj.x));
          ny = __dadd_rn(ny, __dmul_rn(w, xj.y));
        }
        den = __dadd_rn(den, w);
      }
      nx = block_sum_fixed(nx, red);
      ny = block_sum_fixed(ny, red);
      den = block_sum_fixed(den, red);
      if (threadIdx.x == 0) pos[i] = den > 0.0 ? make_double2(__ddiv_rn(nx, den), __ddiv_rn(ny, den)) : xi;
      __syncthreads();
    }
  }
  if (bad) dev_fail(status, SSM_E_DISCONNECTED);
}

// Gauss-Seidel sweeps of the sparse model (Eq. 4 in Algorithm 1's in-place
// order), FP64, one block: node i's deg(i) + k terms are spread over the
// threads (term index t: neighbour t < deg(i), else pivot t - deg(i)), each
// thread adds its terms in ascending index order, the block adds the
// threads' sums in a fixed tree, and node i moves before node i + 1 starts
__global__ void __launch_bounds__(kGsThreads) k_sparse_gs_f64(int32_t n, const int32_t *__restrict__ rowptr,
                                                              const int32_t *__restrict__ colidx, int32_t k,
                                                              const int32_t *__restrict__ pivots,
                                                              const uint16_t *__restrict__ dip,
                                                              const int32_t *__restrict__ cnt_off,
                                                              const uint32_t *__restrict__ cnt, double2 *pos,
                                                              int32_t iters, double2 *__restrict__ prev,
                                                              int32_t *__restrict__ status) {
  __shared__ double red[kGsThreads / 32];
  for (int a = threadIdx.x; a < k; a += blockDim.x)
    if ((unsigned)__ldg(pivots + a) >= (unsigned)n) dev_fail(status, SSM_E_ARG);
  for (int it = 0; it < iters; ++it) {
    if (it == iters - 1)
      for (int i = threadIdx.x; i < n; i += blockDim.x) prev[i] = pos[i];
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      const double2 xi = pos[i];
      const int rb = __ldg(rowptr + i), deg = __ldg(rowptr + i + 1) - rb;
      double nx = 0.0, ny = 0.0, den = 0.0;
      for (int t = threadIdx.x; t < deg + k; t += blockDim.x) {
        if (t < deg) {
          const double2 xj = pos[__ldg(colidx + rb + t)];
          const double dx = __dsub_rn(xi.x, xj.x), dy = __dsub_rn(xi.y, xj.y);
          const double r = fs_dist_rn(dx, dy);
          if (r > 0.0) {
            nx = __dadd_rn(nx, __dadd_rn(xj.x, __ddiv_rn(dx, r)));
            ny = __dadd_rn(ny, __dadd_rn(xj.y, __ddiv_rn(dy, r)));
          } else {
            nx = __dadd_rn(nx, xj.x);
            ny = __dadd_rn(ny, xj.y);
          }
          den = __dadd_rn(den, 1.0);
          continue;
        }
        const int a = t - deg;
        const int d = __ldg(dip + (size_t)a * n + i);
        if (d < 2) continue;
        const int o = __ldg(cnt_off + a), ecc = __ldg(cnt_off + a + 1) - o - 1;
        const double sv = (double)__ldg(cnt + o + min(d >> 1, ecc));
        const double dd = (double)d;
        const double w = __ddiv_rn(sv, __dmul_rn(dd, dd));
        int p = __ldg(pivots + a);
        if ((unsigned)p >= (unsigned)n) p = 0;
        const double2 xp = pos[p];
        const double dx = __dsub_rn(xi.x, xp.x), dy = __dsub_rn(xi.y, xp.y);
        const double r = fs_dist_rn(dx, dy);
        if (r > 0.0) {
          nx = __dadd_rn(nx, __dmul_rn(w, __dadd_rn(xp.x, __ddiv_rn(__dmul_rn(dd, dx), r))));
          ny = __dadd_rn(ny, __dmul_rn(w, __dadd_rn(xp.y, __ddiv_rn(__dmul_rn(dd, dy), r))));
        } else {
          nx = __dadd_rn(nx, __dmul_rn(w, xp.x));
          ny = __dadd_rn(ny, __dmul_rn(w, xp.y));
        }
        den = __dadd_rn(den, w);
      }
      nx = block_sum_fixed(nx, red);
      ny = block_sum_fixed(ny, red);
      den = block_sum_fixed(den, red);
      if (threadIdx.x == 0) pos[i] = den > 0.0 ? make_double2(__ddiv_rn(nx, den), __ddiv_rn(ny, den)) : xi;
      __syncthreads();
    }
  }
}

// relative change ||X' - X||_F / ||X||_F in FP64, one block, fixed order
template <class V>
__global__ void __launch_bounds__(1024) k_full_relchange(int32_t n, const V *__restrict__ before,
                                                         const V *__restrict__ after, double *__restrict__ out) {
  __shared__ double red[32];
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const V a = before[i], b = after[i];
    const double ex = (double)b.x - (double)a.x, ey = (double)b.y - (double)a.y;
    num += ex * ex + ey * ey;
    den += (double)a.x * (double)a.x + (double)a.y * (double)a.y;
  }
  num = block_sum_fixed(num, red);
  den = block_sum_fixed(den, red);
  if (threadIdx.x == 0) *out = den > 0.0 ? sqrt(num) / sqrt(den) : 0.0;
}

template <class V>
__global__ void k_full_copy(int32_t n, const V *__restrict__ src, V *__restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace ssm

SSM_API size_t ssm_full_iterate_workspace(int32_t n, int32_t precision) {
  if (n < 1 || (precision != 32 && precision != 64)) return 0;
  ssm::Carver c(nullptr, 0);
  c.take<char>((size_t)n * (precision == 64 ? sizeof(double2) : sizeof(float2)));
  return c.size();
}

SSM_API int ssm_full_iterate(int32_t n, const uint16_t *D, void *pos, int32_t precision, int32_t order, int32_t iters,
                             double *rel_change, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !D || !pos || !rel_change || !status || !ws) return fail(SSM_E_ARG, "ssm_full_iterate: null pointer or bad size");
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_full_iterate: precision must be 32 or 64");
  if (order != 0 && order != 1) return fail(SSM_E_ARG, "ssm_full_iterate: order must be 0 (Jacobi) or 1 (Gauss-Seidel)");
  if (order == 1 && precision != 64) return fail(SSM_E_ARG, "ssm_full_iterate: the Gauss-Seidel order runs in FP64");
  if (iters < 1) return fail(SSM_E_ARG, "ssm_full_iterate: iters must be >= 1");
  if ((int64_t)n * n >= ((int64_t)1 << 40)) return fail(SSM_E_ARG, "ssm_full_iterate: n too large");
  Carver c(ws, ws_bytes);
  void *tmp = c.take<char>((size_t)n * (precision == 64 ? sizeof(double2) : sizeof(float2)));
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_full_iterate: workspace %zu bytes, need %zu", ws_bytes, c.size());
  const unsigned blocks = (unsigned)((n + kFullThreads - 1) / kFullThreads);
  const int cb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)num_sms() * 8);
  if (order == 1) {
    note_launch(), k_full_gs_f64<<<1, kGsThreads, 0, s>>>(n, D, (double2 *)pos, iters, (double2 *)tmp, status);
    note_launch(), k_full_relchange<double2><<<1, 1024, 0, s>>>(n, (const double2 *)tmp, (const double2 *)pos, rel_change);
    SSM_TRY_CUDA(cudaGetLastError());
    return SSM_OK;
  }
  // Jacobi: ping-pong between pos and tmp; an odd count ends in tmp and is copied back
  for (int t = 0; t < iters; ++t) {
    void *pin = (t & 1) ? tmp : pos, *pout = (t & 1) ? pos : tmp;
    if (precision == 64)
      note_launch(), k_full_jacobi_f64<<<blocks, kFullThreads, 0, s>>>(n, D, (const double2 *)pin, (double2 *)pout, status);
    else
      note_launch(), k_full_jacobi_f32<<<blocks, kFullThreads, 0, s>>>(n, D, (const float2 *)pin, (float2 *)pout, status);
    if (t == iters - 1) {
      if (precision == 64)
        note_launch(), k_full_relchange<double2><<<1, 1024, 0, s>>>(n, (const double2 *)pin, (const double2 *)pout, rel_change);
      else
        note_launch(), k_full_relchange<float2><<<1, 1024, 0, s>>>(n, (const float2 *)pin, (const float2 *)pout, rel_change);
    }
  }
  if (iters & 1) {
    if (precision == 64)
      note_launch(), k_full_copy<double2><<<cb, 256, 0, s>>>(n, (const double2 *)tmp, (double2 *)pos);
    else
      note_launch(), k_full_copy<float2><<<cb, 256, 0, s>>>(n, (const float2 *)tmp, (float2 *)pos);
  }
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

SSM_API size_t ssm_iterate_gs_workspace(int32_t n) {
  if (n < 1) return 0;
  ssm::Carver c(nullptr, 0);
  c.take<double2>((size_t)n);
  return c.size();
}

SSM_API int ssm_iterate_gs(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                           const int32_t *pivots, const uint16_t *dip, const int32_t *cnt_off, const uint32_t *cnt,
                           double *pos, int32_t iters, double *rel_change, int32_t *status, void *ws, size_t ws_bytes,
                           cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || m < 0 || !rowptr || !colidx || !pivots || !dip || !cnt_off || !cnt || !pos || !rel_change || !status || !ws)
    return fail(SSM_E_ARG, "ssm_iterate_gs: null pointer or bad size");
  if (k < 1 || k > 65535) return fail(SSM_E_ARG, "ssm_iterate_gs: need 1 <= k <= 65535");
  if (iters < 1) return fail(SSM_E_ARG, "ssm_iterate_gs: iters must be >= 1");
  Carver c(ws, ws_bytes);
  double2 *prev = c.take<double2>((size_t)n);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_iterate_gs: workspace %zu bytes, need %zu", ws_bytes, c.size());
  note_launch(), k_sparse_gs_f64<<<1, kGsThreads, 0, s>>>(n, rowptr, colidx, k, pivots, dip, cnt_off, cnt,
                                                         (double2 *)pos, iters, prev, status);
  note_launch(), k_full_relchange<double2><<<1, 1024, 0, s>>>(n, prev, (const double2 *)pos, rel_change);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
