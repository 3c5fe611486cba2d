// Stress majorization sweep (Eq. 4; Algorithm 1 lines 5-10) in the Jacobi
// schedule: every x_i^{t+1} is computed from X^t, so one kernel launch is one
// iteration and the only device-wide dependency is the kernel boundary.
//
// Per node i (Eq. 4, unit edge lengths, w_ij = 1 on edges):
//   num = sum_{j in N(i)} (x_j + (x_i - x_j)/r_ij)
//       + sum_{a: d_ia >= 2} w'_ia (x_pa + d_ia (x_i - x_pa)/r_ia)
//   den = deg(i) + sum_{a: d_ia >= 2} w'_ia,   x_i^{t+1} = num / den
//   w'_ia = s / d_ia^2,  s = cnt[cnt_off[a] + min(floor(d_ia/2), ecc_a)]
// A term with r == 0 contributes w * x_j only.  d_ia <= 1 skips the pivot
// (the pivot itself, or a neighbour already counted as an edge term).
//
// GB300 layout: the k pivot positions and the count tables sit in shared
// memory (loaded once per persistent block), d_ip is streamed from HBM with
// one coalesced row segment per pivot per warp, neighbour positions are
// gathered from L2.  Warps take 32*NPT-node tiles from an atomic counter so
// uneven rows balance across the 152 SMs; nodes of very high degree are
// processed by the whole warp.  The relative change ||X^{t+1}-X^t||/||X^t||
// is reduced in FP64 in a fixed order by the last block to finish.
#include <algorithm>

#include "common.cuh"

namespace ssm {

constexpr int kSweepThreads = 256;
constexpr int kHeavyDegree = 64;  // rows longer than this are walked by the whole warp
constexpr size_t kSmemBudget = 160 * 1024;
constexpr int kMaxPivotsSweep = 4096;

struct SweepArgs {
  int32_t n, k;
  const int32_t *rowptr, *colidx, *pivots, *cnt_off;
  const uint16_t *dip;
  const uint32_t *cnt;
  int32_t cnt_len;
  int32_t cnt_in_smem;
  unsigned *tile_ctr;    // next tile to hand out
  unsigned *done_ctr;    // blocks finished
  double *tile_part;     // [ntiles][2] (sum dx^2, sum x^2) per tile
  int32_t *stop;         // set when the relative change fell below tol
  int32_t *iters_done;
  double *rel_change;
  double tol;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// last block: reduce the tile partials in a fixed order, publish the change
__device__ void finish_iteration(const SweepArgs &A, unsigned ntiles) {
  __shared__ unsigned s_ticket;
  __shared__ double s_red[2][kSweepThreads / 32];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(A.done_ctr, 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  double num = 0.0, den = 0.0;
  for (unsigned t = threadIdx.x; t < ntiles; t += blockDim.x) {
    num += __ldcg(A.tile_part + 2 * (size_t)t);
    den += __ldcg(A.tile_part + 2 * (size_t)t + 1);
  }
  num = warp_sum(num);
  den = warp_sum(den);
  if ((threadIdx.x & 31) == 0) {
    s_red[0][threadIdx.x >> 5] = num;
    s_red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    num = 0.0;
    den = 0.0;
    for (int w = 0; w < kSweepThreads / 32; ++w) {
      num += s_red[0][w];
      den += s_red[1][w];
    }
    const double rel = den > 0.0 ? sqrt(num) / sqrt(den) : 0.0;
    *A.rel_change = rel;
    *A.iters_done += 1;
    if (A.tol > 0.0 && rel < A.tol) *A.stop = 1;
    *A.tile_ctr = 0;
    *A.done_ctr = 0;
  }
}

// ----------------------------------------------------------------- FP32
template <int NPT>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_f32(SweepArgs A, const float2 *__restrict__ pin,
                                                              float2 *__restrict__ pout) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4 *piv = reinterpret_cast<float4 *>(smem);  // x, y, cnt_off (bits), ecc (bits)
  float *cntf = reinterpret_cast<float *>(piv + A.k);
  if (__ldcg(A.stop)) return;
  const int n = A.n, k = A.k;
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    const int p = __ldg(A.pivots + a);
    const float2 xy = pin[p];
    const int o = __ldg(A.cnt_off + a);
    const int e = __ldg(A.cnt_off + a + 1) - o - 1;
    piv[a] = make_float4(xy.x, xy.y, __int_as_float(o), __int_as_float(e));
  }
  if (A.cnt_in_smem)
    for (int t = threadIdx.x; t < A.cnt_len; t += blockDim.x) cntf[t] = (float)__ldg(A.cnt + t);
  __syncthreads();

  const unsigned lane = threadIdx.x & 31u;
  const unsigned ntiles = (unsigned)((n + 32 * NPT - 1) / (32 * NPT));
  const bool vec = (n % NPT) == 0;
  for (;;) {
    unsigned tile = 0;
    if (lane == 0) tile = atomicAdd(A.tile_ctr, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= ntiles) break;
    const int i0 = (int)(tile * 32u * NPT + lane * NPT);

    float xi[NPT], yi[NPT], nx[NPT], ny[NPT], den[NPT];
    int beg[NPT], end[NPT];
    bool live[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const int i = i0 + j;
      live[j] = i < n;
      float2 x = live[j] ? pin[i] : make_float2(0.f, 0.f);
      xi[j] = x.x;
      yi[j] = x.y;
      nx[j] = 0.f;
      ny[j] = 0.f;
      beg[j] = live[j] ? __ldg(A.rowptr + i) : 0;
      end[j] = live[j] ? __ldg(A.rowptr + i + 1) : 0;
      den[j] = (float)(end[j] - beg[j]);
    }

    // ---- neighbour terms (w = 1, d = 1), CSR order
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      if (end[j] - beg[j] <= kHeavyDegree) {
        for (int t = beg[j]; t < end[j]; ++t) {
          const float2 q = pin[__ldg(A.colidx + t)];
          const float dx = xi[j] - q.x, dy = yi[j] - q.y;
          const float r2 = fmaf(dx, dx, dy * dy);
          const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
          nx[j] += fmaf(dx, inv, q.x);
          ny[j] += fmaf(dy, inv, q.y);
        }
      }
      unsigned heavy = __ballot_sync(0xffffffffu, end[j] - beg[j] > kHeavyDegree);
      while (heavy) {
        const int src = __ffs(heavy) - 1;
        heavy &= heavy - 1u;
        const int hb = __shfl_sync(0xffffffffu, beg[j], src), he = __shfl_sync(0xffffffffu, end[j], src);
        const float hx = __shfl_sync(0xffffffffu, xi[j], src), hy = __shfl_sync(0xffffffffu, yi[j], src);
        float sx = 0.f, sy = 0.f;
        for (int t = hb + (int)lane; t < he; t += 32) {
          const float2 q = pin[__ldg(A.colidx + t)];
          const float dx = hx - q.x, dy = hy - q.y;
          const float r2 = fmaf(dx, dx, dy * dy);
          const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
          sx += fmaf(dx, inv, q.x);
          sy += fmaf(dy, inv, q.y);
        }
        sx = warp_sumf(sx);
        sy = warp_sumf(sy);
        if ((int)lane == src) {
          nx[j] += sx;
          ny[j] += sy;
        }
      }
    }

    // ---- pivot terms a = 0..k-1, d_ia streamed from HBM
    const uint16_t *col = A.dip + i0;
#pragma unroll 4
    for (int a = 0; a < k; ++a) {
      const float4 P = piv[a];
      const int off = __float_as_int(P.z), ecc = __float_as_int(P.w);
      unsigned d[NPT];
      const uint16_t *row = col + (size_t)a * n;
      if (NPT == 2 && vec) {
        const unsigned pk = live[0] ? __ldcs(reinterpret_cast<const unsigned *>(row)) : 0u;
        d[0] = pk & 0xFFFFu;
        d[NPT - 1] = pk >> 16;
      } else {
#pragma unroll
        for (int j = 0; j < NPT; ++j) d[j] = live[j] ? (unsigned)__ldcs(row + j) : 0u;
      }
#pragma unroll
      for (int j = 0; j < NPT; ++j) {
        const bool valid = d[j] >= 2u;
        const int h = min((int)(d[j] >> 1), ecc);
        const float s = valid ? (A.cnt_in_smem ? cntf[off + h] : (float)__ldg(A.cnt + off + h)) : 0.f;
        const float dx = xi[j] - P.x, dy = yi[j] - P.y;
        const float r2 = fmaf(dx, dx, dy * dy);
        const float df = (float)d[j];
        const bool ok = valid && r2 > 0.f;
        const float u = rsqrtf(ok ? df * df * r2 : 1.f);  // 1/(d r)
        const float B = ok ? s * u : 0.f;                 // w d / r = s/(d r)
        float Aw = B * u * r2;                            // w = s/d^2
        if (valid && !(r2 > 0.f)) Aw = s / (df * df);
        nx[j] = fmaf(Aw, P.x, fmaf(B, dx, nx[j]));
        ny[j] = fmaf(Aw, P.y, fmaf(B, dy, ny[j]));
        den[j] += Aw;
      }
    }

    // ---- write X^{t+1}, accumulate the change of this tile
    float cn = 0.f, cd = 0.f;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      if (!live[j]) continue;
      const float x1 = den[j] > 0.f ? nx[j] / den[j] : xi[j];
      const float y1 = den[j] > 0.f ? ny[j] / den[j] : yi[j];
      pout[i0 + j] = make_float2(x1, y1);
      const float ex = x1 - xi[j], ey = y1 - yi[j];
      cn = fmaf(ex, ex, fmaf(ey, ey, cn));
      cd = fmaf(xi[j], xi[j], fmaf(yi[j], yi[j], cd));
    }
    double tn = warp_sum((double)cn), td = warp_sum((double)cd);
    if (lane == 0) {
      A.tile_part[2 * (size_t)tile] = tn;
      A.tile_part[2 * (size_t)tile + 1] = td;
    }
  }
  finish_iteration(A, ntiles);
}

// ----------------------------------------------------------------- FP64
// The same update evaluated in plain double precision, one node per thread:
// the comparison baseline for the FP32 sweep.  Every operation is an
// explicitly rounded IEEE double operation (no fused multiply-add), taken in
// the order in which Eq. 4 is written -- neighbours in CSR order, then pivots
// a = 0..k-1 -- so its results do not depend on compiler contraction.
struct PivD {
  double x, y;
  int off, ecc;
};

__device__ __forceinline__ double dist_rn(double dx, double dy) {
  return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

__global__ void __launch_bounds__(kSweepThreads) k_sweep_f64(SweepArgs A, const double2 *__restrict__ pin,
                                                              double2 *__restrict__ pout) {
  extern __shared__ __align__(16) unsigned char smem[];
  PivD *piv = reinterpret_cast<PivD *>(smem);
  double *cntd = reinterpret_cast<double *>(piv + A.k);
  if (__ldcg(A.stop)) return;
  const int n = A.n, k = A.k;
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    const int p = __ldg(A.pivots + a);
    const double2 xy = pin[p];
    const int o = __ldg(A.cnt_off + a);
    piv[a] = PivD{xy.x, xy.y, o, __ldg(A.cnt_off + a + 1) - o - 1};
  }
  if (A.cnt_in_smem)
    for (int t = threadIdx.x; t < A.cnt_len; t += blockDim.x) cntd[t] = (double)__ldg(A.cnt + t);
  __syncthreads();

  const unsigned lane = threadIdx.x & 31u;
  const unsigned ntiles = (unsigned)((n + 31) / 32);
  for (;;) {
    unsigned tile = 0;
    if (lane == 0) tile = atomicAdd(A.tile_ctr, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= ntiles) break;
    const int i = (int)(tile * 32u + lane);
    const bool live = i < n;
    const double2 x = live ? pin[i] : make_double2(0.0, 0.0);
    double nx = 0.0, ny = 0.0, den = 0.0;
    if (live) {
      const int b = __ldg(A.rowptr + i), e = __ldg(A.rowptr + i + 1);
      for (int t = b; t < e; ++t) {
        const double2 q = pin[__ldg(A.colidx + t)];
        const double dx = __dsub_rn(x.x, q.x), dy = __dsub_rn(x.y, q.y);
        const double r = dist_rn(dx, dy);
        if (r > 0.0) {
          nx = __dadd_rn(nx, __dadd_rn(q.x, __ddiv_rn(dx, r)));
          ny = __dadd_rn(ny, __dadd_rn(q.y, __ddiv_rn(dy, r)));
        } else {
          nx = __dadd_rn(nx, q.x);
          ny = __dadd_rn(ny, q.y);
        }
        den = __dadd_rn(den, 1.0);
      }
      const uint16_t *colp = A.dip + i;
      for (int a = 0; a < k; ++a) {
        const int d = __ldcs(colp + (size_t)a * n);
        if (d < 2) continue;
        const PivD P = piv[a];
        const int h = min(d >> 1, P.ecc);
        const double s = A.cnt_in_smem ? cntd[P.off + h] : (double)__ldg(A.cnt + P.off + h);
        const double dd = (double)d;
        const double w = __ddiv_rn(s, __dmul_rn(dd, dd));
        const double dx = __dsub_rn(x.x, P.x), dy = __dsub_rn(x.y, P.y);
        const double r = dist_rn(dx, dy);
        if (r > 0.0) {
          nx = __dadd_rn(nx, __dmul_rn(w, __dadd_rn(P.x, __ddiv_rn(__dmul_rn(dd, dx), r))));
          ny = __dadd_rn(ny, __dmul_rn(w, __dadd_rn(P.y, __ddiv_rn(__dmul_rn(dd, dy), r))));
        } else {
          nx = __dadd_rn(nx, __dmul_rn(w, P.x));
          ny = __dadd_rn(ny, __dmul_rn(w, P.y));
        }
        den = __dadd_rn(den, w);
      }
    }
    double cn = 0.0, cd = 0.0;
    if (live) {
      const double x1 = den > 0.0 ? __ddiv_rn(nx, den) : x.x;
      const double y1 = den > 0.0 ? __ddiv_rn(ny, den) : x.y;
      pout[i] = make_double2(x1, y1);
      cn = (x1 - x.x) * (x1 - x.x) + (y1 - x.y) * (y1 - x.y);
      cd = x.x * x.x + x.y * x.y;
    }
    cn = warp_sum(cn);
    cd = warp_sum(cd);
    if (lane == 0) {
      A.tile_part[2 * (size_t)tile] = cn;
      A.tile_part[2 * (size_t)tile + 1] = cd;
    }
  }
  finish_iteration(A, ntiles);
}

template <class T>
__global__ void k_copy_back_if_odd(int64_t count, const int32_t *__restrict__ iters_done, const T *__restrict__ src,
                                   T *__restrict__ dst) {
  if ((*iters_done & 1) == 0) return;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = src[t];
}

struct IterWs {
  void *tmp;
  unsigned *ctr;  // [0] tile counter, [1] done counter
  int32_t *stop;
  double *tile_part;
};

static size_t carve_iterate(Carver &c, IterWs &w, int32_t n, int32_t precision) {
  const size_t elem = precision == 64 ? sizeof(double2) : sizeof(float2);
  w.tmp = c.take<char>((size_t)n * elem);
  w.ctr = c.take<unsigned>(2);
  w.stop = c.take<int32_t>(1);
  w.tile_part = c.take<double>(2 * ((size_t)n / 32 + 2));
  return c.size();
}

}  // namespace ssm

SSM_API size_t ssm_iterate_workspace(int32_t n, int32_t k, int32_t precision) {
  (void)k;
  if (n < 1) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::IterWs w;
  return ssm::carve_iterate(c, w, n, precision);
}

SSM_API int ssm_iterate(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k, const int32_t *pivots,
                        const uint16_t *dip, const int32_t *cnt_off, const uint32_t *cnt, int64_t cnt_len,
                        void *pos, int32_t precision, int32_t iters, double tol, int32_t *iters_done,
                        double *rel_change, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !rowptr || !colidx || !pivots || !dip || !cnt_off || !cnt || !pos || !iters_done || !rel_change ||
      !status || !ws)
    return fail(SSM_E_ARG, "ssm_iterate: null pointer or n < 1");
  if (k < 1 || k > kMaxPivotsSweep) return fail(SSM_E_ARG, "ssm_iterate: need 1 <= k <= %d", kMaxPivotsSweep);
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_iterate: precision must be 32 or 64");
  if (iters < 1) return fail(SSM_E_ARG, "ssm_iterate: iters must be >= 1");
  if (cnt_len < k || cnt_len >= ((int64_t)1 << 31)) return fail(SSM_E_ARG, "ssm_iterate: bad count-table length");
  Carver c(ws, ws_bytes);
  IterWs w;
  carve_iterate(c, w, n, precision);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_iterate: workspace %zu bytes, need %zu", ws_bytes, c.size());

  SweepArgs A;
  A.n = n; A.k = k; A.rowptr = rowptr; A.colidx = colidx; A.pivots = pivots; A.cnt_off = cnt_off;
  A.dip = dip; A.cnt = cnt; A.cnt_len = (int32_t)cnt_len;
  A.tile_ctr = w.ctr; A.done_ctr = w.ctr + 1; A.tile_part = w.tile_part; A.stop = w.stop;
  A.iters_done = iters_done; A.rel_change = rel_change; A.tol = tol;

  const size_t piv_bytes = (size_t)k * (precision == 64 ? sizeof(PivD) : sizeof(float4));
  const size_t tab_bytes = (size_t)cnt_len * (precision == 64 ? sizeof(double) : sizeof(float));
  A.cnt_in_smem = piv_bytes + tab_bytes <= kSmemBudget;
  const size_t smem = piv_bytes + (A.cnt_in_smem ? tab_bytes : 0);

  const void *kern;
  if (precision == 64) kern = (const void *)k_sweep_f64;
  else if (n % 2 == 0) kern = (const void *)k_sweep_f32<2>;
  else kern = (const void *)k_sweep_f32<1>;
  SSM_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SSM_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSweepThreads, smem));
  if (per_sm < 1) return fail(SSM_E_ARG, "ssm_iterate: %zu bytes of shared memory do not fit", smem);
  const int64_t tiles = precision == 64 ? (n + 31) / 32 : (n + 63) / 64;
  const int64_t want = (tiles + (kSweepThreads / 32) - 1) / (kSweepThreads / 32);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * num_sms(), want));

  SSM_TRY_CUDA(cudaMemsetAsync(w.ctr, 0, 2 * sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(w.stop, 0, sizeof(int32_t), s));
  SSM_TRY_CUDA(cudaMemsetAsync(iters_done, 0, sizeof(int32_t), s));
  SSM_TRY_CUDA(cudaMemsetAsync(rel_change, 0, sizeof(double), s));
  for (int t = 0; t < iters; ++t) {
    const bool even = (t & 1) == 0;
    if (precision == 64) {
      const double2 *pin = (const double2 *)(even ? pos : w.tmp);
      double2 *pout = (double2 *)(even ? w.tmp : pos);
      k_sweep_f64<<<blocks, kSweepThreads, smem, s>>>(A, pin, pout);
    } else if (n % 2 == 0) {
      const float2 *pin = (const float2 *)(even ? pos : w.tmp);
      float2 *pout = (float2 *)(even ? w.tmp : pos);
      k_sweep_f32<2><<<blocks, kSweepThreads, smem, s>>>(A, pin, pout);
    } else {
      const float2 *pin = (const float2 *)(even ? pos : w.tmp);
      float2 *pout = (float2 *)(even ? w.tmp : pos);
      k_sweep_f32<1><<<blocks, kSweepThreads, smem, s>>>(A, pin, pout);
    }
  }
  const int cb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)num_sms() * 8);
  if (precision == 64)
    k_copy_back_if_odd<double2><<<cb, 256, 0, s>>>(n, iters_done, (const double2 *)w.tmp, (double2 *)pos);
  else
    k_copy_back_if_odd<float2><<<cb, 256, 0, s>>>(n, iters_done, (const float2 *)w.tmp, (float2 *)pos);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
