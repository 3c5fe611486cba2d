// Initial layout (Algorithm 1 lines 3-4): PivotMDS over the k pivots
// (Brandes and Pich 2007, cited by the paper) and the edge-length rescale.
//
// With Delta = [d_ia^2] (n x k) and C = -1/2 J_n Delta J_k (double centring),
//   C^T C = 1/4 J_k (Delta^T Delta - s s^T / n) J_k,   s_a = sum_i d_ia^2,
// so the only O(n k^2) work is the integer Gram matrix G = Delta^T Delta.
// G is accumulated exactly (128-bit integers), which makes it independent of
// summation order; everything after it is k x k FP64:
//   k_dmax      largest d_ia (how many digits the Gram needs)
//   k_gram_tc   G = Delta^T Delta on the tensor cores (gram_tc.cu)
//   k_colsum    s_a
//   k_prepare_b, k_row_means, k_center
//               B = 1/4 J (G - s s^T/n) J
//   k_square    M = (B / max|B|)^(2^kEigPowerLog2) by FP64 squarings (grid)
//   k_eigen     top-2 eigenpairs of B: FP64 subspace iteration on M with
//               Rayleigh-Ritz and re-orthogonalised Gram-Schmidt (a
//               cooperative grid: the k x k products over all blocks, the
//               small steps on identical copies in every block), then a
//               Rayleigh-Ritz step with B
//   k_project   x_i = C v = -1/2 (sum_a d_ia^2 v_a - rbar_i sigma - kappa),
//               the sum in compensated (two-float) FP32 arithmetic
//   k_edge_sum_* / k_rescale: scale so that sum_E ||x_i - x_j|| = m.
#include <algorithm>

#include "common.cuh"
#include "gram_tc.cuh"

namespace ssm {

#ifndef SSM_EIG_P
#define SSM_EIG_P 4
#endif
#ifndef SSM_EIG_POWER_LOG2
#define SSM_EIG_POWER_LOG2 2
#endif
constexpr int kEigP = SSM_EIG_P;  // subspace dimension
// the iteration runs on (B / max|B|)^(2^this): higher powers speed up close
// eigenvalue pairs but drown the second pair below FP64 precision when
// lambda_2 / lambda_1 is small, so the fourth power is kept
constexpr int kEigPowerLog2 = SSM_EIG_POWER_LOG2;
constexpr int kEigThreads = 256;
constexpr int kMaxPivotsMds = 1024;
constexpr int kEigScratch = (kEigThreads / 32 + 1) * (kEigP * (kEigP + 1) / 2);  // doubles for block_sum

// s_a = sum_i d_ia^2 (exact: below 2^63 for n < 2^31)
// s[a] = sum_i d_ia^2 (exact; s zeroed by the caller).  Blocks take chunks of
// kColChunk nodes of one pivot row, eight distances per 16-byte load.
constexpr int kColChunk = 65536;
__global__ void k_colsum(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                         unsigned long long *__restrict__ s) {
  __shared__ unsigned long long part[32];
  const int64_t nchunks = (n + kColChunk - 1) / kColChunk;
  for (int64_t task = blockIdx.x; task < (int64_t)k * nchunks; task += gridDim.x) {
    const int a = (int)(task / nchunks);
    const int64_t c0 = (task - (int64_t)a * nchunks) * kColChunk;
    const int64_t c1 = min((int64_t)n, c0 + kColChunk);
    const uint16_t *row = dip + (size_t)a * n;
    unsigned long long acc = 0;
    // rows start at multiples of n entries: 16-byte loads from the first aligned entry on
    int64_t v0 = c0;
    while (v0 < c1 && (((size_t)(row + v0)) & 15) != 0) ++v0;
    for (int64_t i = c0 + threadIdx.x; i < v0; i += blockDim.x) {
      const unsigned long long d = __ldg(row + i);
      acc += d * d;
    }
    const int64_t nv = (c1 - v0) / 8;
    const uint4 *vrow = reinterpret_cast<const uint4 *>(row + v0);
    for (int64_t q = threadIdx.x; q < nv; q += blockDim.x) {
      const uint4 w = __ldg(vrow + q);
      const unsigned x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const unsigned long long lo = x[h] & 0xFFFFu, hi = x[h] >> 16;
        acc += lo * lo + hi * hi;
      }
    }
    for (int64_t i = v0 + nv * 8 + threadIdx.x; i < c1; i += blockDim.x) {
      const unsigned long long d = __ldg(row + i);
      acc += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < (int)blockDim.x / 32; ++w) t += part[w];
      atomicAdd(s + a, t);
    }
    __syncthreads();
  }
}

// B = 1/4 J (G - s s^T / n) J in three steps, the element-wise ones spread
// over the grid (FP64 runs at 1/64 of the FP32 rate, so one block spent
// about 0.1 ms on the k^2 elements):
//   k_prepare_b  B[a][b] = G[a][b] - s_a s_b / n (G from its upper triangle)
__global__ void k_prepare_b(int32_t n, int32_t k, const unsigned long long *__restrict__ Glo,
                            const unsigned long long *__restrict__ Ghi, const unsigned long long *__restrict__ s,
                            double *__restrict__ B) {
  const double two64 = 18446744073709551616.0;
  const double inv_n = 1.0 / (double)n;
  const int64_t kk = (int64_t)k * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < kk; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / k), b = (int)(t - (int64_t)a * k);
    const int lo_ = min(a, b), hi_ = max(a, b);
    const size_t o = (size_t)lo_ * k + hi_;
    const double g = (double)Ghi[o] * two64 + (double)Glo[o];
    B[t] = g - ((double)s[a] * (double)s[b]) * inv_n;
  }
}

//   k_row_means  rowmean[a] = mean of row a, rowmean[k] = their mean (one
//                block of 1024 threads).  B is exactly symmetric (G from one
//                triangle, s_a s_b commutes), so row a is summed down column
//                a: the same numbers in the same order, with coalesced loads
__global__ void k_row_means(int32_t k, const double *__restrict__ B, double *__restrict__ rowmean) {
  __shared__ double red[32];
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < k; ++b) acc += B[(size_t)b * k + a];
    rowmean[a] = acc / (double)k;
  }
  __syncthreads();
  double g = 0.0;
  for (int a = threadIdx.x; a < k; a += blockDim.x) g += rowmean[a];
  for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) t += red[w];
    rowmean[k] = t / (double)k;
  }
}

//   k_center     B[a][b] = 1/4 (B[a][b] - rowmean[a] - rowmean[b] + rowmean[k])
__global__ void k_center(int32_t k, double *__restrict__ B, const double *__restrict__ rowmean) {
  const double gm = rowmean[k];
  const int64_t kk = (int64_t)k * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < kk; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / k), b = (int)(t - (int64_t)a * k);
    B[t] = 0.25 * (B[t] - rowmean[a] - rowmean[b] + gm);
  }
}

// ------------------------------------------------------------- eigen-solve
// *scale = 1 / max |B_ij| (one block)
__global__ void k_absmax_inv(int64_t count, const double *__restrict__ B, double *__restrict__ scale) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t t = threadIdx.x; t < count; t += blockDim.x) m = fmax(m, fabs(B[t]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) t = fmax(t, red[w]);
    *scale = t > 0.0 ? 1.0 / t : 1.0;
  }
}

// C = (sA)(sA) for a symmetric k x k matrix A, s = *scale (or 1): 16 x 16 output tiles
__global__ void __launch_bounds__(256) k_square_f64(int32_t k, const double *__restrict__ A,
                                                    const double *__restrict__ scale, double *__restrict__ C) {
  __shared__ double ta[16][17], tb[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r = blockIdx.y * 16 + ty, c = blockIdx.x * 16 + tx;
  const double sc = scale ? *scale : 1.0;
  double acc = 0.0;
  for (int k0 = 0; k0 < k; k0 += 16) {
    ta[ty][tx] = (r < k && k0 + tx < k) ? A[(size_t)r * k + k0 + tx] * sc : 0.0;
    tb[ty][tx] = (k0 + ty < k && c < k) ? A[(size_t)(k0 + ty) * k + c] * sc : 0.0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) acc = fma(ta[ty][t], tb[t][tx], acc);
    __syncthreads();
  }
  if (r < k && c < k) C[(size_t)r * k + c] = acc;
}

// GB300 runs FP64 at 1/64 of the FP32 rate and a warp instruction costs the
// same with one lane as with 32, so what the small k x P steps below cost is
// their count of FP64 warp instructions.

// N' = N rounded up to a power of two (N <= 32) and its log2
template <int N>
struct Halving {
  static_assert(N >= 1 && N <= 32, "1..32 values");
  static constexpr int LOG = N <= 1 ? 0 : N <= 2 ? 1 : N <= 4 ? 2 : N <= 8 ? 3 : N <= 16 ? 4 : 5;
  static constexpr int NP = 1 << LOG;
};

// warp sum of N doubles per lane by recursive halving: at each of the first
// log2 N' shuffle steps (offsets 16, 8, ...) a lane keeps one half of its
// values -- the upper half where the offset's lane bit is set -- and adds the
// partner's copy of that half; the single value left is summed over the
// remaining offsets.  Lane l ends with the total of value l >> (5 - log2 N')
// (N' - 1 + 5 - log2 N' adds per lane instead of 5 N).
template <int N>
__device__ __forceinline__ double warp_sum_halving(const double (&v)[N]) {
  constexpr int LOG = Halving<N>::LOG, NP = Halving<N>::NP;
  const int lane = threadIdx.x & 31;
  double u[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) u[j] = j < N ? v[j] : 0.0;
#pragma unroll
  for (int st = 0; st < LOG; ++st) {
    const int o = 16 >> st, h = NP >> (st + 1);
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double keep = up ? u[h + i] : u[i];
      const double send = up ? u[i] : u[h + i];
      u[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double t = u[0];
#pragma unroll
  for (int o = 16 >> LOG; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// block-wide sum of N doubles per thread (result broadcast to all threads):
// the warps' totals by recursive halving, then lanes 0..N-1 of warp 0 add
// the warps' partials of one value each, in warp order
template <int N>
__device__ void block_sum(double (&v)[N], double *scratch /* [(warps + 1) N] */) {
  constexpr int SH = 5 - Halving<N>::LOG;
  const double t = warp_sum_halving<N>(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((lane & ((1 << SH) - 1)) == 0 && (lane >> SH) < N) scratch[w * N + (lane >> SH)] = t;
  __syncthreads();
  if (w == 0 && lane < N) {
    double a = 0.0;
    for (int q = 0; q < nw; ++q) a += scratch[q * N + lane];
    scratch[nw * N + lane] = a;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < N; ++j) v[j] = scratch[nw * N + j];
  __syncthreads();
}

// (c, s) of the Jacobi rotation that zeroes h_pq.  Any t = tan(angle) gives
// an exact rotation once c = (1 + t^2)^(-1/2) and s = t c hold in FP64, so t
// comes from FP32 arithmetic (it leaves about 1e-7 of h_pq, which the next
// sweep removes) and c from Newton's method for x^(-1/2), y <- y (3 - x y^2)/2,
// twice from the FP32 reciprocal square root.  h_pq and h_qq - h_pp are
// scaled by one power of two first, so that their FP32 copies neither
// overflow nor lose h_pq (an h_pq below 2^-126 of the difference is far
// under the convergence test's threshold).
__device__ __forceinline__ void jacobi_rotation(double hpp, double hqq, double apq, double &c, double &sn) {
  const double d = hqq - hpp;
  const int ea = (__double2hiint(apq) >> 20) & 0x7FF, ed = (__double2hiint(d) >> 20) & 0x7FF;
  const int e = min(max(ea, ed), 2045);                      // biased exponent of the larger
  const double sc = __hiloint2double((2046 - e) << 20, 0);  // 2^(1023 - e): the larger to [1, 2)
  const float af = (float)(apq * sc), df = (float)(d * sc);
  const float th = df / (2.0f * af);
  const float tf = (th >= 0.0f ? 1.0f : -1.0f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
  const double t = (double)tf, x = fma(t, t, 1.0), hx = 0.5 * x;
  double y = (double)rsqrtf((float)x);
  y *= fma(-hx * y, y, 1.5);
  y *= fma(-hx * y, y, 1.5);
  c = y;
  sn = t * y;
}

// cyclic Jacobi on a tiny symmetric P x P matrix (P <= 4) by one warp: a
// sweep's six rotations in three rounds of two disjoint pairs ((0,1)(2,3),
// (0,2)(1,3), (0,3)(1,2)); lanes 0 and 1 form a round's two rotations at
// once and eight lanes apply them to columns, rows and Q.  Eigenvalues on the
// diagonal of H, eigenvectors in the columns of Q, sorted descending.  (FP64
// runs at 1/64 of the FP32 rate on GB300 and a warp instruction costs the
// same with one lane as with 32, so the serial form paid for every element.)
// round r's pair h: (0, r + 1) and the two indices left
__device__ __forceinline__ int pair_lo(int r, int h) { return h == 0 ? 0 : (r == 0 ? 2 : 1); }
__device__ __forceinline__ int pair_hi(int r, int h) { return h == 0 ? r + 1 : (r == 2 ? 2 : 3); }
__device__ __forceinline__ void tiny_jacobi_warp(int P, double *H, double *Q) {
  const int lane = threadIdx.x & 31;
  if (lane < P * P) Q[lane] = (lane / P == lane % P) ? 1.0 : 0.0;
  __syncwarp();
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    if (lane < P * P) {
      const double h = H[lane];
      tot = h * h;
      if (lane / P != lane % P) off = h * h;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (off <= 1e-32 * tot || off == 0.0) break;  // the same sums in every lane
    for (int r = 0; r < 3; ++r) {
      double c = 1.0, sn = 0.0;
      if (lane < 2) {
        const int p = pair_lo(r, lane), q = pair_hi(r, lane);
        if (q < P) {
          const double apq = H[p * P + q];
          if (apq != 0.0) jacobi_rotation(H[p * P + p], H[q * P + q], apq, c, sn);
        }
      }
      const double c0 = __shfl_sync(0xffffffffu, c, 0), s0 = __shfl_sync(0xffffffffu, sn, 0);
      const double c1 = __shfl_sync(0xffffffffu, c, 1), s1 = __shfl_sync(0xffffffffu, sn, 1);
      const int pr = lane >> 2, x = lane & 3;
      const int p = pair_lo(r, pr & 1), q = pair_hi(r, pr & 1);
      const bool act = lane < 8 && q < P && x < P;
      const double cc = pr ? c1 : c0, ss = pr ? s1 : s0;
      if (act) {  // columns p, q
        const double hp = H[x * P + p], hq = H[x * P + q];
        H[x * P + p] = cc * hp - ss * hq;
        H[x * P + q] = ss * hp + cc * hq;
      }
      __syncwarp();
      if (act) {  // rows p, q
        const double hp = H[p * P + x], hq = H[q * P + x];
        H[p * P + x] = cc * hp - ss * hq;
        H[q * P + x] = ss * hp + cc * hq;
      }
      if (act) {  // eigenvector columns p, q
        const double qp = Q[x * P + p], qq = Q[x * P + q];
        Q[x * P + p] = cc * qp - ss * qq;
        Q[x * P + q] = ss * qp + cc * qq;
      }
      __syncwarp();
    }
  }
  // selection sort, descending eigenvalues
  if (lane == 0)
    for (int i = 0; i < P; ++i) {
      int m = i;
      for (int j = i + 1; j < P; ++j)
        if (H[j * P + j] > H[m * P + m]) m = j;
      if (m != i) {
        const double t = H[i * P + i];
        H[i * P + i] = H[m * P + m];
        H[m * P + m] = t;
        for (int r = 0; r < P; ++r) {
          const double u = Q[r * P + i];
          Q[r * P + i] = Q[r * P + m];
          Q[r * P + m] = u;
        }
      }
    }
  __syncwarp();
}

// orthonormalise the P columns of V (k x P, row-major in shared memory) by
// Gram-Schmidt applied twice per column; a column that vanishes is replaced
// by a fixed pseudo-random vector.  (Cholesky-QR in two passes costs fewer
// block sums but leaves the basis less aligned with the previous Ritz
// vectors, and the Rayleigh-Ritz step after it then needs more Jacobi sweeps.)
// The column's norm before the projections rides with the first pass's
// dot products in one block sum; 1/||v|| is formed once, by thread 0.
__device__ void orthonormalise(int k, int P, double *V, double *scratch, unsigned long long salt) {
  __shared__ double s_inv;
  for (int j = 0; j < P; ++j) {
    for (int attempt = 0; attempt < 3; ++attempt) {
      double nrm0 = 0.0, nrm[1] = {0.0};
      if (j == 0) {
        for (int r = threadIdx.x; r < k; r += blockDim.x) nrm[0] += V[r * P + j] * V[r * P + j];
        block_sum<1>(nrm, scratch);
        nrm0 = nrm[0];
      } else {
        for (int pass = 0; pass < 2; ++pass) {
          double dots[kEigP + 1];  // dots[q] = v_q . v_j (q < j); dots[kEigP] = ||v_j||^2 before the projections
#pragma unroll
          for (int q = 0; q <= kEigP; ++q) dots[q] = 0.0;
          for (int r = threadIdx.x; r < k; r += blockDim.x) {
            const double vj = V[r * P + j];
#pragma unroll
            for (int q = 0; q < kEigP; ++q)
              if (q < j) dots[q] += V[r * P + q] * vj;
            if (pass == 0) dots[kEigP] += vj * vj;
          }
          if (pass == 0) {
            block_sum<kEigP + 1>(dots, scratch);
            nrm0 = dots[kEigP];
          } else {
            double d4[kEigP];
#pragma unroll
            for (int q = 0; q < kEigP; ++q) d4[q] = dots[q];
            block_sum<kEigP>(d4, scratch);
#pragma unroll
            for (int q = 0; q < kEigP; ++q) dots[q] = d4[q];
          }
          for (int r = threadIdx.x; r < k; r += blockDim.x)
#pragma unroll
            for (int q = 0; q < kEigP; ++q)
              if (q < j) V[r * P + j] -= dots[q] * V[r * P + q];
          __syncthreads();
        }
        for (int r = threadIdx.x; r < k; r += blockDim.x) nrm[0] += V[r * P + j] * V[r * P + j];
        block_sum<1>(nrm, scratch);
      }
      if (nrm[0] > 1e-24 * nrm0 && nrm[0] > 0.0) {
        if (threadIdx.x == 0) s_inv = 1.0 / sqrt(nrm[0]);
        __syncthreads();
        const double inv = s_inv;
        for (int r = threadIdx.x; r < k; r += blockDim.x) V[r * P + j] *= inv;
        __syncthreads();
        break;
      }
      for (int r = threadIdx.x; r < k; r += blockDim.x)
        V[r * P + j] = (double)(int64_t)(splitmix64_at(salt + 1000003ull * j + 7919ull * attempt, r) >> 11) *
                           (1.0 / 4503599627370496.0) - 1.0;
      __syncthreads();
    }
  }
}

struct EigOut {
  double lam[2];
  double sigma[2];  // sum_a v_a
  double kappa[2];  // sum_a cbar_a v_a - gbar * sigma
  int32_t iters;
  int32_t converged;
};

// top-2 eigenpairs of B (k x k, FP64).  Subspace iteration of dimension P
// runs on M (the 2^kEigPowerLog2-th power of B / max|B|, same eigenvectors,
// ratios of eigenvalues raised to that power, so the subspace converges that
// times faster per iteration) with a Rayleigh-Ritz step every iteration;
// a final Rayleigh-Ritz step with B itself gives the eigenvalues and the
// reported residual.
// The k x k products (A V, one warp per row) are spread over the blocks of a
// cooperative grid: each block writes its rows into Yg (two alternating
// buffers), and after a grid barrier every block copies the whole product
// into its shared memory.  Everything else -- Rayleigh-Ritz, residuals,
// Gram-Schmidt, the convergence decisions -- every block computes on its own
// identical copy, so the blocks stay in step without further exchange; block
// 0 writes the results.
// S: the type of the column sums s_a (exact integers for hop distances,
// FP64 for weighted distances)
template <class S>
__global__ void __launch_bounds__(kEigThreads) k_eigen(int32_t n, int32_t k, const double *__restrict__ B,
                                                       const double *__restrict__ M,
                                                       const S *__restrict__ s,
                                                       double *__restrict__ vout /* [2][k] */,
                                                       EigOut *__restrict__ out, double *__restrict__ eig_user,
                                                       double *__restrict__ Yg /* [2][k][P] */,
                                                       BarrierState *__restrict__ bar,
                                                       int32_t *__restrict__ status, int maxit, double tol) {
  extern __shared__ __align__(16) double sm[];
  const int P = min(kEigP, k);
  double *V = sm;                       // k x P
  double *Y = V + (size_t)k * P;        // k x P
  double *scratch = Y + (size_t)k * P;  // kEigScratch doubles
  __shared__ double H[kEigP * kEigP], Q[kEigP * kEigP];
  __shared__ int s_done;

  for (int t = threadIdx.x; t < k * P; t += blockDim.x)
    V[t] = (double)(splitmix64_at(0x5eed5eedull, (unsigned long long)t) >> 11) * (1.0 / 4503599627370496.0) - 1.0;
  __syncthreads();
  orthonormalise(k, P, V, scratch, 0x1234ull);
  if (threadIdx.x == 0) s_done = 0;
  __syncthreads();

  // Y[:, 0..ncols) = A V[:, 0..ncols) over the grid (see above); false if a
  // grid barrier gave up (status is set, every block stops)
  int nprod = 0;
  auto product = [&](const double *__restrict__ A, int ncols) -> bool {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    double *yg = Yg + (size_t)(nprod & 1) * k * P;
    ++nprod;
    for (int r = blockIdx.x * nwarp + warp; r < k; r += gridDim.x * nwarp) {
      double acc[kEigP];
#pragma unroll
      for (int q = 0; q < kEigP; ++q) acc[q] = 0.0;
      const double *arow = A + (size_t)r * k;
      for (int c = lane; c < k; c += 32) {
        const double av = __ldg(arow + c);
#pragma unroll
        for (int q = 0; q < kEigP; ++q)
          if (q < ncols) acc[q] += av * V[c * P + q];
      }
      // lane l holds the total of column l >> kSh
      constexpr int kSh = 5 - Halving<kEigP>::LOG;
      const double tot = warp_sum_halving<kEigP>(acc);
      const int q = lane >> kSh;
      if ((lane & ((1 << kSh) - 1)) == 0 && q < ncols) yg[r * P + q] = tot;
    }
    if (gridDim.x > 1) {
      if (!grid_barrier(bar, status)) return false;
    } else {
      __syncthreads();
    }
    for (int t = threadIdx.x; t < k * P; t += blockDim.x)
      if ((t % P) < ncols) Y[t] = __ldcg(yg + t);
    __syncthreads();
    return true;
  };

  // one Rayleigh-Ritz step with matrix A on span(V): V <- Ritz vectors,
  // Y <- A V, H diagonal <- Ritz values (descending); returns the relative
  // residual max_{j<2} ||A v_j - h_j v_j|| / |h_0| in thread 0 (0 in the
  // others), or -1 in every thread if a grid barrier gave up
  auto rayleigh_ritz = [&](const double *__restrict__ A) -> double {
    if (!product(A, P)) return -1.0;
    double h[kEigP * (kEigP + 1) / 2];  // H = V^T Y, upper triangle
#pragma unroll
    for (int q = 0; q < kEigP * (kEigP + 1) / 2; ++q) h[q] = 0.0;
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
      int q = 0;
#pragma unroll
      for (int i = 0; i < kEigP; ++i)
#pragma unroll
        for (int j = i; j < kEigP; ++j, ++q)
          if (j < P) h[q] += V[r * P + i] * Y[r * P + j];
    }
    block_sum<kEigP * (kEigP + 1) / 2>(h, scratch);
    if (threadIdx.x == 0) {
      int q = 0;
      for (int i = 0; i < kEigP; ++i)
        for (int j = i; j < kEigP; ++j, ++q)
          if (j < P) {
            H[i * P + j] = h[q];
            H[j * P + i] = h[q];
          }
    }
    if (threadIdx.x < 32) {
      __syncwarp();
      tiny_jacobi_warp(P, H, Q);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < k; r += blockDim.x) {  // W = V Q, A W = Y Q
      double wv[kEigP], yv[kEigP];
#pragma unroll
      for (int j = 0; j < kEigP; ++j) {
        wv[j] = 0.0;
        yv[j] = 0.0;
        if (j < P)
          for (int l = 0; l < P; ++l) {
            wv[j] += V[r * P + l] * Q[l * P + j];
            yv[j] += Y[r * P + l] * Q[l * P + j];
          }
      }
#pragma unroll
      for (int j = 0; j < kEigP; ++j)
        if (j < P) {
          V[r * P + j] = wv[j];
          Y[r * P + j] = yv[j];
        }
    }
    __syncthreads();
    double res[2] = {0.0, 0.0};
    for (int r = threadIdx.x; r < k; r += blockDim.x)
      for (int j = 0; j < 2 && j < P; ++j) {
        const double e = Y[r * P + j] - H[j * P + j] * V[r * P + j];
        res[j] += e * e;
      }
    block_sum<2>(res, scratch);
    if (threadIdx.x != 0) return 0.0;  // only thread 0 reads the residual
    const double h0 = fabs(H[0]);
    return h0 > 0.0 ? sqrt(fmax(res[0], res[1])) / h0 : 0.0;
  };

  // convergence test on B itself: max_{j<2} ||B v_j - q_j v_j|| / |q_0| with
  // the Rayleigh quotients q_j = v_j^T B v_j (the powers of B in M shrink the
  // second pair's share, so a test on M alone would stop early for it)
  auto residual_b = [&]() -> double {
    if (!product(B, min(2, P))) return -1.0;  // Y[:, 0..1] = B V[:, 0..1]
    double q[2] = {0.0, 0.0};
    for (int r = threadIdx.x; r < k; r += blockDim.x)
      for (int j = 0; j < 2 && j < P; ++j) q[j] += V[r * P + j] * Y[r * P + j];
    block_sum<2>(q, scratch);
    double e[2] = {0.0, 0.0};
    for (int r = threadIdx.x; r < k; r += blockDim.x)
      for (int j = 0; j < 2 && j < P; ++j) {
        const double d = Y[r * P + j] - q[j] * V[r * P + j];
        e[j] += d * d;
      }
    block_sum<2>(e, scratch);
    if (threadIdx.x != 0) return 0.0;  // only thread 0 reads the residual
    const double q0 = fabs(q[0]);
    return q0 > 0.0 ? sqrt(fmax(e[0], e[1])) / q0 : 0.0;
  };

  __shared__ int s_stuck;
  double best = 1e300;
  int since_best = 0;
  int it = 0;
  for (; it < maxit; ++it) {
    if (rayleigh_ritz(M) < 0.0) return;
    // Y = M W is kept for the next basis; the test on B uses the V columns only
    for (int t = threadIdx.x; t < k * P; t += blockDim.x) sm[2 * (size_t)k * P + kEigScratch + t] = Y[t];
    __syncthreads();
    const double r = residual_b();
    if (r < 0.0) return;
    for (int t = threadIdx.x; t < k * P; t += blockDim.x) Y[t] = sm[2 * (size_t)k * P + kEigScratch + t];
    __syncthreads();
    if (threadIdx.x == 0) {
      s_done = r <= tol ? 1 : 0;
      // when lambda_2 / lambda_1 is small the second pair sinks below FP64
      // precision in the powers of B and the residual stalls: go on with B
      if (r < 0.9 * best) {
        best = r;
        since_best = 0;
      } else {
        ++since_best;
      }
      s_stuck = since_best >= 50 ? 1 : 0;
    }
    __syncthreads();
    if (s_done || s_stuck) break;
    for (int t = threadIdx.x; t < k * P; t += blockDim.x) V[t] = Y[t];  // next basis: orthonormalised M W
    __syncthreads();
    orthonormalise(k, P, V, scratch, 0x9e37ull + (unsigned long long)it);
  }
  // subspace iteration on B itself (rate lambda_{P+1} / lambda_2 for the
  // second vector, no powers to drown it) until the same test passes
  if (!s_done) {
    for (++it; it < maxit; ++it) {
      const double r = rayleigh_ritz(B);  // V <- Ritz vectors of B, Y <- B V
      if (r < 0.0) return;
      if (threadIdx.x == 0) s_done = r <= tol ? 1 : 0;
      __syncthreads();
      if (s_done) break;
      for (int t = threadIdx.x; t < k * P; t += blockDim.x) V[t] = Y[t];
      __syncthreads();
      orthonormalise(k, P, V, scratch, 0x7f4aull + (unsigned long long)it);
    }
  }
  const double last_res = rayleigh_ritz(B);
  if (last_res < 0.0 || blockIdx.x != 0) return;  // block 0 writes the results
  // top-2 Ritz vectors are columns 0, 1 of V; sign: largest |entry| positive
  __shared__ int s_big[2];
  if (threadIdx.x < 2) {
    const int j = threadIdx.x;
    int big = 0;
    for (int r = 1; r < k; ++r)
      if (fabs(V[r * P + j]) > fabs(V[big * P + j])) big = r;
    s_big[j] = big;
  }
  __syncthreads();
  const double sg0 = V[s_big[0] * P + 0] < 0 ? -1.0 : 1.0;
  const double sg1 = V[s_big[1] * P + 1] < 0 ? -1.0 : 1.0;
  double sums[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const double inv_n = 1.0 / (double)n;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    const double v0 = sg0 * V[r * P + 0], v1 = sg1 * V[r * P + 1];
    vout[r] = v0;
    vout[k + r] = v1;
    const double cbar = (double)s[r] * inv_n;
    sums[0] += v0;
    sums[1] += v1;
    sums[2] += cbar * v0;
    sums[3] += cbar * v1;
    sums[4] += cbar;
  }
  block_sum<5>(sums, scratch);
  if (threadIdx.x == 0) {
    const double gbar = sums[4] / (double)k;
    out->lam[0] = H[0];
    out->lam[1] = P > 1 ? H[1 * P + 1] : 0.0;
    out->sigma[0] = sums[0];
    out->sigma[1] = sums[1];
    out->kappa[0] = sums[2] - gbar * sums[0];
    out->kappa[1] = sums[3] - gbar * sums[1];
    out->iters = it;
    out->converged = s_done;
    if (eig_user) {
      eig_user[0] = out->lam[0];
      eig_user[1] = out->lam[1];
      eig_user[2] = (double)it;
      eig_user[3] = last_res;
    }
    if (!s_done || !(H[0] > 0.0)) dev_fail(status, SSM_E_NUMERIC);
  }
}

// ------------------------------------------------------------- projection
// two-float accumulation for the (x, y) pair at once, in packed FP32x2
// arithmetic with every operation rounded on its own (no contraction):
// (hi, lo) += a * (bh + bl), a exact in FP32; p + pe = a bh exactly, s + e =
// hi + p exactly
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void ff_madd2(float2 &hi, float2 &lo, float a, float2 bh, float2 bl) {
  const float2 a2 = make_float2(a, a);
  const float2 p = __fmul2_rn(a2, bh);
  const float2 pe = __ffma2_rn(a2, bh, neg2(p));
  const float2 s = __fadd2_rn(hi, p);
  const float2 bp = __fadd2_rn(s, neg2(hi));
  const float2 e = __fadd2_rn(__fadd2_rn(hi, neg2(__fadd2_rn(s, neg2(bp)))), __fadd2_rn(p, neg2(bp)));
  lo = __fadd2_rn(lo, __fadd2_rn(e, __ffma2_rn(a2, bl, pe)));
  hi = s;
}

// BIG (read on the device): some d_ia^2 is not exact in FP32 (d > 4095), so
// it is split into two exact parts
__global__ void __launch_bounds__(256) k_project(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                                                 const double *__restrict__ vv, const EigOut *__restrict__ eo,
                                                 const unsigned *__restrict__ dmax, void *__restrict__ pos,
                                                 int precision) {
  extern __shared__ __align__(16) float4 sv[];  // per pivot: (v0 hi, v1 hi), (v0 lo, v1 lo)
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    const double v0 = vv[a], v1 = vv[k + a];
    const float h0 = (float)v0, h1 = (float)v1;
    sv[a] = make_float4(h0, h1, (float)(v0 - (double)h0), (float)(v1 - (double)h1));
  }
  __syncthreads();
  const double sig0 = eo->sigma[0], sig1 = eo->sigma[1], kap0 = eo->kappa[0], kap1 = eo->kappa[1];
  const bool BIG = (unsigned long long)(*dmax) * (*dmax) >= (1ull << 24);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 hi = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);  // (x, y) two-float sums
    unsigned long long rs = 0;
    const uint16_t *col = dip + i;
    // eight pivots' distances in flight per thread, then added in pivot order
    for (int a0 = 0; a0 < k; a0 += 8) {
      unsigned dq[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) dq[q] = a0 + q < k ? (unsigned)__ldg(col + (size_t)(a0 + q) * n) : 0u;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (a0 + q >= k) break;
        const unsigned dd = dq[q] * dq[q];
        rs += dd;
        const float4 v = sv[a0 + q];
        const float2 vh = make_float2(v.x, v.y), vl = make_float2(v.z, v.w);
        if (!BIG) {
          ff_madd2(hi, lo, (float)dd, vh, vl);  // dd exact below 2^24
        } else {
          ff_madd2(hi, lo, (float)(dd & 0xFFFFF000u), vh, vl);  // both parts exact
          ff_madd2(hi, lo, (float)(dd & 0xFFFu), vh, vl);
        }
      }
    }
    const double rbar = (double)rs / (double)k;
    const double x = -0.5 * (((double)hi.x + (double)lo.x) - rbar * sig0 - kap0);
    const double y = -0.5 * (((double)hi.y + (double)lo.y) - rbar * sig1 - kap1);
    if (precision == 64) reinterpret_cast<double2 *>(pos)[i] = make_double2(x, y);
    else reinterpret_cast<float2 *>(pos)[i] = make_float2((float)x, (float)y);
  }
}

// the largest entry: 16-byte loads of eight entries from the first 16-byte
// boundary on (packed 16-bit maxima), the entries before it and past the
// last whole load one at a time
__global__ void k_dmax(int64_t count, const uint16_t *__restrict__ dip, unsigned *__restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t head = min(count, (int64_t)((16u - ((uintptr_t)dip & 15u)) & 15u) / 2);  // dip is 2-byte aligned
  const int64_t nvec = (count - head) / 8;
  const uint4 *v = reinterpret_cast<const uint4 *>(dip + head);
  unsigned m2 = 0;  // two packed 16-bit maxima
  for (int64_t t = gt; t < nvec; t += stride) {
    const uint4 w = __ldg(v + t);
    m2 = __vmaxu2(m2, __vmaxu2(__vmaxu2(w.x, w.y), __vmaxu2(w.z, w.w)));
  }
  unsigned m = max(m2 & 0xFFFFu, m2 >> 16);
  for (int64_t t = gt; t < head; t += stride) m = max(m, (unsigned)__ldg(dip + t));
  for (int64_t t = head + 8 * nvec + gt; t < count; t += stride) m = max(m, (unsigned)__ldg(dip + t));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ------------------------------------------------------------- rescale
// Sum over the edges of ||x_i - x_j|| (each undirected edge once, from its
// lower end i < j), in three steps with a fixed order of summation:
//   k_edge_sum_rows  the sum of every row of at most kEdgeShort entries into
//                    rowsum[i] (a lane per node, eight entries in flight);
//                    longer rows are listed and get rowsum[i] from
//   k_edge_sum_long  a warp per listed row (eight entries per lane in flight,
//                    lanes then a fixed tree) -- hub rows of heavy-tailed
//                    graphs are spread over the grid instead of queuing in
//                    the warp that owns their node;
//   k_edge_sum_total the rows in node order: a fixed share per thread, fixed
//                    trees, the last block forms the scale.
// Weighted graphs (elen) also sum the target lengths l_ij the same way.
constexpr int kEdgeShort = 32;

template <class T2>
__device__ __forceinline__ double edge_len(T2 a, T2 b) {
  using R = decltype(a.x);  // lengths in the precision of the positions, summed in FP64
  const R dx = a.x - b.x, dy = a.y - b.y;
  return (double)sqrt(dx * dx + dy * dy);
}

template <class T2>
__global__ void __launch_bounds__(256) k_edge_sum_rows(int32_t n, const int32_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colidx, const T2 *__restrict__ pos,
                                                       const float *__restrict__ elen, double *__restrict__ rowsum,
                                                       double *__restrict__ rowlen, int32_t *__restrict__ longrows,
                                                       unsigned *__restrict__ nlong) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = __ldg(rowptr + i), e = __ldg(rowptr + i + 1);
    if (e - b > kEdgeShort) {
      longrows[atomicAdd(nlong, 1u)] = (int32_t)i;  // the list's order does not matter: rowsum is by node
      continue;
    }
    const T2 xi = pos[i];
    double acc = 0.0, accl = 0.0;
    for (int t = b; t < e; t += 8) {
      int j[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) j[q] = t + q < e ? __ldg(colidx + t + q) : -1;
      T2 xj[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) xj[q] = j[q] > i ? pos[j[q]] : xi;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (j[q] > i) {
          acc += edge_len(xi, xj[q]);
          if (elen) accl += (double)__ldg(elen + t + q);
        }
    }
    rowsum[i] = acc;
    if (elen) rowlen[i] = accl;
  }
}

template <class T2>
__global__ void __launch_bounds__(256) k_edge_sum_long(const int32_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colidx, const T2 *__restrict__ pos,
                                                       const float *__restrict__ elen,
                                                       const int32_t *__restrict__ longrows,
                                                       const unsigned *__restrict__ nlong, double *__restrict__ rowsum,
                                                       double *__restrict__ rowlen) {
  const int lane = threadIdx.x & 31;
  const unsigned cnt = __ldcg(nlong);
  const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
  for (unsigned r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < cnt; r += nwarps) {
    const int i = __ldg(longrows + r);
    const int hb = __ldg(rowptr + i), he = __ldg(rowptr + i + 1);
    const T2 xi = pos[i];
    double acc = 0.0, accl = 0.0;
    for (int t0 = hb + lane; t0 < he; t0 += 32 * 8) {
      int j[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) j[q] = t0 + 32 * q < he ? __ldg(colidx + t0 + 32 * q) : -1;
      T2 xj[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) xj[q] = j[q] > i ? pos[j[q]] : xi;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (j[q] > i) {
          acc += edge_len(xi, xj[q]);
          if (elen) accl += (double)__ldg(elen + t0 + 32 * q);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_xor_sync(0xffffffffu, acc, o);
      accl += __shfl_xor_sync(0xffffffffu, accl, o);
    }
    if (lane == 0) {
      rowsum[i] = acc;
      if (elen) rowlen[i] = accl;
    }
  }
}

__global__ void __launch_bounds__(256) k_edge_sum_total(int32_t n, const int32_t *__restrict__ rowptr,
                                                        const double *__restrict__ rowsum,
                                                        const double *__restrict__ rowlen, double *__restrict__ part,
                                                        unsigned *__restrict__ done, double *__restrict__ scale,
                                                        int32_t *__restrict__ status) {
  __shared__ double red[8], redl[8];
  __shared__ unsigned s_ticket;
  double acc = 0.0, accl = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    acc += __ldcg(rowsum + i);
    if (rowlen) accl += __ldcg(rowlen + i);
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    accl += __shfl_xor_sync(0xffffffffu, accl, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = acc;
    redl[threadIdx.x >> 5] = accl;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, tl = 0.0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) {
      t += red[w];
      tl += redl[w];
    }
    part[2 * blockIdx.x] = t;
    part[2 * blockIdx.x + 1] = tl;
    __threadfence();
    s_ticket = atomicAdd(done, 1u);
  }
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  // the last block adds the block sums: a fixed share per thread, then a fixed tree
  __threadfence();
  double t = 0.0, tl = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    t += __ldcg(part + 2 * b);
    tl += __ldcg(part + 2 * b + 1);
  }
  for (int o = 16; o > 0; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o);
    tl += __shfl_xor_sync(0xffffffffu, tl, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = t;
    redl[threadIdx.x >> 5] = tl;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double tot = 0.0, totl = 0.0;
  for (int w = 0; w < (int)blockDim.x / 32; ++w) {
    tot += red[w];
    totl += redl[w];
  }
  const double m = rowlen ? totl : (double)__ldg(rowptr + n) * 0.5;
  if (!(tot > 0.0) || !isfinite(tot)) {
    dev_fail(status, SSM_E_NUMERIC);
    *scale = 1.0;
  } else {
    *scale = m / tot;
  }
}

template <class T2>
__global__ void k_rescale(int32_t n, T2 *__restrict__ pos, const double *__restrict__ scale) {
  const double sc = *scale;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T2 x = pos[i];
    x.x = (decltype(x.x))((double)x.x * sc);
    x.y = (decltype(x.y))((double)x.y * sc);
    pos[i] = x;
  }
}

struct MdsWs {
  unsigned long long *Glo, *Ghi, *s;
  double *B, *B2, *Btmp, *M, *bscale, *rowmean, *vv, *part, *scale;
  EigOut *eo;
  unsigned *done, *dmax;
  double *Yg;
  BarrierState *bar;
  double *rowsum, *rowlen;  // [n] per-row edge-length sums (rescale)
  int32_t *longrows;        // [n] rows above kEdgeShort entries
  unsigned *nlong;
};

static size_t carve_mds(Carver &c, MdsWs &w, int32_t n, int32_t k) {
  const size_t kk = (size_t)k * k;
  w.Glo = c.take<unsigned long long>(kk);
  w.Ghi = c.take<unsigned long long>(kk);
  w.s = c.take<unsigned long long>(k);
  w.B = c.take<double>(kk);
  w.B2 = c.take<double>(kk);
  w.Btmp = c.take<double>(kk);
  w.M = c.take<double>(kk);
  w.bscale = c.take<double>(1);
  w.rowmean = c.take<double>((size_t)k + 1);  // the row means and their mean
  w.vv = c.take<double>(2 * (size_t)k);
  w.part = c.take<double>(8192);
  w.scale = c.take<double>(1);
  w.eo = c.take<EigOut>(1);
  w.done = c.take<unsigned>(1);
  w.dmax = c.take<unsigned>(1);
  w.Yg = c.take<double>(2 * (size_t)k * kEigP);
  w.bar = c.take<BarrierState>(1);
  w.rowsum = c.take<double>((size_t)n);
  w.rowlen = c.take<double>((size_t)n);
  w.longrows = c.take<int32_t>((size_t)n);
  w.nlong = c.take<unsigned>(1);
  return c.size();
}

// top-2 eigenpairs of w.B (already formed) and the projection constants
// (from the column sums s_a of Delta) into w.vv / w.eo
template <class S>
static int launch_eigen(int32_t n, int32_t k, MdsWs &w, const S *colsum, double *eig, int32_t *status,
                        cudaStream_t s) {
  const size_t kk = (size_t)k * k;
  const int P = std::min(kEigP, (int)k);
  const size_t esm = (3 * (size_t)k * P + kEigScratch) * sizeof(double);  // V, Y, saved Y, scratch
  SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_eigen<S>));
  note_launch(), k_absmax_inv<<<1, 1024, 0, s>>>((int64_t)kk, w.B, w.bscale);
  const dim3 sq_grid((unsigned)((k + 15) / 16), (unsigned)((k + 15) / 16));
  // M = (B/max|B|)^(2^kEigPowerLog2) by repeated squaring
  {
    const double *src = w.B;
    for (int q = 0; q < kEigPowerLog2; ++q) {
      double *dst = (q == kEigPowerLog2 - 1) ? w.M : ((q & 1) ? w.Btmp : w.B2);
      note_launch(), k_square_f64<<<sq_grid, 256, 0, s>>>(k, src, q == 0 ? w.bscale : nullptr, dst);
      src = dst;
    }
  }
  // one warp per row of the k x k products: as many blocks as the rows need, all resident
  const int want = (k + kEigThreads / 32 - 1) / (kEigThreads / 32);
  const int eblocks = std::max(1, std::min(want, cooperative_blocks((const void *)k_eigen<S>, kEigThreads, esm, 1)));
  if (int rc_ = reset_barrier(w.bar, s)) return rc_;
  int maxit = 2000;
  double tol = 1e-12;
  void *args[] = {&n, &k, &w.B, &w.M, &colsum, &w.vv, &w.eo, &eig, &w.Yg, &w.bar, &status, &maxit, &tol};
  note_launch();
  SSM_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)k_eigen<S>, dim3(eblocks), dim3(kEigThreads), args, esm, s));
  return SSM_OK;
}

// Algorithm 1 line 4: scale so that sum_E ||x_i - x_j|| = sum_E l_ij (m for
// unit edges, elen == nullptr); w.done must be zero
static int launch_rescale(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, void *pos,
                          int32_t precision, MdsWs &w, int32_t *status, cudaStream_t s) {
  const int pb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)num_sms() * 8);
  const int eb = std::min(pb, 4096);  // part holds 2 per block
  double *rowlen = elen ? w.rowlen : nullptr;
  SSM_TRY_CUDA(cudaMemsetAsync(w.nlong, 0, sizeof(unsigned), s));
  if (precision == 64) {
    note_launch(), k_edge_sum_rows<double2><<<pb, 256, 0, s>>>(n, rowptr, colidx, (const double2 *)pos, elen,
                                                               w.rowsum, rowlen, w.longrows, w.nlong);
    note_launch(), k_edge_sum_long<double2><<<pb, 256, 0, s>>>(rowptr, colidx, (const double2 *)pos, elen, w.longrows,
                                                               w.nlong, w.rowsum, rowlen);
  } else {
    note_launch(), k_edge_sum_rows<float2><<<pb, 256, 0, s>>>(n, rowptr, colidx, (const float2 *)pos, elen,
                                                              w.rowsum, rowlen, w.longrows, w.nlong);
    note_launch(), k_edge_sum_long<float2><<<pb, 256, 0, s>>>(rowptr, colidx, (const float2 *)pos, elen, w.longrows,
                                                              w.nlong, w.rowsum, rowlen);
  }
  note_launch(), k_edge_sum_total<<<eb, 256, 0, s>>>(n, rowptr, w.rowsum, rowlen, w.part, w.done, w.scale, status);
  if (precision == 64)
    note_launch(), k_rescale<double2><<<pb, 256, 0, s>>>(n, (double2 *)pos, w.scale);
  else
    note_launch(), k_rescale<float2><<<pb, 256, 0, s>>>(n, (float2 *)pos, w.scale);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

// G = Delta^T Delta into Glo/Ghi (zeroed here) and the largest d_ip entry into *dmax
static int launch_gram(int32_t n, int32_t k, const uint16_t *dip, unsigned *dmax, unsigned long long *Glo,
                       unsigned long long *Ghi, int32_t *status, cudaStream_t s) {
  const size_t kk = (size_t)k * k;
  SSM_TRY_CUDA(cudaMemsetAsync(Glo, 0, kk * sizeof(unsigned long long), s));
  SSM_TRY_CUDA(cudaMemsetAsync(Ghi, 0, kk * sizeof(unsigned long long), s));
  SSM_TRY_CUDA(cudaMemsetAsync(dmax, 0, sizeof(unsigned), s));
  // the largest distance decides how many digits the tensor-core Gram needs
  const int64_t cnt = (int64_t)k * n;
  note_launch(), k_dmax<<<std::min<int64_t>((cnt + 255) / 256, (int64_t)num_sms() * 8), 256, 0, s>>>(cnt, dip, dmax);
  SSM_TRY_CUDA(cudaGetLastError());
  return launch_gram_tc(n, k, dip, dmax, Glo, Ghi, status, s);
}

}  // namespace ssm

SSM_API size_t ssm_gram_workspace(int32_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  return 256;
}

SSM_API int ssm_gram(int32_t n, int32_t k, const uint16_t *dip, uint64_t *g_lo, uint64_t *g_hi, int32_t *status,
                     void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !dip || !g_lo || !g_hi || !status || !ws) return fail(SSM_E_ARG, "ssm_gram: null pointer or n < 1");
  if (k < 1 || k > kMaxPivotsMds) return fail(SSM_E_ARG, "ssm_gram: need 1 <= k <= %d", kMaxPivotsMds);
  if (ws_bytes < ssm_gram_workspace(n, k)) return fail(SSM_E_NOMEM, "ssm_gram: workspace %zu bytes, need 256", ws_bytes);
  return launch_gram(n, k, dip, static_cast<unsigned *>(ws), reinterpret_cast<unsigned long long *>(g_lo),
                     reinterpret_cast<unsigned long long *>(g_hi), status, s);
}

SSM_API size_t ssm_pivotmds_workspace(int32_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::MdsWs w;
  return ssm::carve_mds(c, w, n, k);
}

SSM_API int ssm_pivotmds(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k, const uint16_t *dip,
                         void *pos, int32_t precision, int32_t rescale, double *eig, int32_t *status, void *ws,
                         size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !dip || !pos || !status || !ws || (rescale && (!rowptr || !colidx)))
    return fail(SSM_E_ARG, "ssm_pivotmds: null pointer or n < 1");
  if (k < 2 || k > kMaxPivotsMds || k > n) return fail(SSM_E_ARG, "ssm_pivotmds: need 2 <= k <= min(n, %d)", kMaxPivotsMds);
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_pivotmds: precision must be 32 or 64");
  Carver c(ws, ws_bytes);
  MdsWs w;
  carve_mds(c, w, n, k);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_pivotmds: workspace %zu bytes, need %zu", ws_bytes, c.size());
  const int sms = num_sms();
  SSM_TRY_CUDA(cudaMemsetAsync(w.done, 0, sizeof(unsigned), s));
  {
    const int rc = launch_gram(n, k, dip, w.dmax, w.Glo, w.Ghi, status, s);
    if (rc) return rc;
  }
  SSM_TRY_CUDA(cudaMemsetAsync(w.s, 0, (size_t)k * sizeof(unsigned long long), s));
  {
    const int64_t tasks = (int64_t)k * ((n + kColChunk - 1) / kColChunk);
    note_launch(), k_colsum<<<(unsigned)std::min<int64_t>(tasks, (int64_t)sms * 8), 256, 0, s>>>(n, k, dip, w.s);
  }
  {
    const int64_t kk = (int64_t)k * k;
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((kk + 255) / 256, sms * 4));
    note_launch(), k_prepare_b<<<gb, 256, 0, s>>>(n, k, w.Glo, w.Ghi, w.s, w.B);
    note_launch(), k_row_means<<<1, 1024, 0, s>>>(k, w.B, w.rowmean);
    note_launch(), k_center<<<gb, 256, 0, s>>>(k, w.B, w.rowmean);
  }
  if (int rc = launch_eigen(n, k, w, w.s, eig, status, s)) return rc;
  const int pb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)sms * 8);
  const size_t psm = (size_t)k * sizeof(float4);
  note_launch(), k_project<<<pb, 256, psm, s>>>(n, k, dip, w.vv, w.eo, w.dmax, pos, precision);
  if (rescale) return launch_rescale(n, rowptr, colidx, nullptr, pos, precision, w, status, s);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}


// ------------------------------------------------------------- weighted
// PivotMDS on a float32 distance table (weighted graphs).  delta_ia = d_ia^2
// is formed in FP64 (exactly); with cbar_a the column means,
//   C^T C = 1/4 J_k G' J_k,  G'_ab = sum_i (delta_ia - cbar_a)(delta_ib - cbar_b),
// the column centring applied before the product so that nothing cancels;
// G' is summed in FP64 per fixed node chunk and the chunk partials are added
// in chunk order.
namespace ssm {

constexpr int kWTile = 32;

static int64_t wgram_chunk(int32_t n) {
  int64_t c = ((int64_t)n + 63) / 64;
  c = std::max<int64_t>(1024, std::min<int64_t>(16384, c));
  return (c + kWTile - 1) / kWTile * kWTile;
}

// partc[a * nchunks + c] = sum over the nodes of chunk c of d_ia^2 (fixed tree)
__global__ void __launch_bounds__(256) k_wcolsum_part(int32_t n, int32_t k, const float *__restrict__ dist,
                                                      int64_t chunk, int64_t nchunks, double *__restrict__ partc) {
  __shared__ double red[8];
  for (int64_t task = blockIdx.x; task < (int64_t)k * nchunks; task += gridDim.x) {
    const int a = (int)(task / nchunks);
    const int64_t c = task - (int64_t)a * nchunks;
    const int64_t i0 = c * chunk, i1 = min((int64_t)n, i0 + chunk);
    double acc = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double d = (double)__ldg(dist + (size_t)a * n + i);
      acc += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      partc[task] = t;
    }
    __syncthreads();
  }
}

__global__ void k_wcolsum_final(int32_t k, int64_t nchunks, const double *__restrict__ partc,
                                double *__restrict__ colsum) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int64_t c = 0; c < nchunks; ++c) t += partc[(size_t)a * nchunks + c];
    colsum[a] = t;
  }
}

// one 32 x 32 tile (ta <= tb) of G' over one node chunk; 16 x 16 threads,
// 2 x 2 outputs each; partials into partg[c][a][b]
__global__ void __launch_bounds__(256) k_wgram(int32_t n, int32_t k, const float *__restrict__ dist,
                                               const double *__restrict__ colsum, int64_t chunk, int64_t nchunks,
                                               int32_t ntiles, double *__restrict__ partg) {
  __shared__ double sa[kWTile][kWTile + 1], sb[kWTile][kWTile + 1];  // [node][pivot]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t npairs = (int64_t)ntiles * (ntiles + 1) / 2;
  const double inv_n = 1.0 / (double)n;
  for (int64_t task = blockIdx.x; task < npairs * nchunks; task += gridDim.x) {
    const int64_t c = task / npairs;
    int64_t pr = task - c * npairs;
    int ta = 0;
    while (pr >= ntiles - ta) {
      pr -= ntiles - ta;
      ++ta;
    }
    const int tb = ta + (int)pr;
    const int a0 = ta * kWTile, b0 = tb * kWTile;
    const int64_t i0 = c * chunk, i1 = min((int64_t)n, i0 + chunk);
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t ib = i0; ib < i1; ib += kWTile) {
      // stage 32 nodes x 32 pivots of each side, centred by the column means
      for (int e = threadIdx.x; e < kWTile * kWTile; e += blockDim.x) {
        const int pv = e / kWTile, nd = e % kWTile;
        const int64_t i = ib + nd;
        double va = 0.0, vb = 0.0;
        if (i < i1) {
          if (a0 + pv < k) {
            const double d = (double)__ldg(dist + (size_t)(a0 + pv) * n + i);
            va = d * d - colsum[a0 + pv] * inv_n;
          }
          if (b0 + pv < k) {
            const double d = (double)__ldg(dist + (size_t)(b0 + pv) * n + i);
            vb = d * d - colsum[b0 + pv] * inv_n;
          }
        }
        sa[nd][pv] = va;
        sb[nd][pv] = vb;
      }
      __syncthreads();
#pragma unroll 4
      for (int nd = 0; nd < kWTile; ++nd) {
        const double x0 = sa[nd][2 * ty], x1 = sa[nd][2 * ty + 1];
        const double y0 = sb[nd][2 * tx], y1 = sb[nd][2 * tx + 1];
        acc[0][0] += x0 * y0;
        acc[0][1] += x0 * y1;
        acc[1][0] += x1 * y0;
        acc[1][1] += x1 * y1;
      }
      __syncthreads();
    }
    double *pg = partg + (size_t)c * k * k;
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int a = a0 + 2 * ty + p, b = b0 + 2 * tx + q;
        if (a < k && b < k) pg[(size_t)a * k + b] = acc[p][q];
      }
  }
}

// G'_ab (a <= b, mirrored) = sum of the chunk partials in chunk order
__global__ void k_wgram_reduce(int32_t k, int64_t nchunks, const double *__restrict__ partg, double *__restrict__ G) {
  const int64_t kk = (int64_t)k * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < kk; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / k), b = (int)(t - (int64_t)a * k);
    if (a > b) continue;
    double g = 0.0;
    for (int64_t c = 0; c < nchunks; ++c) g += partg[(size_t)c * kk + t];
    G[(size_t)a * k + b] = g;
    G[(size_t)b * k + a] = g;
  }
}


// x_i = C v = -1/2 (sum_a d_ia^2 v_a - rbar_i sigma - kappa), FP64
__global__ void __launch_bounds__(256) k_wproject(int32_t n, int32_t k, const float *__restrict__ dist,
                                                  const double *__restrict__ vv, const EigOut *__restrict__ eo,
                                                  void *__restrict__ pos, int precision) {
  extern __shared__ __align__(16) double svv[];  // v0[k], v1[k]
  for (int a = threadIdx.x; a < 2 * k; a += blockDim.x) svv[a] = vv[a];
  __syncthreads();
  const double sig0 = eo->sigma[0], sig1 = eo->sigma[1], kap0 = eo->kappa[0], kap1 = eo->kappa[1];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = 0.0, y = 0.0, rs = 0.0;
    for (int a = 0; a < k; ++a) {
      const double d = (double)__ldg(dist + (size_t)a * n + i);
      const double dd = d * d;
      rs += dd;
      x += dd * svv[a];
      y += dd * svv[k + a];
    }
    const double rbar = rs / (double)k;
    x = -0.5 * (x - rbar * sig0 - kap0);
    y = -0.5 * (y - rbar * sig1 - kap1);
    if (precision == 64) reinterpret_cast<double2 *>(pos)[i] = make_double2(x, y);
    else reinterpret_cast<float2 *>(pos)[i] = make_float2((float)x, (float)y);
  }
}

struct WMdsWs {
  double *colsum, *partc, *partg;
};

static size_t carve_wmds(Carver &c, MdsWs &w, WMdsWs &x, int32_t n, int32_t k) {
  carve_mds(c, w, n, k);
  const int64_t ch = wgram_chunk(n), nch = ((int64_t)n + ch - 1) / ch;
  x.colsum = c.take<double>((size_t)k);
  x.partc = c.take<double>((size_t)k * nch);
  x.partg = c.take<double>((size_t)nch * k * k);
  return c.size();
}

}  // namespace ssm

SSM_API size_t ssm_pivotmds_weighted_workspace(int32_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::MdsWs w;
  ssm::WMdsWs x;
  return ssm::carve_wmds(c, w, x, n, k);
}

SSM_API int ssm_pivotmds_weighted(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen,
                                  int32_t k, const float *dist, void *pos, int32_t precision, int32_t rescale,
                                  double *eig, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !dist || !pos || !status || !ws || (rescale && (!rowptr || !colidx || !elen)))
    return fail(SSM_E_ARG, "ssm_pivotmds_weighted: null pointer or n < 1");
  if (k < 2 || k > kMaxPivotsMds || k > n)
    return fail(SSM_E_ARG, "ssm_pivotmds_weighted: need 2 <= k <= min(n, %d)", kMaxPivotsMds);
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_pivotmds_weighted: precision must be 32 or 64");
  Carver c(ws, ws_bytes);
  MdsWs w;
  WMdsWs x;
  carve_wmds(c, w, x, n, k);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_pivotmds_weighted: workspace %zu bytes, need %zu", ws_bytes, c.size());
  const int sms = num_sms();
  const int64_t ch = wgram_chunk(n), nch = ((int64_t)n + ch - 1) / ch;
  const int ntiles = (k + kWTile - 1) / kWTile;
  SSM_TRY_CUDA(cudaMemsetAsync(w.done, 0, sizeof(unsigned), s));
  note_launch(), k_wcolsum_part<<<(unsigned)std::min<int64_t>((int64_t)k * nch, (int64_t)sms * 8), 256, 0, s>>>(
      n, k, dist, ch, nch, x.partc);
  note_launch(), k_wcolsum_final<<<std::max(1, (k + 255) / 256), 256, 0, s>>>(k, nch, x.partc, x.colsum);
  const int64_t gtasks = (int64_t)ntiles * (ntiles + 1) / 2 * nch;
  note_launch(), k_wgram<<<(unsigned)std::min<int64_t>(gtasks, (int64_t)sms * 8), 256, 0, s>>>(
      n, k, dist, x.colsum, ch, nch, ntiles, x.partg);
  const int64_t kk = (int64_t)k * k;
  note_launch(), k_wgram_reduce<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((kk + 255) / 256, sms * 4)), 256, 0,
                                  s>>>(k, nch, x.partg, w.B);
  // B = 1/4 (G' - rowmean_a - rowmean_b + grand mean)
  note_launch(), k_row_means<<<1, 1024, 0, s>>>(k, w.B, w.rowmean);
  note_launch(), k_center<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((kk + 255) / 256, sms * 4)), 256, 0, s>>>(
      k, w.B, w.rowmean);
  if (int rc = launch_eigen(n, k, w, (const double *)x.colsum, eig, status, s)) return rc;
  const int pb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)sms * 8);
  note_launch(), k_wproject<<<pb, 256, 2 * (size_t)k * sizeof(double), s>>>(n, k, dist, w.vv, w.eo, pos, precision);
  if (rescale) return launch_rescale(n, rowptr, colidx, elen, pos, precision, w, status, s);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
