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
// The FP32 kernel evaluates the same update about x_i (W = sum_a w'_ia):
//   x_i^{t+1} = x_i + (sum_a (B_a - w'_ia)(x_i - x_pa)
//                      + sum_j (x_j - x_i)(1 - 1/r_ij)) / den,  B_a = w'_ia d_ia / r_ia,
// since num = x_i den + those two sums; every sum is over differences, so the
// result does not depend on where the layout sits, and a pivot costs two
// accumulations per node instead of four.
//
// FP32 kernel, GB300 layout:
//  * a lane owns kNpl = 4 consecutive nodes (two packed pairs); their d_ia for
//    one pivot arrive in one 8-byte load, and the pivot's position and table
//    row serve all four.  ssm_iterate first re-lays d_ip into 128-node tiles
//    ([tile][pivot][128 nodes]), so a warp streams one contiguous block per
//    tile, a 256-byte row per pivot at a fixed stride (no per-load address
//    arithmetic);
//  * full-table mode (graphs whose largest d_ip fits a k x (dmax+1) table in
//    shared memory, e.g. small-world graphs): the table holds (w, w d) for
//    every pivot and distance, w = s / d^2 (stored as -w), so a term is one
//    table gather, one rsqrt (u = 1/r) and B - w = (w d) u - w; it adds
//    (B - w)(x_i - x_p).  The denominator deg(i) + sum_a w'_ia does not
//    change between iterations and is summed once per ssm_iterate call;
//  * clamped mode (large distances): s comes from a per-pivot table indexed
//    directly by d (0 for d < 2, cnt[min(d/2, ecc)] up to d = 2 ecc + 2, then
//    |R(a)|), and the term uses one rsqrt per node: with q = d^2 r^2,
//    u = q^{-1/2}, B = s u = w d / r and W = B u r^2 = s / d^2 = w, it adds
//    (B - W)(x_i - x_p) to the numerator and W to the denominator;
//  * in both modes the node pair is evaluated with packed FP32x2 arithmetic
//    where the operands pair up naturally; r^2 gets + 1e-24 so coincident
//    points (r == 0, x_i - x_p = 0) add nothing about x_i, i.e. w x_p, as the
//    r == 0 rule says (the clamped mode
//    also adds 1e-36 to q so it stays positive at d = 0; relative change of a
//    term with r >= 1e-6 below 1e-12); tables and pivot positions sit in
//    shared memory, loaded once per persistent block;
//  * the neighbour terms of every node are summed first by k_sweep_nbr, one
//    thread per row of up to kShortDeg entries, one warp per row up to
//    kMidDeg, one block per longer row (each sum in a fixed order); the
//    tile kernel reads them with the node's other per-node data;
//  * warps take 128-node tiles from an atomic counter; when there are too few
//    tiles to keep every warp busy to the end, each tile's pivots are split
//    into nsplit ranges taken as separate tasks, and the last range of a tile
//    to finish adds the ranges' partial sums in range order (independent of
//    timing) and updates the tile's nodes.
// The relative change ||X^{t+1}-X^t||/||X^t|| is reduced in FP64 in a fixed
// order by the last block to finish.
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace ssm {

constexpr int kSweepThreads = 256;
constexpr size_t kSmemBudget = 200 * 1024;
constexpr int kFullPlane = 6112;  // full-table mode: k (max d + 1) <= this; w and w d in two planes of this many floats
constexpr unsigned kFullPlaneBytes = kFullPlane * 4u;
// full-table mode: both planes in static shared memory (a fixed address, so a
// table read is one shared load at the node's byte offset plus a constant)
__shared__ __align__(16) float g_wtab[2 * kFullPlane];
// How the full-table kernel reads its table: 0 inline-asm shared loads from
// the two planes at 32-bit shared addresses, 1 plain shared loads from the two
// planes (measured within 1 %; an interleaved (w, w d) entry per node was 5 %
// slower)
#ifndef SSM_SWEEP_FULL_LDS
#define SSM_SWEEP_FULL_LDS 0
#endif
constexpr int kFullLds = SSM_SWEEP_FULL_LDS;
// bytes per table entry in the offsets that the tiled copy carries
constexpr unsigned kTabEntryBytes = 4u;
constexpr int kMaxPivotsSweep = 4096;
constexpr float kR2Floor = 1e-24f;
#ifndef SSM_SWEEP_PREFETCH
#define SSM_SWEEP_PREFETCH 8
#endif
#ifndef SSM_SWEEP_MIN_BLOCKS
#define SSM_SWEEP_MIN_BLOCKS 2
#endif
#ifndef SSM_SWEEP_FULL_MIN_BLOCKS
#define SSM_SWEEP_FULL_MIN_BLOCKS 3
#endif
constexpr int kPrefetch = SSM_SWEEP_PREFETCH;  // pivots whose d words are loaded ahead
// 1: the tile's positions are read again for the update instead of being kept in registers
#ifndef SSM_SWEEP_RELOAD_X
#define SSM_SWEEP_RELOAD_X 0
#endif
#ifndef SSM_SWEEP_NPL
#define SSM_SWEEP_NPL 4
#endif
constexpr int kNpl = SSM_SWEEP_NPL;        // nodes per lane in the FP32 sweep (2 or 4)
constexpr int kPpl = kNpl / 2;             // node pairs per lane (packed FP32x2)
constexpr int kTileNodes = 32 * kNpl;      // nodes per warp task
static_assert(kNpl == 2 || kNpl == 4, "two or four nodes per lane");
// the kPpl 32-bit words (two 16-bit distances each) a lane loads per pivot
typedef std::conditional<kPpl == 2, uint2, unsigned>::type DWords;
__device__ __forceinline__ unsigned dword(uint2 w, int j) { return j == 0 ? w.x : w.y; }
__device__ __forceinline__ unsigned dword(unsigned w, int) { return w; }

struct SweepArgs {
  int32_t n, k;
  const int32_t *rowptr, *colidx, *pivots, *cnt_off;
  const uint16_t *dip;
  const unsigned *dtile;  // d_ip re-laid as [tile][pivot][32 lanes][kPpl words of two nodes] (kTileNodes-node tiles)
  const uint32_t *cnt;
  int32_t cnt_len;
  int32_t stab_len;       // 2 cnt_len + k
  const float *stab;      // [stab_len] s by d, per pivot (global copy)
  const float *wtab;      // [2][kFullPlane]: w by pivot and distance ([k][dmax+1]), then w d (full-table mode)
  int32_t dmax;           // largest d_ip entry (full-table mode)
  const float *den;       // [n] deg(i) + sum_a w'_ia (full-table mode)
  const float2 *nb;       // [n] neighbour sums of this iteration (k_sweep_nbr)
  unsigned *tile_ctr;     // next task to hand out
  unsigned *done_ctr;     // blocks finished
  double *tile_part;      // [ntiles][2] (sum dx^2, sum x^2) per tile
  int32_t nsplit;         // pivot ranges per tile (1: a warp takes whole tiles)
  int32_t psplit;         // pivots per range
  float2 *part;           // [3 kPpl][ntiles * nsplit][32] partial sums of the ranges (nsplit > 1)
  unsigned *arrive;       // [ntiles] ranges of the tile finished so far (nsplit > 1)
  int32_t *stop;          // set when the relative change fell below tol
  int32_t *iters_done;
  double *rel_change;
  double tol;
  int32_t *status;
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

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Programmatic dependent launch: the sweep's kernels are launched so that the
// next one may start while the previous one drains; it waits here before it
// touches anything the previous kernel writes (a no-op without that launch mode).
__device__ __forceinline__ void wait_previous_kernel() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// lets the next kernel's blocks be scheduled as this kernel's blocks leave
// (they still wait for its completion in wait_previous_kernel)
__device__ __forceinline__ void allow_next_kernel() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float lds_f32(unsigned addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
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
  // four independent partial sums per thread keep loads in flight; they are
  // added in a fixed order, so the result does not depend on timing
  double nq[4] = {0.0, 0.0, 0.0, 0.0}, dq[4] = {0.0, 0.0, 0.0, 0.0};
  const unsigned step = 4u * blockDim.x;
  for (unsigned t0 = threadIdx.x; t0 < ntiles; t0 += step) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const unsigned t = t0 + (unsigned)q * blockDim.x;
      if (t < ntiles) {
        const double2 v = __ldcg(reinterpret_cast<const double2 *>(A.tile_part) + t);
        nq[q] += v.x;
        dq[q] += v.y;
      }
    }
  }
  double num = (nq[0] + nq[1]) + (nq[2] + nq[3]), den = (dq[0] + dq[1]) + (dq[2] + dq[3]);
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

// neighbour term less x_i: x_j + (x_i - x_j)/r - x_i = (x_j - x_i)(1 - 1/r)
// (r == 0: x_j - x_i = 0)
__device__ __forceinline__ void edge_term(float xi, float yi, float2 q, float &sx, float &sy) {
  const float ex = q.x - xi, ey = q.y - yi;
  const float r2 = fmaf(ex, ex, ey * ey);
  const float f = r2 > 0.f ? 1.f - rsqrt_approx(r2) : 0.f;
  sx = fmaf(ex, f, sx);
  sy = fmaf(ey, f, sy);
}

// one lane walks a short row in batches of kNbrBatch: the batch's column
// indices load together, then its positions, so a row of up to kNbrBatch
// entries costs two dependent memory latencies (terms still added in row order)
#ifndef SSM_NBR_BATCH
#define SSM_NBR_BATCH 8
#endif
constexpr int kNbrBatch = SSM_NBR_BATCH;  // column indices (then positions) a lane loads at once

__device__ __forceinline__ void light_row(const float2 *__restrict__ pin, const int32_t *__restrict__ colidx, int beg,
                                          int end, float xi, float yi, float &sx, float &sy) {
  for (int t = beg; t < end; t += kNbrBatch) {
    int j[kNbrBatch];
#pragma unroll
    for (int q = 0; q < kNbrBatch; ++q) j[q] = t + q < end ? __ldg(colidx + t + q) : -1;
    float2 x[kNbrBatch];
#pragma unroll
    for (int q = 0; q < kNbrBatch; ++q) x[q] = j[q] >= 0 ? pin[j[q]] : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < kNbrBatch; ++q)
      if (j[q] >= 0) edge_term(xi, yi, x[q], sx, sy);
  }
}

// the whole warp walks one row segment [b, e) around (hx, hy); the sums land in every lane
__device__ __forceinline__ void warp_row(const float2 *__restrict__ pin, const int32_t *__restrict__ colidx, int b,
                                         int e, float hx, float hy, float &sx, float &sy) {
  const int lane = threadIdx.x & 31;
  sx = 0.f;
  sy = 0.f;
  int t = b + lane;
  for (; t + 32 < e; t += 64) {
    const float2 q0 = pin[__ldg(colidx + t)], q1 = pin[__ldg(colidx + t + 32)];
    edge_term(hx, hy, q0, sx, sy);
    edge_term(hx, hy, q1, sx, sy);
  }
  for (; t < e; t += 32) edge_term(hx, hy, pin[__ldg(colidx + t)], sx, sy);
  sx = warp_sumf(sx);
  sy = warp_sumf(sy);
}

// Neighbour sums nb[i] = sum_{j in N(i)} (x_j + (x_i - x_j)/r_ij - x_i) =
// sum_j (x_j - x_i)(1 - 1/r_ij) (r == 0: 0) for one iteration.  Blocks [0, nlong) take one long row each (a
// block-stride walk, then a fixed-order block sum), the next ceil(nmid / 8)
// blocks one medium row per warp, the rest one node per thread (rows of at
// most kShortDeg entries; longer rows were listed).  Every sum has a fixed
// order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) k_sweep_nbr(int32_t n, const int32_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ colidx, const float2 *__restrict__ pin,
                                                   int32_t nlong, const int32_t *__restrict__ long_rows, int32_t nmid,
                                                   const int32_t *__restrict__ mid_rows, float2 *__restrict__ nb,
                                                   const int32_t *__restrict__ stop) {
  allow_next_kernel();
  wait_previous_kernel();
  if (__ldcg(stop)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int b = blockIdx.x;
  if (b < nlong) {
    __shared__ float red[2][8];
    const int i = __ldg(long_rows + b);
    const int rb = __ldg(rowptr + i), re = __ldg(rowptr + i + 1);
    const float2 xi = pin[i];
    float sx = 0.f, sy = 0.f;
    for (int t = rb + (int)threadIdx.x; t < re; t += (int)blockDim.x) edge_term(xi.x, xi.y, pin[__ldg(colidx + t)], sx, sy);
    sx = warp_sumf(sx);
    sy = warp_sumf(sy);
    if (lane == 0) {
      red[0][warp] = sx;
      red[1][warp] = sy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float ax = 0.f, ay = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        ax += red[0][w];
        ay += red[1][w];
      }
      nb[i] = make_float2(ax, ay);
    }
    return;
  }
  b -= nlong;
  const int midb = (nmid + 7) / 8;
  if (b < midb) {
    const int r = b * 8 + warp;
    if (r >= nmid) return;
    const int i = __ldg(mid_rows + r);
    const float2 xi = pin[i];
    float sx, sy;
    warp_row(pin, colidx, __ldg(rowptr + i), __ldg(rowptr + i + 1), xi.x, xi.y, sx, sy);
    if (lane == 0) nb[i] = make_float2(sx, sy);
    return;
  }
  b -= midb;
  const int i = b * (int)blockDim.x + (int)threadIdx.x;
  if (i >= n) return;
  const int rb = __ldg(rowptr + i), re = __ldg(rowptr + i + 1);
  if (re - rb > kShortDeg) return;
  const float2 xi = pin[i];
  float sx = 0.f, sy = 0.f;
  light_row(pin, colidx, rb, re, xi.x, xi.y, sx, sy);
  nb[i] = make_float2(sx, sy);
}

// lists the rows longer than kShortDeg (medium: up to kMidDeg) for k_sweep_nbr;
// counts[0] = medium rows, counts[1] = long rows
__global__ void k_nbr_classify(int32_t n, const int32_t *__restrict__ rowptr, unsigned *__restrict__ counts,
                               int32_t *__restrict__ mid_rows, int32_t *__restrict__ long_rows) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int deg = rowptr[i + 1] - rowptr[i];
    if (deg > kMidDeg)
      long_rows[atomicAdd(counts + 1, 1u)] = (int32_t)i;
    else if (deg > kShortDeg)
      mid_rows[atomicAdd(counts, 1u)] = (int32_t)i;
  }
}

// ----------------------------------------------------------------- FP32
__device__ __forceinline__ float2 lds_f32x2(unsigned addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}

// MODE: kClampSmem / kClampGlobal (s table in shared / global memory), kFull
constexpr int kClampSmem = 0, kClampGlobal = 1, kFull = 2;

template <int MODE>
__global__ void __launch_bounds__(kSweepThreads, MODE == 2 ? SSM_SWEEP_FULL_MIN_BLOCKS : SSM_SWEEP_MIN_BLOCKS) k_sweep_f32(SweepArgs A, const float2 *__restrict__ pin,
                                                              float2 *__restrict__ pout) {
  constexpr bool SMEM = MODE == kClampSmem;
  constexpr bool FULL = MODE == kFull;
  extern __shared__ __align__(16) unsigned char smem[];
  float4 *pxy = reinterpret_cast<float4 *>(smem);       // (-x, -x, -y, -y) per pivot
  uint2 *pidx = reinterpret_cast<uint2 *>(pxy + A.k);   // (table address base, clamp) per pivot
  float *stab = reinterpret_cast<float *>(pidx + A.k);  // s by d
  const int n = A.n, k = A.k;
  // with pivot ranges split into tasks (graphs of few tiles) the next
  // iteration's neighbour kernel may take the slots of finished blocks early;
  // with whole tiles that measured slower, so there it is not let in
  if (A.nsplit > 1) allow_next_kernel();
  // the weight tables do not depend on the previous kernels: load them first
  if (SMEM)
    for (int t = threadIdx.x; t < A.stab_len; t += blockDim.x) stab[t] = __ldg(A.stab + t);
  if constexpr (FULL)
    for (int t = threadIdx.x; t < k * (A.dmax + 1); t += blockDim.x) {
      g_wtab[t] = __ldg(A.wtab + t);
      g_wtab[kFullPlane + t] = __ldg(A.wtab + kFullPlane + t);
    }
  wait_previous_kernel();
  if (__ldcg(A.stop)) return;
  // Table address of node distance d for pivot a: with c = bits(2^23 + min(d, D_a))
  // (a float whose low bits are the integer), addr = 4 c + base_a where
  // base_a = table start + 4 offset_a - 4 * 0x4B000000 (mod 2^32).
  const unsigned tab0 = SMEM ? (unsigned)__cvta_generic_to_shared(stab) : 0u;
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    int p = __ldg(A.pivots + a);
    if ((unsigned)p >= (unsigned)n) {  // a pivot id outside the graph: recorded, read as node 0
      dev_fail(A.status, SSM_E_ARG);
      p = 0;
    }
    const float2 xy = pin[p];
    const int o = __ldg(A.cnt_off + a), e = __ldg(A.cnt_off + a + 1);
    // pivot a's table: d = 0 .. D_a = 2 ecc_a + 2 at 2 off_a + a (D_a >= 2, so a region
    // of the pivot alone, ecc_a = 0, still gets s = |R(a)| = 1 at d >= 2)
    const unsigned soff = 2u * (unsigned)o + (unsigned)a, dcap = 2u * (unsigned)(e - o);
    pxy[a] = make_float4(-xy.x, -xy.x, -xy.y, -xy.y);
    pidx[a] = make_uint2(tab0 + 4u * soff - 4u * 0x4B000000u, 0x4B000000u | dcap);
  }
  unsigned wtab0 = 0u;
  if constexpr (FULL) wtab0 = (unsigned)__cvta_generic_to_shared(g_wtab);
  __syncthreads();

  const unsigned lane = threadIdx.x & 31u;
  const unsigned ntiles = (unsigned)((n + kTileNodes - 1) / kTileNodes);
  const unsigned nsplit = (unsigned)A.nsplit, ntasks = ntiles * nsplit;
  // loop-invariant constant pairs, kept in registers (opaque to the compiler so
  // it does not rebuild them from immediates inside the pivot loop)
  float2 kMagic2 = make_float2(-8388608.f, -8388608.f);
  asm volatile("" : "+f"(kMagic2.x), "+f"(kMagic2.y));
  for (;;) {
    unsigned task = 0;
    if (lane == 0) task = atomicAdd(A.tile_ctr, 1u);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= ntasks) break;
    const unsigned tile = task / nsplit, split = task - tile * nsplit;
    const int a_lo = (int)split * A.psplit, a_hi = min(k, a_lo + A.psplit);

    // ---- a tile of kTileNodes nodes: this lane owns i0 .. i0 + kNpl - 1, as
    // kPpl pairs (2j, 2j + 1) whose arithmetic is packed FP32x2
    const int i0 = (int)(tile * (unsigned)kTileNodes + (unsigned)kNpl * lane);
    float2 xi2[kPpl], yi2[kPpl], xs[kNpl];
#pragma unroll
    for (int q = 0; q < kNpl; ++q) xs[q] = i0 + q < n ? pin[i0 + q] : make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kPpl; ++j) {
      xi2[j] = make_float2(xs[2 * j].x, xs[2 * j + 1].x);
      yi2[j] = make_float2(xs[2 * j].y, xs[2 * j + 1].y);
    }

    // pivot terms, a in [a_lo, a_hi).  The d words of the next kPrefetch pivots
    // are always in flight; lanes past the last node read zeros (d = 0: no
    // term).  A pivot adds w x_p + B (x_i - x_p) to the numerator and w to the
    // denominator (B = w d / r); about x_i that is (B - w)(x_i - x_p) added to
    // ax, ay (and w to den in the clamped mode)
    float2 ax2[kPpl], ay2[kPpl], den2[kPpl];
#pragma unroll
    for (int j = 0; j < kPpl; ++j) {
      ax2[j] = ay2[j] = den2[j] = make_float2(0.f, 0.f);
    }
    // this tile's d words: pivot a of lane l at tp[a * 32] (one contiguous
    // 32 kPpl-word row per pivot, kPpl words -- kNpl distances -- per lane)
    const DWords *tp = reinterpret_cast<const DWords *>(A.dtile) + (size_t)tile * (size_t)k * 32u + lane;
    auto load_words = [&](int a) -> DWords { return __ldg(tp + (unsigned)a * 32u); };
    float2 kTiny2 = make_float2(kR2Floor, kR2Floor), kTinyQ2 = make_float2(1e-36f, 1e-36f);
    float2 kMinus2 = make_float2(-1.f, -1.f);
    asm volatile("" : "+f"(kTiny2.x), "+f"(kTiny2.y), "+f"(kTinyQ2.x), "+f"(kTinyQ2.y));
    if (!FULL) asm volatile("" : "+f"(kMinus2.x), "+f"(kMinus2.y));
    // full-table mode: a d word holds the byte offsets 4 (a (dmax + 1) + d) of
    // two nodes' table entries; -w and w d of a node pair land in register
    // pairs (the two planes sit a fixed kFullPlaneBytes apart), so every
    // product is packed
    auto pivot_term_full = [&](int a, DWords pw) {
      const float4 P = pxy[a];  // (-x, -x, -y, -y)
      const float2 px2 = make_float2(P.x, P.y), py2 = make_float2(P.z, P.w);
#pragma unroll
      for (int j = 0; j < kPpl; ++j) {
        const unsigned pk = dword(pw, j);
        float2 nw2, wd2;
        if constexpr (kFullLds == 0) {
          const unsigned al = wtab0 + (pk & 0xFFFFu), ah = wtab0 + (pk >> 16);
          nw2 = make_float2(lds_f32(al), lds_f32(ah));
          wd2 = make_float2(lds_f32(al + kFullPlaneBytes), lds_f32(ah + kFullPlaneBytes));
        } else {
          const char *tb = reinterpret_cast<const char *>(g_wtab);
          const unsigned ol = pk & 0xFFFFu, oh = pk >> 16;
          nw2 = make_float2(*reinterpret_cast<const float *>(tb + ol), *reinterpret_cast<const float *>(tb + oh));
          wd2 = make_float2(*reinterpret_cast<const float *>(tb + kFullPlaneBytes + ol),
                            *reinterpret_cast<const float *>(tb + kFullPlaneBytes + oh));
        }
        const float2 dx2 = __fadd2_rn(xi2[j], px2);
        const float2 dy2 = __fadd2_rn(yi2[j], py2);
        const float2 r2 = __ffma2_rn(dx2, dx2, __ffma2_rn(dy2, dy2, kTiny2));
        float2 u2;
        u2.x = rsqrt_approx(r2.x);
        u2.y = rsqrt_approx(r2.y);
        const float2 c2 = __ffma2_rn(wd2, u2, nw2);  // B - w = w d / r - w
        ax2[j] = __ffma2_rn(c2, dx2, ax2[j]);
        ay2[j] = __ffma2_rn(c2, dy2, ay2[j]);
      }
    };
    auto pivot_term = [&](int a, DWords pw) {
      if constexpr (FULL) {
        pivot_term_full(a, pw);
        return;
      }
      const float4 P = pxy[a];  // (-x, -x, -y, -y)
      const uint2 I = pidx[a];
      const float2 px2 = make_float2(P.x, P.y), py2 = make_float2(P.z, P.w);
      const float cap = __uint_as_float(I.y);
#pragma unroll
      for (int j = 0; j < kPpl; ++j) {
        const unsigned pk = dword(pw, j);
        // 2^23 + d as a float for each node (exact), and the same clamped at 2^23 + D_a
        float2 f2;
        f2.x = __uint_as_float(__byte_perm(pk, 0x4B00u, 0x5410u));
        f2.y = __uint_as_float(__byte_perm(pk, 0x4B00u, 0x5432u));
        float2 s2;
        if (SMEM) {
          s2.x = lds_f32(4u * __float_as_uint(fminf(f2.x, cap)) + I.x);
          s2.y = lds_f32(4u * __float_as_uint(fminf(f2.y, cap)) + I.x);
        } else {
          const unsigned soff = (I.x + 4u * 0x4B000000u) >> 2;
          s2.x = __ldg(A.stab + soff + (__float_as_uint(fminf(f2.x, cap)) - 0x4B000000u));
          s2.y = __ldg(A.stab + soff + (__float_as_uint(fminf(f2.y, cap)) - 0x4B000000u));
        }
        const float2 d2 = __fadd2_rn(f2, kMagic2);
        const float2 dx2 = __fadd2_rn(xi2[j], px2);
        const float2 dy2 = __fadd2_rn(yi2[j], py2);
        // r^2 + 1e-24: coincident points (r == 0) add w x_p only, as the r == 0 rule says
        const float2 r2 = __ffma2_rn(dx2, dx2, __ffma2_rn(dy2, dy2, kTiny2));
        // + 1e-36 keeps q > 0 when d = 0 (the node is pivot a; s = 0 there)
        const float2 q2 = __ffma2_rn(__fmul2_rn(d2, d2), r2, kTinyQ2);
        float2 u2;
        u2.x = rsqrt_approx(q2.x);
        u2.y = rsqrt_approx(q2.y);
        const float2 B2 = __fmul2_rn(s2, u2);                  // s/(d r) = w d / r
        const float2 W2 = __fmul2_rn(__fmul2_rn(B2, u2), r2);  // s/d^2 = w
        const float2 c2 = __ffma2_rn(W2, kMinus2, B2);         // B - w
        ax2[j] = __ffma2_rn(c2, dx2, ax2[j]);
        ay2[j] = __ffma2_rn(c2, dy2, ay2[j]);
        den2[j] = __fadd2_rn(den2[j], W2);
      }
    };
    DWords buf[kPrefetch];
    int a0 = a_lo;
    if (a_hi - a_lo >= 2 * kPrefetch) {
#pragma unroll
      for (int t = 0; t < kPrefetch; ++t) buf[t] = load_words(a0 + t);
      for (; a0 + 2 * kPrefetch <= a_hi; a0 += kPrefetch) {
#pragma unroll
        for (int t = 0; t < kPrefetch; ++t) {
          const DWords pw = buf[t];
          buf[t] = load_words(a0 + kPrefetch + t);
          pivot_term(a0 + t, pw);
        }
      }
#pragma unroll
      for (int t = 0; t < kPrefetch; ++t) pivot_term(a0 + t, buf[t]);
      a0 += kPrefetch;
    }
    for (; a0 < a_hi; ++a0) pivot_term(a0, load_words(a0));
    if (nsplit > 1) {
      // publish this range's sums; the last range of the tile adds all of them
      // in range order and goes on to update the nodes.  Layout:
      // part[(q kPpl + j) stride + task 32 + lane], q = ax, ay, den
      const size_t stride = (size_t)ntasks * 32u;
      float2 *pp = A.part + (size_t)task * 32u + lane;
#pragma unroll
      for (int j = 0; j < kPpl; ++j) {
        pp[(0 * kPpl + j) * stride] = ax2[j];
        pp[(1 * kPpl + j) * stride] = ay2[j];
        if (!FULL) pp[(2 * kPpl + j) * stride] = den2[j];
      }
      __threadfence();
      __syncwarp();
      unsigned prior = 0;
      if (lane == 0) prior = atomicAdd(A.arrive + tile, 1u);
      prior = __shfl_sync(0xffffffffu, prior, 0);
      if (prior != nsplit - 1) continue;
      __threadfence();
      if (lane == 0) A.arrive[tile] = 0u;  // ready for the next iteration
      const float2 *q = A.part + (size_t)tile * nsplit * 32u + lane;
#pragma unroll
      for (int j = 0; j < kPpl; ++j) {
        float2 s0 = __ldcg(q + (0 * kPpl + j) * stride), s1 = __ldcg(q + (1 * kPpl + j) * stride);
        float2 s2 = FULL ? make_float2(0.f, 0.f) : __ldcg(q + (2 * kPpl + j) * stride);
        for (unsigned r = 1; r < nsplit; ++r) {
          const float2 *qr = q + (size_t)r * 32u;
          s0 = __fadd2_rn(s0, __ldcg(qr + (0 * kPpl + j) * stride));
          s1 = __fadd2_rn(s1, __ldcg(qr + (1 * kPpl + j) * stride));
          if (!FULL) s2 = __fadd2_rn(s2, __ldcg(qr + (2 * kPpl + j) * stride));
        }
        ax2[j] = s0;
        ay2[j] = s1;
        den2[j] = s2;
      }
    }

    // X^{t+1} and this tile's share of the relative change
    float cn = 0.f, cd = 0.f;
    int rprev = 0;
    if (!FULL && i0 < n) rprev = __ldg(A.rowptr + i0);
#pragma unroll
    for (int q = 0; q < kNpl; ++q) {
      const int i = i0 + q;
      const int j = q >> 1;
      const bool hi = (q & 1) != 0;
      const bool live = i < n;
      // neighbour terms (w = 1, d = 1) less deg(i) x_i, summed by k_sweep_nbr
      const float2 nbq = live ? __ldg(A.nb + i) : make_float2(0.f, 0.f);
      float dn;
      if (FULL) {
        dn = live ? __ldg(A.den + i) : 0.f;
      } else {
        const int rnext = live ? __ldg(A.rowptr + i + 1) : rprev;
        dn = (hi ? den2[j].y : den2[j].x) + (float)(rnext - rprev);
        rprev = rnext;
      }
      const float nx = hi ? ax2[j].y : ax2[j].x;
      const float ny = hi ? ay2[j].y : ay2[j].x;
      // a NaN (clamped mode: in the weights; full-table mode: in the numerator) is an error
      const float chk = FULL ? nx + ny : (hi ? den2[j].y : den2[j].x);
      if (live && !(chk == chk)) dev_fail(A.status, SSM_E_NUMERIC);
      if (live) {
#if SSM_SWEEP_RELOAD_X
        const float2 x = pin[i];
#else
        const float2 x = xs[q];
#endif
        const float ex = dn > 0.f ? (nx + nbq.x) / dn : 0.f, ey = dn > 0.f ? (ny + nbq.y) / dn : 0.f;
        pout[i] = make_float2(x.x + ex, x.y + ey);
        cn = fmaf(ex, ex, fmaf(ey, ey, cn));
        cd = fmaf(x.x, x.x, fmaf(x.y, x.y, cd));
      }
    }
    const double tn = warp_sum((double)cn), td = warp_sum((double)cd);
    if (lane == 0) {
      A.tile_part[2 * (size_t)tile] = tn;
      A.tile_part[2 * (size_t)tile + 1] = td;
    }
  }
  finish_iteration(A, ntiles);
}

// ----------------------------------------------------------------- setup (once per ssm_iterate)
// dtile[((t k + a) 32 + l) kPpl + j] = e(d_ip[a][i]) | e(d_ip[a][i + 1]) << 16 with
// i = t kTileNodes + kNpl l + 2 j (d = 0 past the last node); e(d) = d, or in
// full-table mode (row = dmax + 1 > 0) the byte offset kTabEntryBytes (a row + d)
// of the node's entry in the shared-memory table.  A distance above the table
// (a wrong dmax hint) is recorded as SSM_E_ARG and clamped, so no table read
// leaves the table
__global__ void k_tile_dip(int32_t n, int32_t k, int32_t row, const uint16_t *__restrict__ dip,
                           unsigned *__restrict__ dtile, int32_t *__restrict__ status, int32_t pair_loads) {
  // node pair p = (2p, 2p + 1) of pivot a lands in word (t k + a) P + (p mod P), t = p div P,
  // P = kTileNodes / 2 pairs per tile; blocks step over pivots in y, pairs in x
  constexpr int64_t P = kTileNodes / 2;
  const int64_t npairs = ((int64_t)(n + kTileNodes - 1) / kTileNodes) * P;
  const unsigned top = row > 0 ? (unsigned)row - 1u : 0u;
  auto enc = [&](int a, unsigned lo, unsigned hi) -> unsigned {
    if (row > 0) {
      if (lo > top || hi > top) {
        dev_fail(status, SSM_E_ARG);
        lo = min(lo, top);
        hi = min(hi, top);
      }
      lo = kTabEntryBytes * ((unsigned)a * (unsigned)row + lo);
      hi = kTabEntryBytes * ((unsigned)a * (unsigned)row + hi);
    }
    return lo | (hi << 16);
  };
  if (pair_loads == 2) {
    // n a multiple of 8, dip 16-byte aligned: four pairs (one 16-byte load,
    // one 16-byte store of four consecutive words of a tile) per thread
    const int64_t nquads = npairs / 4;
    for (int a = blockIdx.y; a < k; a += gridDim.y) {
      const uint4 *drow = reinterpret_cast<const uint4 *>(dip + (size_t)a * n);
      for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nquads; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = 4 * g;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (2 * p + 7 < n) v = __ldg(drow + g);  // else past the last node: zeros (n % 8 == 0: all or nothing)
        const uint4 out = make_uint4(enc(a, v.x & 0xFFFFu, v.x >> 16), enc(a, v.y & 0xFFFFu, v.y >> 16),
                                     enc(a, v.z & 0xFFFFu, v.z >> 16), enc(a, v.w & 0xFFFFu, v.w >> 16));
        *reinterpret_cast<uint4 *>(dtile + ((p / P) * k + a) * P + (p % P)) = out;
      }
    }
    return;
  }
  for (int a = blockIdx.y; a < k; a += gridDim.y) {
    const uint16_t *drow = dip + (size_t)a * n;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = 2 * p;
      unsigned lo = 0u, hi = 0u;
      if (pair_loads && i + 1 < n) {  // n even and dip 4-byte aligned: the pair is one aligned word
        const unsigned v = __ldg(reinterpret_cast<const unsigned *>(drow + i));
        lo = v & 0xFFFFu;
        hi = v >> 16;
      } else {
        if (i < n) lo = (unsigned)__ldg(drow + i);
        if (i + 1 < n) hi = (unsigned)__ldg(drow + i + 1);
      }
      dtile[((p / P) * k + a) * P + (p % P)] = enc(a, lo, hi);
    }
  }
}


// s-by-d table: stab[2 off_a + a + d] = (d >= 2) ? cnt[off_a + min(d/2, ecc_a)] : 0,
// d = 0 .. 2 ecc_a + 2 (larger d clamp to the last entry, |R(a)|)
__global__ void k_build_stab(int32_t k, const int32_t *__restrict__ cnt_off, const uint32_t *__restrict__ cnt,
                             float *__restrict__ stab) {
  for (int a = blockIdx.x; a < k; a += gridDim.x) {
    const int o = cnt_off[a], ecc = cnt_off[a + 1] - o - 1;
    for (int d = threadIdx.x; d <= 2 * ecc + 2; d += blockDim.x)
      stab[2 * o + a + d] = d >= 2 ? (float)cnt[o + min(d >> 1, ecc)] : 0.f;
  }
}

// full-table mode: wtab[a (dmax+1) + d] = -w and wtab[kFullPlane + a (dmax+1) + d]
// = w d, w = s / d^2 with s as in k_build_stab (0 for d < 2), rounded from double
__global__ void k_build_wtab(int32_t k, int32_t dmax, const int32_t *__restrict__ cnt_off,
                             const uint32_t *__restrict__ cnt, float *__restrict__ wtab) {
  const int64_t total = (int64_t)k * (dmax + 1);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / (dmax + 1)), d = (int)(t - (int64_t)a * (dmax + 1));
    const int o = cnt_off[a], ecc = cnt_off[a + 1] - o - 1;
    float w = 0.f, wd = 0.f;
    if (d >= 2) {
      const double sd = (double)cnt[o + min(d >> 1, ecc)], dd = (double)d;
      w = (float)(sd / (dd * dd));
      wd = (float)(sd / dd);
    }
    wtab[t] = -w;
    wtab[kFullPlane + t] = wd;
  }
}

// full-table mode: den[i] = deg(i) + sum_{a = 0..k-1} w'_ia in FP32, pivots in
// order (the sum the clamped mode forms inside every sweep); one warp per tile;
// dtile holds table byte offsets
__global__ void k_sweep_den(int32_t n, int32_t k, const unsigned *__restrict__ dtile,
                            const float *__restrict__ wtab, const int32_t *__restrict__ rowptr,
                            float *__restrict__ den) {
  const unsigned lane = threadIdx.x & 31u;
  const int64_t ntiles = (n + kTileNodes - 1) / kTileNodes;
  for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < ntiles;
       tile += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const DWords *tp = reinterpret_cast<const DWords *>(dtile) + tile * (int64_t)k * 32 + lane;
    float acc[kNpl];
#pragma unroll
    for (int q = 0; q < kNpl; ++q) acc[q] = 0.f;
    for (int a = 0; a < k; ++a) {
      const DWords pw = __ldg(tp + (int64_t)a * 32);
#pragma unroll
      for (int j = 0; j < kPpl; ++j) {
        const unsigned pk = dword(pw, j);
        acc[2 * j] -= __ldg(wtab + (pk & 0xFFFFu) / kTabEntryBytes);  // the table holds -w
        acc[2 * j + 1] -= __ldg(wtab + (pk >> 16) / kTabEntryBytes);
      }
    }
    const int64_t i0 = tile * kTileNodes + (int64_t)kNpl * lane;
#pragma unroll
    for (int q = 0; q < kNpl; ++q)
      if (i0 + q < n) den[i0 + q] = acc[q] + (float)(rowptr[i0 + q + 1] - rowptr[i0 + q]);
  }
}

__global__ void k_dip_max(int64_t count, const uint16_t *__restrict__ dip, unsigned *__restrict__ out) {
  unsigned m = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned)__ldg(dip + t));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
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

template <bool CNT_SMEM>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_f64(SweepArgs A, const double2 *__restrict__ pin,
                                                              double2 *__restrict__ pout) {
  extern __shared__ __align__(16) unsigned char smem[];
  PivD *piv = reinterpret_cast<PivD *>(smem);
  double *cntd = reinterpret_cast<double *>(piv + A.k);
  if (__ldcg(A.stop)) return;
  const int n = A.n, k = A.k;
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    int p = __ldg(A.pivots + a);
    if ((unsigned)p >= (unsigned)n) {  // a pivot id outside the graph: recorded, read as node 0
      dev_fail(A.status, SSM_E_ARG);
      p = 0;
    }
    const double2 xy = pin[p];
    const int o = __ldg(A.cnt_off + a);
    piv[a] = PivD{xy.x, xy.y, o, __ldg(A.cnt_off + a + 1) - o - 1};
  }
  if (CNT_SMEM)
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
        const double s = CNT_SMEM ? cntd[P.off + h] : (double)__ldg(A.cnt + P.off + h);
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
  unsigned *ctr;  // [0] task counter, [1] done counter
  int32_t *stop;
  double *tile_part;
  float *stab;
  float2 *nb;       // [n] neighbour sums
  int32_t *mid_rows, *long_rows;  // [n] rows longer than kShortDeg / kMidDeg
  unsigned *dtile;
  float *wtab;    // full-table mode: w and w d planes
  float *den;     // [n] full-table mode denominators
  unsigned *meta;  // [4] largest d_ip entry, medium rows, long rows
  float2 *part;    // pivot-range partial sums (few-tile graphs), split_cap tasks
  unsigned *arrive;  // [tiles]
  int64_t split_cap;  // tasks the partial sums have room for (0: no splitting)
};

// Splitting tiles into pivot ranges pays only when there are fewer tiles than
// about two per resident warp; the sweep kernel keeps at most kSplitWarpsPerSm
// warps per SM, so larger graphs get no scratch for it.
#ifndef SSM_SWEEP_SPLIT_TASKS
#define SSM_SWEEP_SPLIT_TASKS 4
#endif
constexpr int kSplitTasksPerWarp = SSM_SWEEP_SPLIT_TASKS;  // target tasks per resident warp (0: never split)
constexpr int kMaxSplit = 8;
constexpr int kSplitWarpsPerSm = 32;
static int64_t split_capacity(int32_t n) {
  const int64_t tiles = ((int64_t)n + kTileNodes - 1) / kTileNodes;
  return tiles < 2 * (int64_t)num_sms() * kSplitWarpsPerSm ? kMaxSplit * tiles : 0;
}

// what the last ssm_iterate call on this host thread chose (ssm_last_sweep_config)
static thread_local int32_t g_last_config[4] = {-1, 0, 0, -1};

static size_t carve_iterate(Carver &c, IterWs &w, int32_t n, int64_t m2, int32_t k, int64_t cnt_len,
                            int32_t precision) {
  (void)m2;  // the sweep's scratch does not grow with the edge count
  const size_t elem = precision == 64 ? sizeof(double2) : sizeof(float2);
  w.tmp = c.take<char>((size_t)n * elem);
  w.ctr = c.take<unsigned>(2);
  w.stop = c.take<int32_t>(1);
  w.tile_part = c.take<double>(2 * ((size_t)n / 32 + 2));
  w.stab = c.take<float>((size_t)(2 * cnt_len + k));
  w.nb = precision == 64 ? nullptr : c.take<float2>((size_t)n);
  w.mid_rows = precision == 64 ? nullptr : c.take<int32_t>((size_t)n);
  w.long_rows = precision == 64 ? nullptr : c.take<int32_t>((size_t)n);
  w.dtile = precision == 64 ? nullptr : c.take<unsigned>((size_t)((n + kTileNodes - 1) / kTileNodes) * (size_t)k * 32 * kPpl);
  w.wtab = precision == 64 ? nullptr : c.take<float>(2 * (size_t)kFullPlane);
  w.den = precision == 64 ? nullptr : c.take<float>((size_t)n);
  w.meta = c.take<unsigned>(4);
  w.split_cap = precision == 64 ? 0 : split_capacity(n);
  w.part = w.split_cap ? c.take<float2>(3 * kPpl * 32 * (size_t)w.split_cap) : nullptr;
  w.arrive = w.split_cap ? c.take<unsigned>((size_t)((n + kTileNodes - 1) / kTileNodes)) : nullptr;
  return c.size();
}

}  // namespace ssm

SSM_API size_t ssm_iterate_workspace(int32_t n, int64_t m, int32_t k, int64_t cnt_len, int32_t precision) {
  if (n < 1 || m < 0 || k < 1 || cnt_len < 0) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::IterWs w;
  return ssm::carve_iterate(c, w, n, 2 * m, k, cnt_len, precision);
}

SSM_API int ssm_iterate(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                        const int32_t *pivots, const uint16_t *dip, const int32_t *cnt_off, const uint32_t *cnt,
                        int64_t cnt_len, void *pos, int32_t precision, int32_t iters, double tol,
                        int32_t *iters_done, double *rel_change, int32_t *status, const int32_t *hints, void *ws,
                        size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || m < 0 || !rowptr || !colidx || !pivots || !dip || !cnt_off || !cnt || !pos || !iters_done ||
      !rel_change || !status || !ws)
    return fail(SSM_E_ARG, "ssm_iterate: null pointer or bad size");
  if (k < 1 || k > kMaxPivotsSweep) return fail(SSM_E_ARG, "ssm_iterate: need 1 <= k <= %d", kMaxPivotsSweep);
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_iterate: precision must be 32 or 64");
  if (iters < 1) return fail(SSM_E_ARG, "ssm_iterate: iters must be >= 1");
  if (cnt_len < k || cnt_len >= ((int64_t)1 << 30)) return fail(SSM_E_ARG, "ssm_iterate: bad count-table length");
  Carver c(ws, ws_bytes);
  IterWs w;
  carve_iterate(c, w, n, 2 * m, k, cnt_len, precision);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_iterate: workspace %zu bytes, need %zu", ws_bytes, c.size());

  SweepArgs A;
  A.n = n; A.k = k; A.rowptr = rowptr; A.colidx = colidx; A.pivots = pivots; A.cnt_off = cnt_off;
  A.dip = dip; A.dtile = w.dtile; A.cnt = cnt; A.cnt_len = (int32_t)cnt_len; A.stab_len = (int32_t)(2 * cnt_len + k);
  A.stab = w.stab; A.wtab = nullptr; A.dmax = 0; A.den = nullptr; A.nb = w.nb;
  A.tile_ctr = w.ctr; A.done_ctr = w.ctr + 1; A.tile_part = w.tile_part; A.stop = w.stop;
  A.nsplit = 1; A.psplit = k; A.part = w.part; A.arrive = w.arrive;
  A.iters_done = iters_done; A.rel_change = rel_change; A.tol = tol; A.status = status;

  const int sms = num_sms();
  const int nb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)sms * 8);
  SSM_TRY_CUDA(cudaMemsetAsync(w.ctr, 0, 2 * sizeof(unsigned), s));
  SSM_TRY_CUDA(cudaMemsetAsync(w.stop, 0, sizeof(int32_t), s));
  SSM_TRY_CUDA(cudaMemsetAsync(iters_done, 0, sizeof(int32_t), s));
  SSM_TRY_CUDA(cudaMemsetAsync(rel_change, 0, sizeof(double), s));

  const void *kern;
  size_t smem;
  int64_t tiles;
  unsigned meta[3] = {0, 0, 0};
  bool tsm = true;
  if (precision == 64) {
    const size_t piv = (size_t)k * sizeof(PivD), tab = (size_t)cnt_len * sizeof(double);
    tsm = piv + tab <= kSmemBudget;
    smem = piv + (tsm ? tab : 0);
    kern = tsm ? (const void *)k_sweep_f64<true> : (const void *)k_sweep_f64<false>;
    tiles = (n + 31) / 32;
  } else {
    // the largest distance decides between the full (w, w d) table and the
    // clamped s table; the row lengths decide the neighbour-kernel grid
    // (from the caller's hints when given; otherwise read back once)
    SSM_TRY_CUDA(cudaMemsetAsync(w.meta, 0, 4 * sizeof(unsigned), s));
    note_launch(), k_nbr_classify<<<nb, 256, 0, s>>>(n, rowptr, w.meta + 1, w.mid_rows, w.long_rows);
    if (hints) {
      if (hints[0] < 0 || hints[0] > 65534 || hints[1] < 0 || hints[2] < 0 || hints[1] + hints[2] > n)
        return fail(SSM_E_ARG, "ssm_iterate: bad hints");
      for (int q = 0; q < 3; ++q) meta[q] = (unsigned)hints[q];
    } else {
      const int64_t kn = (int64_t)k * n;
      note_launch(), k_dip_max<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((kn + 255) / 256, sms * 8)), 256, 0,
                                 s>>>(kn, dip, w.meta);
      SSM_TRY_CUDA(cudaMemcpyAsync(meta, w.meta, 3 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
      SSM_TRY_CUDA(cudaStreamSynchronize(s));
    }
    const unsigned dmax = meta[0];
    const bool full = (size_t)k * ((size_t)dmax + 1) <= (size_t)kFullPlane;
    A.dmax = (int32_t)dmax;
    A.wtab = w.wtab;
    A.den = w.den;
    {
      const int64_t npairs = ((int64_t)n + kTileNodes - 1) / kTileNodes * (kTileNodes / 2);
      const int gy = std::min(k, 16);
      const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((npairs + 255) / 256, (int64_t)sms * 8 / gy + 1));
      const int32_t pair_loads = (n % 8 == 0 && (reinterpret_cast<uintptr_t>(dip) & 15u) == 0)  ? 2
                                 : (n % 2 == 0 && (reinterpret_cast<uintptr_t>(dip) & 3u) == 0) ? 1
                                                                                                 : 0;
      note_launch(), k_tile_dip<<<dim3(gx, gy), 256, 0, s>>>(n, k, full ? (int32_t)dmax + 1 : 0, dip, w.dtile, status,
                                                           pair_loads);
    }
    if (full) {
      note_launch(), k_build_wtab<<<std::max(1, std::min(sms * 4, (int)(((int64_t)k * (dmax + 1) + 255) / 256))), 256, 0,
                                    s>>>(k, (int32_t)dmax, cnt_off, cnt, w.wtab);
      note_launch(), k_sweep_den<<<std::max(1, (int)std::min<int64_t>(((int64_t)n + 511) / 512, sms * 8)), 256, 0, s>>>(
          n, k, w.dtile, w.wtab, rowptr, w.den);
    } else {
      note_launch(), k_build_stab<<<std::min(k, sms * 4), 128, 0, s>>>(k, cnt_off, cnt, w.stab);
    }
    const size_t piv = (size_t)k * (sizeof(float4) + sizeof(uint2));
    if (full) {
      smem = piv;  // the table planes are static shared memory
      kern = (const void *)k_sweep_f32<kFull>;
    } else {
      const size_t tab = (size_t)(2 * cnt_len + k) * sizeof(float);
      tsm = piv + tab <= kSmemBudget;
      smem = piv + (tsm ? tab : 0);
      kern = tsm ? (const void *)k_sweep_f32<kClampSmem> : (const void *)k_sweep_f32<kClampGlobal>;
    }
    tiles = (n + kTileNodes - 1) / kTileNodes;
  }
  SSM_TRY_CUDA(allow_dynamic_smem(kern));
  int per_sm = 0;
  SSM_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSweepThreads, smem));
  if (per_sm < 1) return fail(SSM_E_ARG, "ssm_iterate: %zu bytes of shared memory do not fit", smem);
  // one warp per tile, or up to kSplitTasksPerWarp warps per tile on graphs
  // small enough to split (their pivot ranges keep the extra warps busy)
  const int64_t per_tile = (precision == 32 && w.split_cap > 0 && kSplitTasksPerWarp > 0) ? kSplitTasksPerWarp : 1;
  const int64_t want = (tiles * per_tile + (kSweepThreads / 32) - 1) / (kSweepThreads / 32);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, want));
  if (precision == 32 && w.split_cap > 0 && kSplitTasksPerWarp > 0) {
    // about kSplitTasksPerWarp tasks per resident warp, ranges of at least 2 kPrefetch pivots
    const int64_t warps = (int64_t)blocks * (kSweepThreads / 32);
    int64_t S = tiles >= 2 * warps ? 1 : (kSplitTasksPerWarp * warps + tiles - 1) / tiles;
    S = std::min<int64_t>({S, (int64_t)kMaxSplit, std::max<int64_t>(1, k / (2 * kPrefetch)), w.split_cap / tiles});
    if (S > 1) {
      A.psplit = (int32_t)((k + S - 1) / S);
      A.nsplit = (int32_t)((k + A.psplit - 1) / A.psplit);
      SSM_TRY_CUDA(cudaMemsetAsync(w.arrive, 0, (size_t)tiles * sizeof(unsigned), s));
    }
  }

  g_last_config[0] = precision == 64 ? (tsm ? 3 : 4) : (kern == (const void *)k_sweep_f32<kFull> ? 2 : (tsm ? 0 : 1));
  g_last_config[1] = A.nsplit;
  g_last_config[2] = blocks;
  g_last_config[3] = precision == 64 ? -1 : (int32_t)meta[0];
  const int32_t nmid = (int32_t)meta[1], nlong = (int32_t)meta[2];
  const unsigned nbr_blocks = (unsigned)(nlong + (nmid + 7) / 8 + (n + 255) / 256);
  for (int t = 0; t < iters; ++t) {
    const bool even = (t & 1) == 0;
    void *pin = even ? pos : w.tmp, *pout = even ? w.tmp : pos;
    if (precision == 32) {
      // both kernels of an iteration are launched as programmatic dependents of
      // the kernel before them (each waits in wait_previous_kernel)
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(nbr_blocks);
      cfg.blockDim = dim3(256);
      cfg.stream = s;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      note_launch();
      SSM_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_sweep_nbr, n, rowptr, colidx, (const float2 *)pin, nlong,
                                      (const int32_t *)w.long_rows, nmid, (const int32_t *)w.mid_rows, w.nb,
                                      (const int32_t *)w.stop));
      cfg.gridDim = dim3(blocks);
      cfg.blockDim = dim3(kSweepThreads);
      cfg.dynamicSmemBytes = smem;
      void *args[] = {&A, &pin, &pout};
      note_launch();
      SSM_TRY_CUDA(cudaLaunchKernelExC(&cfg, kern, args));
      continue;
    }
    void *args[] = {&A, &pin, &pout};
    note_launch();
    SSM_TRY_CUDA(cudaLaunchKernel(kern, dim3(blocks), dim3(kSweepThreads), args, smem, s));
  }
  const int cb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)sms * 8);
  if (precision == 64)
    note_launch(), k_copy_back_if_odd<double2><<<cb, 256, 0, s>>>(n, iters_done, (const double2 *)w.tmp, (double2 *)pos);
  else
    note_launch(), k_copy_back_if_odd<float2><<<cb, 256, 0, s>>>(n, iters_done, (const float2 *)w.tmp, (float2 *)pos);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

SSM_API int ssm_iterate_hints(int32_t n, const int32_t *rowptr, int32_t k, const uint16_t *dip, int32_t *hints,
                              void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || k < 1 || !rowptr || !dip || !hints || !ws) return fail(SSM_E_ARG, "ssm_iterate_hints: bad argument");
  if (ws_bytes < 256) return fail(SSM_E_NOMEM, "ssm_iterate_hints: workspace %zu bytes, need 256", ws_bytes);
  unsigned *meta = (unsigned *)ws;
  const int sms = num_sms();
  SSM_TRY_CUDA(cudaMemsetAsync(meta, 0, 4 * sizeof(unsigned), s));
  const int64_t kn = (int64_t)k * n;
  note_launch(), k_dip_max<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((kn + 255) / 256, sms * 8)), 256, 0, s>>>(
      kn, dip, meta);
  note_launch(), k_row_classes<<<(int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)sms * 8), 256, 0, s>>>(
      n, rowptr, meta + 1);
  unsigned h[3] = {0, 0, 0};
  SSM_TRY_CUDA(cudaMemcpyAsync(h, meta, 3 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  SSM_TRY_CUDA(cudaStreamSynchronize(s));
  for (int q = 0; q < 3; ++q) hints[q] = (int32_t)h[q];
  return SSM_OK;
}

SSM_API void ssm_last_sweep_config(int32_t *out) {
  for (int i = 0; i < 4; ++i) out[i] = ssm::g_last_config[i];
}
