// The Gram matrix of PivotMDS on the 5th-generation tensor cores.
//
// PivotMDS (Algorithm 1 line 3, after Brandes & Pich) needs C^T C for the
// n x k matrix C of double-centred squared distances; the centring is
// applied afterwards on the k x k level, so the dense contraction is the
// integer Gram matrix G[a][b] = sum_i d_ia^2 d_ib^2, wanted exactly (it feeds
// an FP64 eigen-solve that must match the oracle to 1e-10).
//
// Exactness on FP16 tensor cores: every squared distance (below 2^32) is cut
// into D digits of 5 bits, s = sum_p 2^(5p) s_p with 0 <= s_p <= 31, so
//   G = sum_{p,q} 2^(5(p+q)) S_p^T S_q.
// A digit is exact in FP16, a digit product is at most 961, and an
// accumulator is read out after at most kTcFlush chunks of 64 nodes (16384
// nodes), so it holds an integer below 961 * 16384 < 2^24 -- exact in FP32.
// D = ceil(bits(max d^2) / 5) comes from the largest distance on the device
// (2 digits for small-world graphs, 4 for d <= 1023).  When every squared
// distance is below 2^7 (d <= 11) one 7-bit digit does instead: FP16 holds it
// exactly, a product is at most 127^2, and an accumulator read out every
// 2^18 / s_max^2 chunks (at least kTcFlush7: 1024 nodes) stays below 2^24;
// those read-outs add into 64-bit sums in shared memory (one per tile
// entry), and only the slice's totals go to G.
//
// Work units are (output tile, digit block, chunk of 64 nodes): a 128 x 128
// tile of pivots a (tile ta) by pivots b (tile tb >= ta, by symmetry), a
// block of up to two A digits by up to two B digits (up to four digit pairs,
// one TMEM accumulator of 128 columns each, 512 columns), 64 nodes.  The
// units are laid out tile-block-major and cut into one contiguous slice per
// CTA (one CTA per SM), so every SM gets the same number of chunks.  Per
// chunk each warp loads eight pivot rows of both tiles with coalesced loads (a
// lane takes two consecutive nodes; the next chunk's rows are loaded while
// this one is converted), cuts them into digits and writes the digit planes
// into shared memory in the 128-byte-swizzled K-major layout (a row of 64
// nodes is 128 bytes, its 16-byte chunks permuted by the row index, so the
// 32 lanes hit 32 banks).  One thread issues the tcgen05.mma of every pair
// (M = N = 128, K = 16, FP16 in, FP32 accumulate) and commits them to the
// mbarrier of the buffer; the planes are double-buffered, so the warps build
// chunk c + 1 while the tensor cores work on chunk c.  When the slice moves to
// another tile or digit block, after kTcFlush chunks, and at its end, the CTA
// drains the MMAs and every warp reads 32 TMEM lanes of every accumulator
// (tcgen05.ld), weighs each pair by 2^(5(p+q)), adds the pairs in 128-bit
// integers and adds them into the 128-bit G with atomics (order-free, exact).
// All waits are bounded (SSM_E_TIMEOUT).
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "gram_tc.cuh"

namespace ssm {

constexpr int kTcThreads = 512;        // 16 warps, 8 pivot rows of each tile per warp
constexpr int kTcChunk = 64;           // nodes per plane row (128 bytes of FP16, 4 MMAs of K = 16)
constexpr int kTcFlush = 256;          // chunks per accumulator read-out (16384 nodes: below 2^24)
constexpr int kTcFlush7 = 16;          // the same with one 7-bit digit, at its largest (127^2 1024 < 2^24)
static_assert((1 << 18) / (127 * 127) >= kTcFlush7, "one-digit read-out period");
constexpr unsigned kTcAccBytes = 128u * 128u * 8u;  // 64-bit sums of one tile (single-digit mode)
constexpr int kTcDigBits = 5;          // digit width
constexpr int kTcDigBlock = 2;         // digits per A block and per B block
constexpr unsigned kTcPlaneBytes = 128u * kTcChunk * 2u;              // 128 pivots x 64 nodes, FP16
constexpr unsigned kTcBufBytes = 2u * kTcDigBlock * kTcPlaneBytes;    // A and B digit planes of one chunk
constexpr unsigned long long kTcWaitNs = 200000000ull;                // 200 ms

__device__ __forceinline__ uint32_t tc_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle (8 rows x 128
// bytes per atom, 1024 bytes between atoms along M), version 1
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024u >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: FP16 A and B (K-major), FP32 accumulator, M = N = 128
constexpr uint32_t kTcIdesc = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool tc_try(uint32_t mbar, unsigned phase) {
  unsigned done = 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(mbar), "r"(phase)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, unsigned phase) {
  if (tc_try(mbar, phase)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (tc_try(mbar, phase)) return true;
    if (globaltimer_ns() - t0 > kTcWaitNs) return false;
  }
}

// FP16 pair of digit p (bits 5p .. 5p + 4) of two squared distances s0, s1
// (exact: (1024 + v) - 1024).  L packs bits 0..15 of both, M bits 15..30.
// With mask 0x007F007F and p = 0 it is the single 7-bit digit.
__device__ __forceinline__ uint32_t tc_digits(uint32_t s0, uint32_t s1, uint32_t L, uint32_t M, int p,
                                              uint32_t mask = 0x001F001Fu) {
  uint32_t w;
  if (p < 3)
    w = (L >> (kTcDigBits * p)) & mask;
  else if (p < 6)
    w = (M >> (kTcDigBits * (p - 3))) & 0x001F001Fu;
  else
    w = __byte_perm(s0 >> 30, s1 >> 30, 0x5410);
  w |= 0x64006400u;
  const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&w), __half2half2(__ushort_as_half(0x6400)));
  return *reinterpret_cast<const uint32_t *>(&h);
}

// single-digit mode: the FP16 pair (d0^2, d1^2) of two distances below 2^5
// packed in 16-bit halves (1024 + d is exact in FP16, and so are its
// difference with 1024 and that difference squared)
__device__ __forceinline__ uint32_t tc_square_pair(uint32_t dd) {
  uint32_t w = dd | 0x64006400u;
  const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&w), __half2half2(__ushort_as_half(0x6400)));
  const __half2 q = __hmul2(h, h);
  return *reinterpret_cast<const uint32_t *>(&q);
}

// distances of nodes i, i + 1 of one pivot row packed in 16-bit halves (zero
// past n and for rows past k)
__device__ __forceinline__ uint32_t tc_load_pair(const uint16_t *__restrict__ dip, int32_t n, int row, int32_t k,
                                                 int i, bool wide) {
  if (row >= k || i >= n) return 0u;
  const uint16_t *p = dip + (size_t)row * n + i;
  if (wide) return __ldg(reinterpret_cast<const unsigned *>(p));
  const uint32_t d0 = __ldg(p);
  const uint32_t d1 = (i + 1 < n) ? (uint32_t)__ldg(p + 1) : 0u;
  return d0 | (d1 << 16);
}

struct TcUnit {
  int ta, tb, pa0, qb0, npa, nqb;
};

__device__ __forceinline__ TcUnit tc_unit(int tg, int groups, int nblk, int T, int D) {
  TcUnit U;
  int t = tg / groups;
  const int grp = tg - t * groups;
  int ta = 0;
  while (t >= T - ta) { t -= T - ta; ++ta; }
  U.ta = ta;
  U.tb = ta + t;
  U.pa0 = kTcDigBlock * (grp / nblk);
  U.qb0 = kTcDigBlock * (grp % nblk);
  U.npa = min(kTcDigBlock, D - U.pa0);
  U.nqb = min(kTcDigBlock, D - U.qb0);
  return U;
}

// read every accumulator of unit U out of TMEM and add it into G (all threads)
__device__ __forceinline__ void tc_flush(const TcUnit &U, uint32_t tmem, int32_t k, int warp, int lane,
                                         unsigned long long *__restrict__ Glo, unsigned long long *__restrict__ Ghi) {
  // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (tile rows) and the 32
  // columns 32 (w div 4) .. + 31 of every accumulator, 8 at a time
  const int q4 = warp & 3;
  const int a = 128 * U.ta + 32 * q4 + lane;
  const int np = U.npa * U.nqb;
#pragma unroll 1
  for (int part = 0; part < 4; ++part) {
    const int cb = 32 * (warp >> 2) + 8 * part;
    unsigned long long lo[8], hi[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) lo[e] = hi[e] = 0ull;
    for (int j = 0; j < np; ++j) {
      const int ja = j / U.nqb, jb = j - ja * U.nqb;
      uint32_t v[8];
      const uint32_t taddr =
          tmem + ((uint32_t)(32 * q4) << 16) + 128u * (unsigned)(ja * kTcDigBlock + jb) + (unsigned)cb;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      const int sh = kTcDigBits * (U.pa0 + ja + U.qb0 + jb);  // at most 60
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const unsigned long long x = (unsigned long long)__uint_as_float(v[e]);
        const unsigned long long xl = x << sh;
        const unsigned long long xh = sh == 0 ? 0ull : x >> (64 - sh);
        const unsigned long long old = lo[e];
        lo[e] += xl;
        hi[e] += xh + (lo[e] < old ? 1ull : 0ull);
      }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int b = 128 * U.tb + cb + e;
      if (a >= k || b >= k || a > b || (lo[e] | hi[e]) == 0ull) continue;
      const size_t o = (size_t)a * k + b;
      const unsigned long long old = atomicAdd(Glo + o, lo[e]);
      const unsigned long long carry = (old + lo[e] < old) ? 1ull : 0ull;
      if (hi[e] + carry) atomicAdd(Ghi + o, hi[e] + carry);
    }
  }
}

// single-digit mode: add the one accumulator of the current unit into the
// 64-bit tile sums acc[col][row] (column-major: a warp's lanes hit
// consecutive words), each entry owned by one thread
__device__ __forceinline__ void tc_acc_tmem(uint32_t tmem, int warp, int lane, unsigned long long *acc) {
  const int q4 = warp & 3, row = 32 * q4 + lane;
#pragma unroll 1
  for (int part = 0; part < 4; ++part) {
    const int cb = 32 * (warp >> 2) + 8 * part;
    uint32_t v[8];
    const uint32_t taddr = tmem + ((uint32_t)(32 * q4) << 16) + (unsigned)cb;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[(cb + e) * 128 + row] += (unsigned long long)__uint_as_float(v[e]);
  }
}

// single-digit mode: the tile sums of unit U into G (128-bit atomics), then cleared
__device__ __forceinline__ void tc_acc_out(const TcUnit &U, int32_t k, int warp, int lane, unsigned long long *acc,
                                           unsigned long long *__restrict__ Glo,
                                           unsigned long long *__restrict__ Ghi) {
  const int q4 = warp & 3, row = 32 * q4 + lane;
  const int a = 128 * U.ta + row;
  for (int c = 0; c < 32; ++c) {
    const int col = 32 * (warp >> 2) + c;
    const int b = 128 * U.tb + col;
    unsigned long long &x = acc[col * 128 + row];
    if (a < k && b < k && a <= b && x != 0ull) {
      const size_t o = (size_t)a * k + b;
      const unsigned long long old = atomicAdd(Glo + o, x);
      if (old + x < old) atomicAdd(Ghi + o, 1ull);
    }
    x = 0ull;
  }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(int32_t n, int32_t k, const uint16_t *__restrict__ dip,
                                                           int32_t wide, const unsigned *__restrict__ dmax,
                                                           unsigned long long *__restrict__ Glo,
                                                           unsigned long long *__restrict__ Ghi,
                                                           int32_t *__restrict__ status) {
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) uint64_t s_mbar[2];
  __shared__ uint32_t s_tmem;

  // digits of the largest squared distance, digit blocks, this CTA's slice
  const unsigned dm = *dmax;
  const unsigned long long s_max = (unsigned long long)dm * dm;
  int bits = 1;
  while (bits < 64 && (s_max >> bits) != 0ull) ++bits;
  const bool one = s_max < 128ull;  // single 7-bit digit
  const int D = one ? 1 : (bits + kTcDigBits - 1) / kTcDigBits;
  // read-out period: with one digit every partial sum stays below
  // 64 chunks s_max^2 <= 2^24 (at least kTcFlush7 chunks for s_max <= 127)
  const int flush = one ? (int)min((unsigned long long)kTcFlush, (1ull << 18) / max(1ull, s_max * s_max)) : kTcFlush;
  const uint32_t dmask = one ? 0x007F007Fu : 0x001F001Fu;
  const int ppo = one ? 1 : kTcDigBlock;  // planes per operand in a buffer
  const unsigned buf_bytes = 2u * (unsigned)ppo * kTcPlaneBytes;
  const int nblk = (D + kTcDigBlock - 1) / kTcDigBlock;
  const int groups = nblk * nblk;
  const int T = (k + 127) / 128;
  const int nch = (n + kTcChunk - 1) / kTcChunk;
  const int64_t W = (int64_t)(T * (T + 1) / 2) * groups * nch;
  const int64_t per = (W + gridDim.x - 1) / gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * per, end = min(W, beg + per);
  if (beg >= end) return;  // uniform: the whole CTA leaves before any TMEM use
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool wide4 = wide != 0;

  // planes (1024-byte aligned for the swizzle): buffer u at base + u buf_bytes,
  // A digit slot j at + j planes, B digit slot j at + (ppo + j) planes
  const uint32_t base = (tc_smem(tc_raw) + 1023u) & ~1023u;
  unsigned char *const gbase = tc_raw + (base - tc_smem(tc_raw));
  // single-digit mode: the tile sums after the two (smaller) buffers
  unsigned long long *const acc = reinterpret_cast<unsigned long long *>(gbase + 2u * buf_bytes);
  if (one)
    for (unsigned t = tid; t < 128u * 128u; t += blockDim.x) acc[t] = 0ull;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(tc_smem(&s_tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&s_mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&s_mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = s_tmem;
  const uint32_t mbar0 = tc_smem(&s_mbar[0]), mbar1 = tc_smem(&s_mbar[1]);

  // this warp's pivot rows are m = 8 warp + r (r < 8) of both tiles, this
  // lane's nodes 2 lane, 2 lane + 1 of the chunk
  uint32_t ca[8], cb[8];  // distances of the chunk being converted
  // (tile-block, chunk) of the current unit, advanced without divisions
  int tg = (int)(beg / nch), ch = (int)(beg - (int64_t)tg * nch);
  {
    const TcUnit U = tc_unit(tg, groups, nblk, T, D);
    const int i = kTcChunk * ch + 2 * lane;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      ca[r] = tc_load_pair(dip, n, 128 * U.ta + 8 * warp + r, k, i, wide4);
      cb[r] = U.ta == U.tb ? 0u : tc_load_pair(dip, n, 128 * U.tb + 8 * warp + r, k, i, wide4);
    }
  }

  bool ok = true;
  int it = 0;        // chunks issued by this CTA (buffer it & 1, its (it >> 1)-th commit)
  int since = 0;     // chunks accumulated since the last read-out
  int cur_tg = -1;
  TcUnit U{};
  for (int64_t idx = beg; idx < end; ++idx, ++it) {
    if (cur_tg >= 0 && (tg != cur_tg || since == flush)) {
      // drain the MMAs, then read the accumulators out
      const bool drained = tc_wait((it - 1) & 1 ? mbar1 : mbar0, (unsigned)((it - 1) >> 1) & 1u);
      if (!__syncthreads_and(drained ? 1 : 0)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (one) {
        tc_acc_tmem(tmem, warp, lane, acc);
        if (tg != cur_tg) tc_acc_out(U, k, warp, lane, acc, Glo, Ghi);  // each thread its own entries
      } else {
        tc_flush(U, tmem, k, warp, lane, Glo, Ghi);
      }
      since = 0;
    }
    if (tg != cur_tg) {
      cur_tg = tg;
      U = tc_unit(tg, groups, nblk, T, D);
    }
    const bool diag = U.ta == U.tb;
    // on a diagonal tile with equal digit blocks the B planes are the A planes
    const bool share = diag && U.pa0 == U.qb0;
    const bool needM = U.pa0 + U.npa > 3 || U.qb0 + U.nqb > 3;
    const int u = it & 1;
    const uint32_t mb = u ? mbar1 : mbar0;
    // buffer u is free again once the MMAs of chunk it - 2 are done (the
    // verdict is made uniform at the barrier below)
    const bool freed = it < 2 || tc_wait(mb, (unsigned)((it - 2) >> 1) & 1u);
    unsigned char *const buf = gbase + u * buf_bytes;
    if (one) {
      // one digit: the planes hold the FP16 squares themselves
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const unsigned off = (unsigned)warp * 1024u + (unsigned)r * 128u + ((unsigned)((lane >> 2) ^ r) << 4) +
                             ((unsigned)(lane & 3) << 2);
        *reinterpret_cast<uint32_t *>(buf + off) = tc_square_pair(ca[r]);
        if (!share) *reinterpret_cast<uint32_t *>(buf + kTcPlaneBytes + off) = tc_square_pair(cb[r]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const uint32_t da = ca[r];
        const uint32_t a0 = (da & 0xFFFFu) * (da & 0xFFFFu), a1 = (da >> 16) * (da >> 16);
        const uint32_t La = __byte_perm(a0, a1, 0x5410), Ma = needM ? __byte_perm(a0 >> 15, a1 >> 15, 0x5410) : 0u;
        // row m = 8 warp + r: atom m / 8 = warp, row m mod 8 = r; 16-byte chunk
        // lane / 4 swizzled by r, bytes 4 (lane mod 4) in it
        const unsigned off = (unsigned)warp * 1024u + (unsigned)r * 128u + ((unsigned)((lane >> 2) ^ r) << 4) +
                             ((unsigned)(lane & 3) << 2);
#pragma unroll
        for (int j = 0; j < kTcDigBlock; ++j)
          if (j < U.npa)
            *reinterpret_cast<uint32_t *>(buf + j * kTcPlaneBytes + off) =
                tc_digits(a0, a1, La, Ma, U.pa0 + j, dmask);
        if (!share) {
          uint32_t b0 = a0, b1 = a1, Lb = La, Mb = Ma;
          if (!diag) {
            const uint32_t db = cb[r];
            b0 = (db & 0xFFFFu) * (db & 0xFFFFu);
            b1 = (db >> 16) * (db >> 16);
            Lb = __byte_perm(b0, b1, 0x5410);
            Mb = needM ? __byte_perm(b0 >> 15, b1 >> 15, 0x5410) : 0u;
          }
#pragma unroll
          for (int j = 0; j < kTcDigBlock; ++j)
            if (j < U.nqb)
              *reinterpret_cast<uint32_t *>(buf + (ppo + j) * kTcPlaneBytes + off) =
                  tc_digits(b0, b1, Lb, Mb, U.qb0 + j, dmask);
        }
      }
    }
    // the next chunk's distances, in flight while the MMAs are issued
    int tg1 = tg, ch1 = ch + 1;
    if (ch1 == nch) {
      ch1 = 0;
      ++tg1;
    }
    if (idx + 1 < end) {
      const TcUnit U1 = tg1 == tg ? U : tc_unit(tg1, groups, nblk, T, D);
      const int i = kTcChunk * ch1 + 2 * lane;
      const int ra = 128 * U1.ta + 8 * warp, rb = 128 * U1.tb + 8 * warp;
      if (wide4 && kTcChunk * (ch1 + 1) <= n) {
        // the chunk lies inside the rows: 4-byte loads one row (n / 2 words) apart
        const unsigned *pa = reinterpret_cast<const unsigned *>(dip) + ((size_t)ra * n + i) / 2;
        const unsigned *pb = reinterpret_cast<const unsigned *>(dip) + ((size_t)rb * n + i) / 2;
        const size_t row = (size_t)n / 2;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          ca[r] = ra + r < k ? __ldg(pa + r * row) : 0u;
          cb[r] = (U1.ta != U1.tb && rb + r < k) ? __ldg(pb + r * row) : 0u;
        }
      } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          ca[r] = tc_load_pair(dip, n, ra + r, k, i, wide4);
          cb[r] = U1.ta == U1.tb ? 0u : tc_load_pair(dip, n, rb + r, k, i, wide4);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the planes are read by the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;");
    const int stuck = __syncthreads_or(freed ? 0 : 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (stuck) {
      ok = false;
      break;
    }
    if (tid == 0) {
      const uint32_t bs = base + (unsigned)u * buf_bytes;
      for (int ja = 0; ja < U.npa; ++ja)
        for (int jb = 0; jb < U.nqb; ++jb) {
          const uint32_t acc_col = tmem + 128u * (unsigned)(ja * kTcDigBlock + jb);
#pragma unroll
          for (int st = 0; st < kTcChunk / 16; ++st) {
            // K slice st: bytes 32 st of every 128-byte row (the swizzle is applied by the hardware)
            const uint64_t da = tc_desc(bs + (unsigned)ja * kTcPlaneBytes + 32u * st);
            const uint64_t db = tc_desc(bs + (unsigned)((share ? 0 : ppo) + jb) * kTcPlaneBytes + 32u * st);
            const uint32_t acc = (since > 0 || st > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_col),
                "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc));
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
    }
    ++since;
    tg = tg1;
    ch = ch1;
  }
  // the last commit covers every MMA issued before it
  const uint32_t mlast = ((it - 1) & 1) ? mbar1 : mbar0;
  const unsigned plast = (unsigned)((it - 1) >> 1) & 1u;
  if (ok && !tc_wait(mlast, plast)) ok = false;
  ok = __syncthreads_and(ok ? 1 : 0) != 0;  // uniform: the TMEM reads are warp-collective
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (one) {
      tc_acc_tmem(tmem, warp, lane, acc);
      tc_acc_out(U, k, warp, lane, acc, Glo, Ghi);
    } else {
      tc_flush(U, tmem, k, warp, lane, Glo, Ghi);
    }
  } else {
    if (tid == 0) dev_fail(status, SSM_E_TIMEOUT);
    // let whatever is still in flight finish (bounded) before the TMEM goes
    if (it > 0) tc_wait(mlast, plast);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// the larger of the two layouts: two-digit-block buffers, or single-digit
// buffers and the tile sums
size_t gram_tc_smem() { return std::max<size_t>(2u * kTcBufBytes, 2u * 2u * kTcPlaneBytes + kTcAccBytes) + 1024u; }

int launch_gram_tc(int32_t n, int32_t k, const uint16_t *dip, const unsigned *dmax, unsigned long long *Glo,
                   unsigned long long *Ghi, int32_t *status, cudaStream_t s) {
  const size_t smem = gram_tc_smem();
  // two distances per 4-byte load when every row starts on a 4-byte boundary
  const int wide = ((n & 1) == 0 && ((uintptr_t)dip & 3u) == 0) ? 1 : 0;
  SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_gram_tc));
  note_launch(), k_gram_tc<<<num_sms(), kTcThreads, smem, s>>>(n, k, dip, wide, dmax, Glo, Ghi, status);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

}  // namespace ssm
