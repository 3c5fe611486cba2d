// Full stress of a layout (Eq. 1, w_ij = d_ij^-2) with the optimal scale
// (Section 4: every drawing is rescaled to its lowest stress before it is
// reported), exhaustive over all pairs or over sampled pairs.
//
// Pair distances come from the multi-source bitset BFS (bfs.cu) run from a
// batch of sources into a [sources][n] uint16 table, or, for sampled pairs on
// graphs the pulled BFS handles, straight from the level bits of each pass
// (the distance of (s, v) is the level at which bit s of v first appears, so
// the full table is never written); a pair kernel then accumulates, in FP64
// and in a fixed order,
//   sum (r/d - 1)^2 = sum (r-d)^2/d^2,  S1 = sum r/d,  S2 = sum r^2/d^2,  N,
// and the final kernel forms {raw, alpha* = S1/S2, N - S1^2/S2, normalized}.
#include <algorithm>

#include "bfs.cuh"
#include "weighted.cuh"

namespace ssm {

constexpr int kPairThreads = 256;
constexpr int kExhaustiveBatch = 1024;  // sources per BFS batch (32 bitset words)

__global__ void k_sample_sources(int32_t n, int32_t S, uint64_t seed, int32_t *__restrict__ src) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S; j += gridDim.x * blockDim.x)
    src[j] = (int32_t)(((splitmix64_at(seed, (uint64_t)j) >> 32) * (uint64_t)n) >> 32);
}

__global__ void k_batch_sources(int32_t base, int32_t B, int32_t *__restrict__ src) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < B; j += gridDim.x * blockDim.x) src[j] = base + j;
}

// a pair distance that cannot be used: unreachable (or the same node)
__device__ __forceinline__ bool bad_dist(uint16_t d) { return d == 0xFFFFu || d == 0u; }
__device__ __forceinline__ bool bad_dist(float d) { return !(d > 0.0f) || isinf(d); }

template <class T2, class D>
__device__ __forceinline__ void pair_terms(const T2 *__restrict__ pos, int i, int j, D d, double (&acc)[4]) {
  const T2 a = pos[i], b = pos[j];
  const double dx = (double)a.x - (double)b.x, dy = (double)a.y - (double)b.y;
  const double r = sqrt(dx * dx + dy * dy);
  const double t = r / (double)d;
  acc[0] += (t - 1.0) * (t - 1.0);
  acc[1] += t;
  acc[2] += t * t;
  acc[3] += 1.0;
}

__device__ __forceinline__ void block_store_sums(double (&acc)[4], double *__restrict__ part) {
  __shared__ double red[kPairThreads / 32][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[threadIdx.x >> 5][q] = acc[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < kPairThreads / 32; ++w) t += red[w][threadIdx.x];
    part[4 * (size_t)blockIdx.x + threadIdx.x] = t;
  }
}

// exhaustive batch: sources base..base+B-1, pairs (base+a, v) with v > base+a
template <class T2, class D>
__global__ void __launch_bounds__(kPairThreads) k_pairs_exhaustive(int32_t n, int32_t base, int32_t B,
                                                                    const D *__restrict__ dist,
                                                                    const T2 *__restrict__ pos,
                                                                    double *__restrict__ part,
                                                                    int32_t *__restrict__ status) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t total = (int64_t)B * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / n), v = (int)(t - (int64_t)a * n);
    const int i = base + a;
    if (v <= i) continue;
    const D d = __ldg(dist + t);
    if (bad_dist(d)) {
      dev_fail(status, SSM_E_DISCONNECTED);
      continue;
    }
    pair_terms(pos, i, v, d, acc);
  }
  block_store_sums(acc, part);
}

// sampled pair t = j T + l: source src[j], target from splitmix64 draw S + t
// (uniform over the other n - 1 nodes)
__device__ __forceinline__ int sampled_target(int32_t n, int32_t S, uint64_t seed, int64_t t, int s) {
  const uint64_t u = splitmix64_at(seed, (uint64_t)S + (uint64_t)t);
  const int v = (int)(((u >> 32) * (uint64_t)(n - 1)) >> 32);
  return v + ((v >= s) ? 1 : 0);
}

// sampled: source j (src[j]), targets l = 0..T-1 from the splitmix64 stream;
// with run_if, only if *run_if != 0 (the pulled BFS gave up and the table was
// written instead)
template <class T2, class D>
__global__ void __launch_bounds__(kPairThreads) k_pairs_sampled(int32_t n, int32_t S, int32_t T, uint64_t seed,
                                                                 const int32_t *__restrict__ src,
                                                                 const D *__restrict__ dist,
                                                                 const T2 *__restrict__ pos,
                                                                 double *__restrict__ part,
                                                                 int32_t *__restrict__ status,
                                                                 const unsigned *__restrict__ run_if) {
  if (run_if && __ldcg(run_if) == 0u) return;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t total = (int64_t)S * T;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / T);
    const int s = __ldg(src + j);
    const int v = sampled_target(n, S, seed, t, s);
    const D d = __ldg(dist + (size_t)j * n + v);
    if (bad_dist(d)) {
      dev_fail(status, SSM_E_DISCONNECTED);
      continue;
    }
    pair_terms(pos, s, v, d, acc);
  }
  block_store_sums(acc, part);
}

// sampled pairs of the sources of one pulled-BFS pass (j = base .. base +
// nsrc - 1), their distances read from the pass's level bits: d(s, v) = the
// level L whose word holds bit j - base for node v; partial sums per block
template <class T2>
__global__ void __launch_bounds__(kPairThreads) k_pairs_from_levels(int32_t n, int32_t S, int32_t T, uint64_t seed,
                                                                     const int32_t *__restrict__ src, PullPass P,
                                                                     const T2 *__restrict__ pos,
                                                                     double *__restrict__ part,
                                                                     int32_t *__restrict__ status) {
  if (__ldcg(P.gaveup)) return;  // the table path takes over
  const unsigned nlev = min(__ldcg(P.nlev), kPullPassLevels);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t total = (int64_t)P.nsrc * T;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / T);
    const int j = P.base + a;
    const int s = __ldg(src + j);
    const int v = sampled_target(n, S, seed, (int64_t)j * T + (t - (int64_t)a * T), s);
    const unsigned bit = 1u << (a & 31);
    const unsigned *f = P.F + (size_t)v * kPullPassWords + (a >> 5);
    unsigned d = 0xFFFFu;
    for (unsigned L = 0; L < nlev; ++L)
      if (__ldcg(f + (size_t)L * n * kPullPassWords) & bit) {
        d = L;
        break;
      }
    if (bad_dist((uint16_t)d)) {
      dev_fail(status, SSM_E_DISCONNECTED);
      continue;
    }
    pair_terms(pos, s, v, (uint16_t)d, acc);
  }
  block_store_sums(acc, part);
}

// fixed-order sum of all block partials, then the stress values; with
// use_alt, the partials part_alt[0 .. nparts_alt) instead when *use_alt == 0
// (the pulled BFS completed and its passes summed the pairs)
__global__ void k_stress_final(int32_t n, int64_t nparts, const double *__restrict__ part, int sampled,
                               double *__restrict__ out, double *__restrict__ sums,
                               const double *__restrict__ part_alt = nullptr, int64_t nparts_alt = 0,
                               const unsigned *__restrict__ use_alt = nullptr) {
  __shared__ double red[32][4];
  if (use_alt && __ldcg(use_alt) == 0u) {
    part = part_alt;
    nparts = nparts_alt;
  }
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t b = threadIdx.x; b < nparts; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += part[4 * b + q];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[threadIdx.x >> 5][q] = acc[q];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int w = 0; w < (int)blockDim.x / 32; ++w)
    for (int q = 0; q < 4; ++q) s[q] += red[w][q];
  const double pairs = 0.5 * (double)n * (double)(n - 1);
  const double f = sampled ? pairs / s[3] : 1.0;
  if (sums)
    for (int q = 0; q < 4; ++q) sums[q] = s[q];
  out[0] = s[0] * f;
  out[1] = s[2] > 0.0 ? s[1] / s[2] : 0.0;
  out[2] = (s[2] > 0.0 ? s[3] - s[1] * s[1] / s[2] : s[3]) * f;
  out[3] = out[2] / pairs;
}

static int pair_blocks() { return num_sms() * 8; }

struct StressWs {
  int32_t *src;
  uint16_t *dist;
  double *part;
  double *part_pull;  // [passes][pair blocks][4] sampled sums from the pulled BFS's level bits
  void *bfs;
  size_t bfs_bytes;
};

static size_t carve_stress(Carver &c, StressWs &w, int32_t n, int64_t m2, int32_t S, int32_t nbatches) {
  w.src = c.take<int32_t>(S);
  w.dist = c.take<uint16_t>((size_t)S * n);
  w.part = c.take<double>(4 * (size_t)pair_blocks() * (size_t)nbatches);
  w.part_pull = c.take<double>(4 * (size_t)pair_blocks() * (size_t)((S + kPullPassSources - 1) / kPullPassSources));
  w.bfs_bytes = msbfs_workspace(n, m2, S);
  w.bfs = c.take<char>(w.bfs_bytes);
  return c.size();
}

static void stress_shape(int32_t n, int32_t nsources, int32_t *S, int32_t *nbatches) {
  if (nsources > 0) {
    *S = nsources;
    *nbatches = 1;
  } else {
    *S = std::min<int32_t>(n, kExhaustiveBatch);
    *nbatches = (n + *S - 1) / *S;
  }
}

}  // namespace ssm

SSM_API size_t ssm_stress_workspace(int32_t n, int64_t m, int32_t nsources, int32_t ntargets) {
  (void)ntargets;
  if (n < 2 || m < 0 || nsources < 0) return 0;
  int32_t S, nb;
  ssm::stress_shape(n, nsources, &S, &nb);
  ssm::Carver c(nullptr, 0);
  ssm::StressWs w;
  return ssm::carve_stress(c, w, n, 2 * m, S, nb);
}

SSM_API int ssm_stress(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, const void *pos,
                       int32_t precision,
                       int32_t nsources, int32_t ntargets, uint64_t seed, double *out, double *sums, int32_t *status,
                       void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 2 || m < 0 || !rowptr || !colidx || !pos || !out || !status || !ws)
    return fail(SSM_E_ARG, "ssm_stress: null pointer or bad size");
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_stress: precision must be 32 or 64");
  if (nsources < 0 || nsources > 65535 || (nsources > 0 && ntargets < 1))
    return fail(SSM_E_ARG, "ssm_stress: need 0 <= nsources <= 65535 and ntargets >= 1 when sampling");
  int32_t S, nb;
  stress_shape(n, nsources, &S, &nb);
  if ((int64_t)n * ((S + 31) / 32) >= ((int64_t)1 << 31)) return fail(SSM_E_ARG, "ssm_stress: n*ceil(S/32) too large");
  Carver c(ws, ws_bytes);
  StressWs w;
  carve_stress(c, w, n, 2 * m, S, nb);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_stress: workspace %zu bytes, need %zu", ws_bytes, c.size());
  const int pb = pair_blocks();
  const unsigned *gaveup = nullptr;
  int64_t npull = 0;
  if (nsources > 0) {
    note_launch(), k_sample_sources<<<std::max(1, (S + 255) / 256), 256, 0, s>>>(n, S, seed, w.src);
    // each pass of the pulled BFS sums its sources' pairs from its level bits
    const PullPassFn from_levels = [&](const PullPass &P) -> int {
      double *part = w.part_pull + 4 * (size_t)pb * (size_t)P.pass;
      npull = std::max<int64_t>(npull, (int64_t)pb * (P.pass + 1));
      if (precision == 64)
        note_launch(), k_pairs_from_levels<double2><<<pb, kPairThreads, 0, s>>>(n, S, ntargets, seed, w.src, P,
                                                                                (const double2 *)pos, part, status);
      else
        note_launch(), k_pairs_from_levels<float2><<<pb, kPairThreads, 0, s>>>(n, S, ntargets, seed, w.src, P,
                                                                               (const float2 *)pos, part, status);
      SSM_TRY_CUDA(cudaGetLastError());
      return SSM_OK;
    };
    int rc = launch_msbfs(n, 2 * m, rowptr, colidx, S, w.src, w.dist, status, w.bfs, w.bfs_bytes, s, &from_levels,
                          &gaveup);
    if (rc) return rc;
    if (precision == 64)
      note_launch(), k_pairs_sampled<double2, uint16_t><<<pb, kPairThreads, 0, s>>>(n, S, ntargets, seed, w.src, w.dist,
                                                           (const double2 *)pos, w.part, status, gaveup);
    else
      note_launch(), k_pairs_sampled<float2, uint16_t><<<pb, kPairThreads, 0, s>>>(n, S, ntargets, seed, w.src, w.dist,
                                                          (const float2 *)pos, w.part, status, gaveup);
  } else {
    for (int b = 0; b < nb; ++b) {
      const int32_t base = b * S, B = std::min<int32_t>(S, n - base);
      note_launch(), k_batch_sources<<<std::max(1, (B + 255) / 256), 256, 0, s>>>(base, B, w.src);
      int rc = launch_msbfs(n, 2 * m, rowptr, colidx, B, w.src, w.dist, status, w.bfs, w.bfs_bytes, s);
      if (rc) return rc;
      double *part = w.part + 4 * (size_t)pb * b;
      if (precision == 64)
        note_launch(), k_pairs_exhaustive<double2, uint16_t><<<pb, kPairThreads, 0, s>>>(n, base, B, w.dist, (const double2 *)pos, part,
                                                                status);
      else
        note_launch(), k_pairs_exhaustive<float2, uint16_t><<<pb, kPairThreads, 0, s>>>(n, base, B, w.dist, (const float2 *)pos, part,
                                                               status);
    }
  }
  note_launch(), k_stress_final<<<1, 1024, 0, s>>>(n, (int64_t)pb * nb, w.part, nsources > 0, out, sums, w.part_pull,
                                                   npull, gaveup);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

// ------------------------------------------------------------- weighted
// The same sums with weighted distances: the float32 least path sums of the
// weighted search (weighted.cu) from the sources, in batches.
namespace ssm {
struct WStressWs {
  int32_t *src;
  float *dist;
  double *part;
  void *sssp;
  size_t sssp_bytes;
};
static size_t carve_wstress(Carver &c, WStressWs &w, int32_t n, int32_t S, int32_t nbatches) {
  w.src = c.take<int32_t>(S);
  w.dist = c.take<float>((size_t)S * n);
  w.part = c.take<double>(4 * (size_t)pair_blocks() * (size_t)nbatches);
  w.sssp_bytes = sssp_ws_bytes(n, S);
  w.sssp = c.take<char>(w.sssp_bytes);
  return c.size();
}
}  // namespace ssm

SSM_API size_t ssm_stress_weighted_workspace(int32_t n, int32_t nsources) {
  if (n < 2 || nsources < 0) return 0;
  int32_t S, nb;
  ssm::stress_shape(n, nsources, &S, &nb);
  ssm::Carver c(nullptr, 0);
  ssm::WStressWs w;
  return ssm::carve_wstress(c, w, n, S, nb);
}

SSM_API int ssm_stress_weighted(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen,
                                const void *pos, int32_t precision, int32_t nsources, int32_t ntargets, uint64_t seed,
                                double *out, double *sums, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s) {
  using namespace ssm;
  if (n < 2 || !rowptr || !colidx || !elen || !pos || !out || !status || !ws)
    return fail(SSM_E_ARG, "ssm_stress_weighted: null pointer or bad size");
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_stress_weighted: precision must be 32 or 64");
  if (nsources < 0 || nsources > 65535 || (nsources > 0 && ntargets < 1))
    return fail(SSM_E_ARG, "ssm_stress_weighted: need 0 <= nsources <= 65535 and ntargets >= 1 when sampling");
  int32_t S, nb;
  stress_shape(n, nsources, &S, &nb);
  Carver c(ws, ws_bytes);
  WStressWs w;
  carve_wstress(c, w, n, S, nb);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_stress_weighted: workspace %zu bytes, need %zu", ws_bytes, c.size());
  const int pb = pair_blocks();
  if (nsources > 0) {
    note_launch(), k_sample_sources<<<std::max(1, (S + 255) / 256), 256, 0, s>>>(n, S, seed, w.src);
    int rc = launch_sssp(n, rowptr, colidx, elen, S, w.src, w.dist, status, w.sssp, w.sssp_bytes, s);
    if (rc) return rc;
    if (precision == 64)
      note_launch(), k_pairs_sampled<double2, float><<<pb, kPairThreads, 0, s>>>(n, S, ntargets, seed, w.src, w.dist,
                                                                            (const double2 *)pos, w.part, status, nullptr);
    else
      note_launch(), k_pairs_sampled<float2, float><<<pb, kPairThreads, 0, s>>>(n, S, ntargets, seed, w.src, w.dist,
                                                                           (const float2 *)pos, w.part, status, nullptr);
  } else {
    for (int b = 0; b < nb; ++b) {
      const int32_t base = b * S, B = std::min<int32_t>(S, n - base);
      note_launch(), k_batch_sources<<<std::max(1, (B + 255) / 256), 256, 0, s>>>(base, B, w.src);
      int rc = launch_sssp(n, rowptr, colidx, elen, B, w.src, w.dist, status, w.sssp, w.sssp_bytes, s);
      if (rc) return rc;
      double *part = w.part + 4 * (size_t)pb * b;
      if (precision == 64)
        note_launch(), k_pairs_exhaustive<double2, float><<<pb, kPairThreads, 0, s>>>(n, base, B, w.dist,
                                                                               (const double2 *)pos, part, status);
      else
        note_launch(), k_pairs_exhaustive<float2, float><<<pb, kPairThreads, 0, s>>>(n, base, B, w.dist,
                                                                              (const float2 *)pos, part, status);
    }
  }
  note_launch(), k_stress_final<<<1, 1024, 0, s>>>(n, (int64_t)pb * nb, w.part, nsources > 0, out, sums);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
