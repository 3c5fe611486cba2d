// Status strings, per-thread error text, device queries.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>

#include "common.cuh"

namespace ssm {

static thread_local char g_last_error[512] = "";
static std::atomic<unsigned long long> g_launches{0};
// wait limit of the device-wide barriers set by ssm_set_wait_limit_ns (0: the default)
static std::atomic<unsigned> g_wait_limit_ns{0};
// the limit as a host word that a copy can read while another thread changes g_wait_limit_ns
static thread_local unsigned g_wait_limit_copy = 0;

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_status(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return SSM_OK;
  return fail(SSM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int num_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

cudaError_t allow_dynamic_smem(const void *kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

int reset_barrier(BarrierState *b, cudaStream_t stream) {
  SSM_TRY_CUDA(cudaMemsetAsync(b, 0, sizeof(BarrierState), stream));
  g_wait_limit_copy = g_wait_limit_ns.load(std::memory_order_relaxed);
  if (g_wait_limit_copy != 0)
    SSM_TRY_CUDA(cudaMemcpyAsync(&b->limit_ns, &g_wait_limit_copy, sizeof(unsigned), cudaMemcpyHostToDevice, stream));
  return SSM_OK;
}

int cooperative_blocks(const void *kernel, int threads, size_t smem, int max_per_sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) return 0;
  if (per_sm > max_per_sm) per_sm = max_per_sm;
  return per_sm * num_sms();
}

}  // namespace ssm

SSM_API const char *ssm_status_string(int code) {
  switch (code) {
    case SSM_OK: return "ok";
    case SSM_E_ARG: return "invalid argument";
    case SSM_E_GRAPH: return "edge endpoint out of range";
    case SSM_E_DISCONNECTED: return "graph is disconnected";
    case SSM_E_DIST_OVERFLOW: return "hop distance above 65534";
    case SSM_E_NOMEM: return "workspace too small";
    case SSM_E_CUDA: return "CUDA error";
    case SSM_E_TIMEOUT: return "device-wide wait timed out";
    case SSM_E_NUMERIC: return "numerical failure";
    default: return "unknown status";
  }
}

SSM_API const char *ssm_last_error(void) { return ssm::g_last_error; }

SSM_API unsigned long long ssm_kernel_launches(void) { return ssm::g_launches.load(std::memory_order_relaxed); }

SSM_API int ssm_check(const int32_t *status, cudaStream_t stream) {
  int32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, status, sizeof h, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return ssm::cuda_status(e, "ssm_check");
  if (h != 0) return ssm::fail(h, "device reported: %s", ssm_status_string(h));
  return SSM_OK;
}

SSM_API unsigned long long ssm_set_wait_limit_ns(unsigned long long ns) {
  if (ns > 0xFFFFFFFFull) ns = 0xFFFFFFFFull;
  return ssm::g_wait_limit_ns.exchange((unsigned)ns);
}

namespace ssm {
__global__ void k_row_classes(int32_t n, const int32_t *__restrict__ rowptr, unsigned *__restrict__ counts) {
  unsigned mid = 0, lng = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int deg = rowptr[i + 1] - rowptr[i];
    mid += (deg > kShortDeg && deg <= kMidDeg) ? 1u : 0u;
    lng += deg > kMidDeg ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mid += __shfl_xor_sync(0xffffffffu, mid, o);
    lng += __shfl_xor_sync(0xffffffffu, lng, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (mid) atomicAdd(counts, mid);
    if (lng) atomicAdd(counts + 1, lng);
  }
}
}  // namespace ssm
