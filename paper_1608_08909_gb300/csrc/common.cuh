// Shared device/host helpers of libssm: status reporting, workspace carving,
// a device-wide barrier with a time limit, warp-aggregated queue appends.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ssm.h"

#define SSM_API extern "C" __attribute__((visibility("default")))

namespace ssm {

// ---------------------------------------------------------------- host side
int fail(int code, const char *fmt, ...);          // records ssm_last_error, returns code
int cuda_status(cudaError_t e, const char *what);  // SSM_OK or SSM_E_CUDA (recorded)
int num_sms();                                     // SM count of the current device
// Counts one kernel enqueued by this library; every launch site calls it just
// before its launch ("note_launch(), k<<<...>>>(...)" keeps if/else one-liners
// single expressions).  ssm_kernel_launches() reports the running total.
void note_launch();
#define SSM_TRY_CUDA(call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return ::ssm::cuda_status(e_, #call); \
  } while (0)

// Carves 256-byte-aligned sub-buffers out of a workspace.  With base ==
// nullptr it only adds up the size (for the *_workspace queries).
struct Carver {
  char *base;
  size_t cap;
  size_t off = 0;
  bool ok = true;
  Carver(void *b, size_t c) : base((char *)b), cap(c) {}
  template <class T>
  T *take(size_t count) {
    size_t o = (off + 255) & ~size_t(255);
    size_t bytes = count * sizeof(T);
    off = o + bytes;
    if (!base) return nullptr;
    if (off > cap) { ok = false; return nullptr; }
    return (T *)(base + o);
  }
  size_t size() const { return (off + 255) & ~size_t(255); }
};

// Device-wide barrier state, reset by reset_barrier() before each persistent
// launch.  limit_ns is the longest one wait may take before the barrier gives
// up (0: kBarrierTimeoutNs); it is non-zero only while a caller has set a
// shorter limit with ssm_set_wait_limit_ns.
struct BarrierState {
  unsigned count;
  unsigned gen;
  unsigned abort;
  unsigned limit_ns;
};

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s per wait

// Neighbour rows of the sweep by length: up to kShortDeg entries one thread,
// up to kMidDeg one warp, longer rows one block (the graph builder counts
// the two longer classes for the sweep's launch shape).
constexpr int kShortDeg = 32;
constexpr int kMidDeg = 1024;

// Zeroes *b on `stream` and, while a shorter wait limit is set, stores it.
int reset_barrier(BarrierState *b, cudaStream_t stream);

// ---------------------------------------------------------------- device side
__device__ __forceinline__ void dev_fail(int32_t *status, int code) {
  if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Device-wide barrier for a cooperative (co-resident) grid.  Every block
// must call it the same number of times.  Returns false when the wait gave
// up (after kBarrierTimeoutNs, recording SSM_E_TIMEOUT) or another block
// gave up; the caller must then leave the kernel.
__device__ __forceinline__ bool grid_barrier(BarrierState *b, int32_t *status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    unsigned g = ld_acquire_u32(&b->gen);
    unsigned arrived = atom_add_acq_rel_u32(&b->count, 1u);
    if (arrived == gridDim.x - 1) {
      b->count = 0;
      __threadfence();
      st_release_u32(&b->gen, g + 1);
    } else {
      const unsigned long long limit = b->limit_ns ? (unsigned long long)b->limit_ns : kBarrierTimeoutNs;
      unsigned long long t0 = globaltimer_ns();
      unsigned nap = 32;
      while (ld_acquire_u32(&b->gen) == g) {
        // back off so that waiting blocks do not crowd the L2 slice that the
        // working blocks need
        __nanosleep(nap);
        if (nap < 256) nap <<= 1;
        if (ld_acquire_u32(&b->abort)) { ok = 0; break; }
        if (globaltimer_ns() - t0 > limit) {
          dev_fail(status, SSM_E_TIMEOUT);
          atomicExch(&b->abort, 1u);
          ok = 0;
          break;
        }
      }
    }
    if (ok && ld_acquire_u32(&b->abort)) ok = 0;
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// counts[0] += rows with kShortDeg < length <= kMidDeg, counts[1] += longer rows
__global__ void k_row_classes(int32_t n, const int32_t *__restrict__ rowptr, unsigned *__restrict__ counts);

// All 32 lanes must call this together.  Lanes with pred append `val` to
// q[*qcount ...]; one atomic per warp.
__device__ __forceinline__ void warp_append(bool pred, unsigned val, unsigned *q, unsigned *qcount) {
  const unsigned lane = threadIdx.x & 31u;
  unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (!mask) return;
  unsigned base = 0;
  const int leader = __ffs(mask) - 1;
  if ((int)lane == leader) base = atomicAdd(qcount, (unsigned)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) q[base + __popc(mask & ((1u << lane) - 1u))] = val;
}

// Warp-cooperative walk over the neighbour lists of up to 32 items (one per
// lane, item valid iff beg < end).  Calls f for every
// neighbour slot as f(owner_lane, active, v), 32 slots at a time, with all
// lanes converged (active == false on padding slots).  Balances hubs across
// the warp.
template <class F>
__device__ __forceinline__ void warp_for_each_neighbor(int beg, int end, const int32_t *__restrict__ colidx,
                                                       F &&f) {
  const unsigned lane = threadIdx.x & 31u;
  int deg = end > beg ? end - beg : 0;
  int incl = deg;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += t;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  for (int base = 0; base < total; base += 32) {
    const int idx = base + (int)lane;
    const bool act = idx < total;
    // owner = first lane whose inclusive prefix exceeds idx
    int lo = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      int probe = lo + step - 1;
      int pv = __shfl_sync(0xffffffffu, incl, probe);
      if (pv <= idx) lo += step;
    }
    const int owner = lo > 31 ? 31 : lo;
    const int o_incl = __shfl_sync(0xffffffffu, incl, owner);
    const int o_deg = __shfl_sync(0xffffffffu, deg, owner);
    const int o_beg = __shfl_sync(0xffffffffu, beg, owner);
    int v = 0;
    if (act) v = __ldg(colidx + o_beg + (idx - (o_incl - o_deg)));
    f(owner, act, v);
  }
}

// Batched form of warp_for_each_neighbor for latency-bound BFS levels: each
// step covers U*32 neighbour slots.  gather(u, owner, v) runs for every active
// slot first (so its memory operations for the U slots are in flight
// together), then emit(u, owner, v, act) runs for every slot with all lanes
// converged.
template <int U, class Gather, class Emit>
__device__ __forceinline__ void warp_for_each_neighbor_batched(int beg, int end, const int32_t *__restrict__ colidx,
                                                               Gather &&gather, Emit &&emit) {
  const unsigned lane = threadIdx.x & 31u;
  const int deg = end > beg ? end - beg : 0;
  int incl = deg;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += t;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  for (int base = 0; base < total; base += 32 * U) {
    int v[U], own[U];
    bool act[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + 32 * u + (int)lane;
      act[u] = idx < total;
      int lo = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int pv = __shfl_sync(0xffffffffu, incl, lo + step - 1);
        if (pv <= idx) lo += step;
      }
      own[u] = lo > 31 ? 31 : lo;
      const int o_incl = __shfl_sync(0xffffffffu, incl, own[u]);
      const int o_deg = __shfl_sync(0xffffffffu, deg, own[u]);
      const int o_beg = __shfl_sync(0xffffffffu, beg, own[u]);
      v[u] = act[u] ? __ldg(colidx + o_beg + (idx - (o_incl - o_deg))) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) act[u] = act[u] && gather(u, own[u], v[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) emit(u, own[u], v[u], act[u]);
  }
}

// Appends val for the lanes with pred to q (with a shared-memory counter) and
// returns each appending lane's slot; all lanes must call it together.
__device__ __forceinline__ unsigned warp_slot(bool pred, unsigned *s_counter) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (!mask) return 0u;
  unsigned base = 0;
  const int leader = __ffs(mask) - 1;
  if ((int)lane == leader) base = atomicAdd(s_counter, (unsigned)__popc(mask));
  return __shfl_sync(0xffffffffu, base, leader) + __popc(mask & ((1u << lane) - 1u));
}

__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
  // value c of the counter-based splitmix64 stream (Steele, Lea, Flood 2014)
  uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Persistent cooperative launch sized to the device: blocks = SMs * resident.
int cooperative_blocks(const void *kernel, int threads, size_t smem, int max_per_sm);
// Lets `kernel` take as much dynamic shared memory as the device allows.  The
// attribute is the same on every call, so calls on concurrent host threads
// (each launching with its own size) cannot undo one another.
cudaError_t allow_dynamic_smem(const void *kernel);

}  // namespace ssm
