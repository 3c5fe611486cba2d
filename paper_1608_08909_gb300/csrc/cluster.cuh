// Thread-block cluster helpers (inline PTX): the CTA's rank, the hardware
// cluster barrier, and loads, stores and atomics on another CTA's shared
// memory (distributed shared memory).
#pragma once
#include <cstdint>

namespace ssm {

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// all threads of all CTAs of the cluster; release/acquire for shared and global memory
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t dsmem_addr(const void *p, unsigned rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t d;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
  return d;
}

// atomicMin on a DSMEM word when pred holds (returns 0 otherwise).  No branch
// and no compiler memory barrier, so the atomics of several slots are in
// flight together; ordering against other threads comes from the barriers.
__device__ __forceinline__ unsigned dsmem_atomic_min_if(bool pred, uint32_t a, unsigned v) {
  unsigned old = 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
      "@p atom.shared::cluster.min.u32 %0, [%1], %3;\n\t}"
      : "+r"(old)
      : "r"(a), "r"((unsigned)pred), "r"(v));
  return old;
}

__device__ __forceinline__ unsigned dsmem_atomic_add_if(bool pred, uint32_t a, unsigned v) {
  unsigned old = 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
      "@p atom.shared::cluster.add.u32 %0, [%1], %3;\n\t}"
      : "+r"(old)
      : "r"(a), "r"((unsigned)pred), "r"(v));
  return old;
}

__device__ __forceinline__ void dsmem_st_v4(uint32_t a, int4 e) {
  asm volatile("st.shared::cluster.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(e.x), "r"(e.y), "r"(e.z), "r"(e.w));
}

__device__ __forceinline__ void dsmem_st_u32(uint32_t a, unsigned v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ void dsmem_st_u64(uint32_t a, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned dsmem_ld_u32(uint32_t a) {
  unsigned v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}

__device__ __forceinline__ unsigned dsmem_cas_u32(uint32_t a, unsigned cmp, unsigned v) {
  unsigned old;
  asm volatile("atom.shared::cluster.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "r"(a), "r"(cmp), "r"(v) : "memory");
  return old;
}

}  // namespace ssm
