// Exclusive prefix sum of int32 counts on the device (three passes over
// tiles: per-tile scan, scan of the tile totals, add tile offsets).
#pragma once
#include "common.cuh"

namespace ssm {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

static inline int64_t scan_tiles(int64_t count) { return (count + kScanTile - 1) / kScanTile; }

// block-wide exclusive scan of one value per thread; returns the block total in *total
static __device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
  __shared__ int warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  int r = incl - v + warp_tot[wid];
  __syncthreads();
  return r;
}

static __global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int *__restrict__ in, int *__restrict__ out,
                                                               int *__restrict__ tile_sums, int64_t count) {
  __shared__ int s_total;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int vals[kScanItems];
  int sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    vals[j] = (base + j < count) ? in[base + j] : 0;
    sum += vals[j];
  }
  int off = block_exclusive_scan(sum, &s_total);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < count) out[base + j] = off;
    off += vals[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = s_total;
}

// one block: exclusive scan of the tile totals in place; grand total to *total_out
static __global__ void __launch_bounds__(kScanThreads) k_scan_sums(int *__restrict__ tile_sums, int64_t ntiles,
                                                              int *__restrict__ total_out) {
  __shared__ int s_total;
  int carry = 0;
  for (int64_t b = 0; b < ntiles; b += kScanThreads) {
    int64_t i = b + threadIdx.x;
    int v = i < ntiles ? tile_sums[i] : 0;
    int off = block_exclusive_scan(v, &s_total);
    if (i < ntiles) tile_sums[i] = off + carry;
    carry += s_total;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

static __global__ void __launch_bounds__(kScanThreads) k_scan_add(int *__restrict__ out, const int *__restrict__ tile_sums,
                                                             int64_t count) {
  const int add = tile_sums[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int j = threadIdx.x; j < kScanTile; j += kScanThreads)
    if (base + j < count) out[base + j] += add;
}

// out[0..count-1] = exclusive scan of in; out[count] = total (out has count+1 slots).
// tile_ws needs scan_tiles(count) ints.
static inline int exclusive_scan(const int *in, int *out, int64_t count, int *tile_ws, cudaStream_t s) {
  int64_t tiles = scan_tiles(count);
  if (tiles == 0) {
    SSM_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
    return SSM_OK;
  }
  note_launch(), k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, tile_ws, count);
  note_launch(), k_scan_sums<<<1, kScanThreads, 0, s>>>(tile_ws, tiles, out + count);
  note_launch(), k_scan_add<<<(unsigned)tiles, kScanThreads, 0, s>>>(out, tile_ws, count);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

}  // namespace ssm
