// Internal entry points of the weighted-graph search (weighted.cu), shared
// with the stress reducer (distances from sampled sources on weighted graphs).
#pragma once
#include "common.cuh"

namespace ssm {

// Blocks the multi-source search runs (one source per block at a time) and
// the workspace bytes of one block's queues.
int sssp_blocks(int32_t k);
size_t sssp_slot_bytes(int32_t n);
size_t sssp_ws_bytes(int32_t n, int32_t k);  // launch_sssp's workspace
// dist[a*n + v] = least float32 path sum from sources[a] to v, for a < k;
// an unreachable node flags SSM_E_DISCONNECTED.  ws holds
// sssp_ws_bytes(n, k) bytes.
int launch_sssp(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t k,
                const int32_t *sources, float *dist, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s);

}  // namespace ssm
