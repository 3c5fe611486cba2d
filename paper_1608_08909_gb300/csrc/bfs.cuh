// Internal entry points of the BFS kernels (bfs.cu), shared by the graph
// builder (connectivity check) and the stress reducer (distances from the
// sampled sources).
#pragma once
#include "common.cuh"

namespace ssm {

// m2 = number of directed edges (colidx entries) in all of these.
size_t maxmin_workspace(int32_t n, int64_t m2);
// max/min-sp pivots; with k == 1 it is a single BFS from `start` that flags
// SSM_E_DISCONNECTED in *status if some node is unreachable.
int launch_maxmin(int32_t n, int64_t m2, const int32_t *rowptr, const int32_t *colidx, int32_t k, int32_t start,
                  int32_t *pivots, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s);

// max/min pivots inside one thread-block cluster (maxmin_cluster.cu), for
// graphs whose mind array fits the cluster's shared memory.  Sets *launched
// when the cluster kernel was enqueued; otherwise the caller uses the grid
// kernel.  spill holds maxmin_cluster_spill_entries(n) entries.
size_t maxmin_cluster_spill_entries(int32_t n);
int launch_maxmin_cluster(int32_t n, const int32_t *rowptr, const int4 *adj, int32_t k, int32_t start,
                          int32_t *pivots, int32_t *status, unsigned *spill, cudaStream_t s, bool *launched);

// multi-source BFS pulled level by level, 256 sources per pass (msbfs_pull.cu);
// sets *gaveup (device, cleared by the caller) if a pass needed more levels
// than it allows, leaving dist to another BFS
size_t msbfs_pull_workspace(int32_t n);
int launch_msbfs_pull(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k, const int32_t *sources,
                      uint16_t *dist, int32_t *status, unsigned *gaveup, void *ws, size_t ws_bytes, cudaStream_t s);

size_t msbfs_workspace(int32_t n, int64_t m2, int32_t k);
// dist[a*n + v] = hop distance from sources[a] to v, for a < k
int launch_msbfs(int32_t n, int64_t m2, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                 const int32_t *sources, uint16_t *dist, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s);

}  // namespace ssm
