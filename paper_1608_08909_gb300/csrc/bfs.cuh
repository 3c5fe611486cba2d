// Internal entry points of the BFS kernels (bfs.cu), shared by the graph
// builder (connectivity check) and the stress reducer (distances from the
// sampled sources).
#pragma once
#include <functional>

#include "common.cuh"

namespace ssm {

// m2 = number of directed edges (colidx entries) in all of these.
size_t maxmin_workspace(int32_t n, int64_t m2);
// max/min-sp pivots; with k == 1 it is a single BFS from `start` that flags
// SSM_E_DISCONNECTED in *status if some node is unreachable.
int launch_maxmin(int32_t n, int64_t m2, const int32_t *rowptr, const int32_t *colidx, int32_t k, int32_t start,
                  int32_t *pivots, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s);

// max/min pivots inside one thread-block cluster (maxmin_cluster.cu), for
// graphs whose mind array fits the cluster's shared memory.  Sets
// *mind_bytes to 4 or 2 when the cluster kernel was enqueued (0: the caller
// uses the grid kernel).  With 2 bytes the caller also queues the grid kernel
// to run only if *fallback (device) was set: a search deeper than 65534
// levels.  spill holds maxmin_cluster_spill_entries(n) entries.  With
// init_mind / init_best (device; mind and the packed maximum after the first
// search, from start, on the whole grid) the cluster starts at pivot 1,
// unless *init_gaveup (device) says that search stopped early.
size_t maxmin_cluster_spill_entries(int32_t n);
int maxmin_cluster_mind_bytes(int32_t n);  // 4 or 2 if the cluster kernel would run, else 0
int launch_maxmin_cluster(int32_t n, const int32_t *rowptr, const int4 *adj, int32_t k, int32_t start,
                          int32_t *pivots, int32_t *status, unsigned *spill, unsigned *fallback,
                          const unsigned *init_mind, const unsigned long long *init_best,
                          const unsigned *init_gaveup, cudaStream_t s, int *mind_bytes);
// records the kernel the last selection took (cluster size, 0 for the grid kernel; mind bytes)
void note_pivot_config(int32_t cluster, int32_t mind_bytes);

// One pass of the pulled BFS, as its caller may read it: for levels
// L < *nlev (device), F holds [L][n][kPullPassWords] words in which bit
// a & 31 of word a >> 5 of node v is set when source base + a (a < nsrc)
// first reached v at level L.  Valid until the next pass starts; nothing in
// it is valid if *gaveup (device) is set.
constexpr int kPullPassWords = 8;
constexpr int kPullPassSources = 256;    // sources per pass
constexpr unsigned kPullPassLevels = 25;  // levels F has room for
struct PullPass {
  const unsigned *F;
  const unsigned *nlev;
  const unsigned *gaveup;
  int32_t base, nsrc, pass;
};
using PullPassFn = std::function<int(const PullPass &)>;

// multi-source BFS pulled level by level, 256 sources per pass (msbfs_pull.cu);
// sets *gaveup (device, cleared by the caller) if a pass needed more levels
// than it allows, leaving dist to another BFS.  With after_pass, each pass is
// handed to it (enqueued behind the pass) instead of being written to dist.
size_t msbfs_pull_workspace(int32_t n);
int launch_msbfs_pull(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k, const int32_t *sources,
                      uint16_t *dist, int32_t *status, unsigned *gaveup, void *ws, size_t ws_bytes, cudaStream_t s,
                      const PullPassFn *after_pass = nullptr);

size_t msbfs_workspace(int32_t n, int64_t m2, int32_t k);
// dist[a*n + v] = hop distance from sources[a] to v, for a < k
// With after_pass (graphs small enough for the pulled BFS), the passes go to it
// and dist is written only if the pulled BFS gives up; *pull_gaveup then gets
// the device flag that says so (nullptr when the pulled BFS was not tried and
// dist is always written).
int launch_msbfs(int32_t n, int64_t m2, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                 const int32_t *sources, uint16_t *dist, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t s,
                 const PullPassFn *after_pass = nullptr, const unsigned **pull_gaveup = nullptr);

}  // namespace ssm
