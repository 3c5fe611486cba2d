/*
 * ssm.h -- C ABI of the GB300 sparse stress layout library (libssm.so).
 *
 * The library computes the sparse stress model of Ortmann, Klimenta and
 * Brandes, "A Sparse Stress Model" (arxiv 1608.08909): Algorithm 1 with the
 * update of Eq. 4 applied Jacobi-style (every node from the previous
 * iterate), on one GPU.  Call order for one layout:
 *
 *   ssm_build_graph -> ssm_select_pivots -> ssm_pivot_bfs -> ssm_aggregate_size
 *   -> ssm_aggregate -> ssm_pivotmds -> ssm_iterate (repeatable) -> ssm_stress
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller unless the
 *     comment says "host".  The library never allocates device memory: each
 *     call that needs scratch takes a caller-allocated device workspace
 *     (ws, ws_bytes) whose size comes from the matching *_workspace query;
 *     it must be 256-byte aligned and is not used after the call's work on
 *     `stream` completes.
 *   - Calls are asynchronous on `stream` unless marked "synchronous".
 *   - The return value reports argument and launch errors found on the host
 *     (SSM_OK or a negative code; ssm_last_error() gives details).  Errors
 *     found by a kernel are written to the caller's device word `status`
 *     (first error wins; 0 means none) and read with ssm_check().  `status`
 *     must be zeroed by the caller before first use.
 *   - Graphs are simple and undirected, stored as CSR: rowptr[n+1] int32,
 *     colidx[2m] int32, every row sorted ascending, no self-loops, no
 *     repeated entries (as produced by ssm_build_graph).  Node ids are 0..n-1.
 *     Calls that take a graph take (n, m, rowptr, colidx) with m = |E|.
 *   - Positions are interleaved (x, y) pairs: float[2n] for precision 32,
 *     double[2n] for precision 64.
 *   - The pivot-distance table d_ip is pivot-major uint16: dip[a*n + i] is the
 *     hop distance between pivot a (the a-th selected pivot) and node i.
 */
#ifndef SSM_H
#define SSM_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SSM_OK 0
#define SSM_E_ARG (-1)           /* null pointer, size out of range, k > n ... */
#define SSM_E_GRAPH (-2)         /* an edge endpoint outside 0..n-1 */
#define SSM_E_DISCONNECTED (-3)  /* the graph has more than one component */
#define SSM_E_DIST_OVERFLOW (-4) /* a hop distance above 65534 (uint16 table) */
#define SSM_E_NOMEM (-5)         /* workspace smaller than its query */
#define SSM_E_CUDA (-6)          /* a CUDA runtime call failed */
#define SSM_E_TIMEOUT (-7)       /* a device-wide wait gave up (see each call) */
#define SSM_E_NUMERIC (-8)       /* non-finite value or a failed eigen-solve */

/* Text for a status code (static storage). */
const char *ssm_status_string(int code);

/* Detail of the last failing call on this host thread (thread-local; static
 * storage valid until the next failing call on the same thread). */
const char *ssm_last_error(void);

/* Number of kernels this library has enqueued since it was loaded, over all
 * host threads and devices (memsets and copies are not counted).  A
 * diagnostic with no counterpart in the paper: a caller reads it before and
 * after a sequence of calls to learn how many kernels the sequence issued. */
unsigned long long ssm_kernel_launches(void);

/* Sets the longest time one wait at a device-wide barrier may take before
 * the kernel gives up with SSM_E_TIMEOUT (the persistent kernels of
 * ssm_select_pivots, ssm_pivot_bfs, ssm_stress and ssm_pivotmds wait at such
 * barriers between their steps); ns = 0 restores the default of 2 s, values
 * above 2^32 - 1 are clamped.  Returns the previous setting.  A diagnostic
 * with no counterpart in the paper, for tests of the timeout path: a limit of
 * a few nanoseconds makes the first wait of such a kernel run out, and the
 * kernel then records SSM_E_TIMEOUT, releases the other blocks and returns.
 * It applies to calls made after it, on every host thread; while it is
 * non-zero each such call also copies the limit from host memory. */
unsigned long long ssm_set_wait_limit_ns(unsigned long long ns);

/* What the last ssm_iterate call on this host thread chose, in out[4] (host):
 *   out[0] the sweep kernel: 0 FP32 with the clamped s table in shared memory,
 *          1 FP32 with the clamped s table in global memory, 2 FP32 with the
 *          full (w', w' d) table, 3 FP64 with the counts in shared memory,
 *          4 FP64 with the counts in global memory (-1: no call yet);
 *   out[1] pivot ranges per 128-node tile (1: a warp takes whole tiles);
 *   out[2] blocks of the sweep grid;  out[3] the largest d_ip entry (FP32) or -1.
 * A diagnostic with no counterpart in the paper. */
void ssm_last_sweep_config(int32_t *out);

/* What the last max/min pivot selection on this host thread chose, in out[2]
 * (host): out[0] the thread-block cluster size of the cluster kernel (0: the
 * cooperative grid kernel; -1: no call yet), out[1] bytes of the distance to
 * the closest pivot per node (4, or 2 for graphs whose 4-byte array does not
 * fit the cluster; a search deeper than 65534 levels then hands the whole
 * selection to the grid kernel on the device).  A diagnostic with no
 * counterpart in the paper. */
void ssm_last_pivot_config(int32_t *out);

/* Synchronous: waits for `stream`, then returns the device status word
 * (SSM_OK if it is 0), or SSM_E_CUDA if the stream reported a CUDA error. */
int ssm_check(const int32_t *status, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Graph.  Section 1: G = (V, E) simple and undirected, n = |V|, m = |E|.
 * Builds the CSR from an undirected edge list (src[e], dst[e]), e < m_in:
 * both directions stored, self-loops and repeated edges dropped, rows
 * sorted ascending, then checks that G is connected (the paper keeps only
 * the largest component, Section 4 "Data"; callers pass that component).
 * rowptr has n+1 entries, colidx room for 2*m_in.  *m_out (host) receives m;
 * row_classes (host int32[2], may be NULL) the number of rows with 33 to
 * 1024 entries and with more than 1024 (the sweep's launch shape: pass them
 * to ssm_iterate as hints[1], hints[2]).  Synchronous.  Errors are returned
 * directly: SSM_E_GRAPH for an endpoint outside 0..n-1, SSM_E_DISCONNECTED
 * if some node is unreachable from node 0.
 * Requires 1 <= n, 0 <= m_in, 2*m_in < 2^31.
 * ------------------------------------------------------------------- */
size_t ssm_build_graph_workspace(int32_t n, int64_t m_in);
int ssm_build_graph(int32_t n, int64_t m_in, const int32_t *src, const int32_t *dst,
                    int32_t *rowptr, int32_t *colidx, int64_t *m_out, int32_t *row_classes,
                    void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Pivot sampling, "max/min sp" (Section 4.1; Algorithm 1 line 1):
 * pivots[0] = start, then repeatedly the node maximising the hop distance to
 * its closest chosen pivot, ties to the lowest node id.  Writes pivots[k]
 * (int32, selection order).  1 <= k <= n.  Device errors: SSM_E_DISCONNECTED,
 * SSM_E_TIMEOUT (a device-wide barrier waited longer than 2 s).
 * ------------------------------------------------------------------- */
size_t ssm_select_pivots_workspace(int32_t n, int64_t m);
int ssm_select_pivots(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                      int32_t start, int32_t *pivots, int32_t *status,
                      void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Pivot sampling, "k-means sp" (Section 4.1, the paper's recommended
 * sampler): k max/min-sp pivots pivots_in[k] (from ssm_select_pivots) and
 * their table dip[k*n] (from ssm_pivot_bfs) are refined by k-means over the
 * nodes' shortest-path entries.  Node i is y_i = (d_0i, ..., d_{k-1,i}) in
 * Z^k; cluster a starts with centre y of pivots_in[a].  Each pass assigns
 * every node to the centre c_a minimising ||y_i - c_a||^2 (ties to the lowest
 * a), compared as alpha_a - beta_a * t_ia with t_ia = y_i . S_a exact,
 * alpha_a = sum_b (S_ab/n_a)^2 (FP64, b ascending) and beta_a = 2/n_a, where
 * c_a = S_a/n_a; then the centres become the members' means (an empty cluster
 * keeps its centre).  At most max_iter passes (the paper caps its k-means at
 * 50); it stops after the first pass, beyond the first, that moves no node.
 * pivots_out[a] (device int32) = the member of cluster a nearest its centre
 * (compared exactly as n_a ||y_i||^2 - 2 t_ia, ties to the lowest node id),
 * or pivots_in[a] if the cluster is empty.  assign[n] (device int32, may be
 * NULL) receives each node's cluster, *iters (device int32) the passes run.
 * The caller then recomputes d_ip for pivots_out with ssm_pivot_bfs.
 * Asynchronous (every pass is enqueued; passes after the stop return at
 * once).  1 <= k <= min(n, 1024), 1 <= max_iter.  Device error SSM_E_ARG
 * when n * max(d) >= 2^32 or n * k * max(d)^2 >= 2^53 (the bounds of the
 * exact integer arithmetic) or a pivot id is outside 0..n-1.
 * ------------------------------------------------------------------- */
size_t ssm_kmeans_pivots_workspace(int32_t n, int32_t k);
int ssm_kmeans_pivots(int32_t n, int32_t k, const uint16_t *dip, const int32_t *pivots_in, int32_t max_iter,
                      int32_t *pivots_out, int32_t *assign, int32_t *iters, int32_t *status,
                      void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Pivot distances d_ip (Algorithm 1 line 2, unit edge lengths): one
 * multi-source BFS from all k pivots at once.  Writes dip[k*n] (uint16,
 * pivot-major).  1 <= k <= 65535, n*ceil(k/32) < 2^31.  Pivots need not be
 * distinct.  Device errors: SSM_E_DISCONNECTED, SSM_E_DIST_OVERFLOW,
 * SSM_E_TIMEOUT, SSM_E_ARG (a pivot id outside 0..n-1).
 * ------------------------------------------------------------------- */
size_t ssm_pivot_bfs_workspace(int32_t n, int64_t m, int32_t k);
int ssm_pivot_bfs(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                  const int32_t *pivots, uint16_t *dip, int32_t *status,
                  void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Regions and distance counts behind the adapted weights (Section 3):
 *   region[i] = the lowest pivot index a minimising d_ia   (R(p) of the paper);
 *   ecc_a     = max over i in R(a) of d_ia;
 *   cnt[cnt_off[a] + t] = |{ i in R(a) : d_ia <= t }|, t = 0..ecc_a,
 * so that w'_ia = s / d_ia^2 with s = cnt[cnt_off[a] + min(floor(d_ia/2), ecc_a)].
 * ssm_aggregate_size (synchronous) returns in *cnt_len (host) the table length
 * sum_a (ecc_a + 1) and in *dip_max (host, may be NULL) the largest d_ia
 * (ssm_iterate's hints[0]); ssm_aggregate fills region[n] int32, cnt_off[k+1] int32,
 * cnt[cnt_len] uint32.  Workspace: ssm_aggregate_workspace(k) bytes for both.
 * Device error SSM_E_ARG if cnt_len does not match the table.
 * ------------------------------------------------------------------- */
size_t ssm_aggregate_workspace(int32_t k);
int ssm_aggregate_size(int32_t n, int32_t k, const uint16_t *dip, int64_t *cnt_len, int32_t *dip_max,
                       void *ws, size_t ws_bytes, cudaStream_t stream);
int ssm_aggregate(int32_t n, int32_t k, const uint16_t *dip, int32_t *region, int32_t *cnt_off,
                  uint32_t *cnt, int64_t cnt_len, int32_t *status,
                  void *ws, size_t ws_bytes, cudaStream_t stream);

/* Regions with the paper's own tie rule (Section 3: R is built
 * incrementally while the distances are computed, a tie going to the
 * partition that is smallest at that moment), instead of ssm_aggregate's lowest pivot
 * index.  Reading: nodes join in the order a multi-source search settles
 * them -- increasing distance to their nearest pivots, equal distances by
 * increasing node id; a node with one nearest pivot joins it, a node with
 * several joins the one whose region has the fewest members at that moment
 * (lowest index on equal sizes).  Writes region[n]; asynchronous.  The
 * walk over tied nodes is sequential (one thread, region sizes in shared
 * memory), so this is slower than ssm_aggregate on graphs with many ties.
 * 1 <= k <= 8192.  Workspace ssm_regions_smallest_workspace(n).
 * ssm_aggregate_regions then builds cnt_off[k+1] and cnt for GIVEN regions
 * (ecc_a = max d_ia over the nodes of region a): synchronous; it stores the
 * table length in *cnt_len (host) and returns SSM_E_NOMEM if it exceeds
 * cnt_cap (cnt untouched; cnt may be NULL when cnt_cap is 0).  Workspace
 * ssm_aggregate_workspace(k).  Device error SSM_E_ARG for a region id
 * outside 0..k-1. */
size_t ssm_regions_smallest_workspace(int32_t n);
int ssm_regions_smallest(int32_t n, int32_t k, const uint16_t *dip, int32_t *region, int32_t *status,
                         void *ws, size_t ws_bytes, cudaStream_t stream);
int ssm_aggregate_regions(int32_t n, int32_t k, const uint16_t *dip, const int32_t *region, int32_t *cnt_off,
                          uint32_t *cnt, int64_t cnt_cap, int64_t *cnt_len, int32_t *status,
                          void *ws, size_t ws_bytes, cudaStream_t stream);

/* ssm_aggregate without any workspace, for callers that cannot allocate
 * device memory: for example a serving process that reserved its whole device
 * memory budget up front and admits work against it byte by byte, or code
 * that runs where the CUDA allocator must not be entered (a host callback, a
 * library whose memory comes from another allocator).  The paper has no
 * counterpart; this is a property of the library, not of the method.
 * Same results as ssm_aggregate.  Its scratch (one word per pivot) is a fixed
 * array in device memory that every GPU loading the library keeps until the
 * process exits, so it handles at most 4096 pivots (SSM_E_ARG beyond).  The
 * first call on each device looks up that array's address, with the device
 * current; make that first call before capturing the stream into a CUDA graph.
 * All calls share the array: calls that overlap on the GPU (other streams or
 * other threads) race and must be serialised by the caller.
 * Synchronous: computes region[n] and the table length, stores the length in
 * *cnt_len (host), and returns SSM_E_NOMEM if it exceeds cnt_cap (cnt untouched;
 * call again with cnt of that size, cnt may be NULL when cnt_cap is 0);
 * otherwise fills cnt_off[k+1] and cnt[*cnt_len] as ssm_aggregate does.
 * Calls no allocating function of CUDA or of any other library. */
int ssm_aggregate_noalloc(int32_t n, int32_t k, const uint16_t *dip, int32_t *region, int32_t *cnt_off,
                          uint32_t *cnt, int64_t cnt_cap, int64_t *cnt_len, int32_t *status,
                          cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Initial layout (Algorithm 1 lines 3-4): PivotMDS over the k pivots
 * (Brandes and Pich 2007), then, if rescale != 0, a uniform scale so that the
 * edge lengths of the layout sum to m (unit edge lengths).
 *   delta_ia = d_ia^2, C = -1/2 J_n Delta J_k (double centring),
 *   v1, v2 = eigenvectors of the two largest eigenvalues of C^T C (k x k, FP64),
 *   each signed so its largest-magnitude entry (lowest index on a tie) is positive,
 *   x_i = ((C v1)_i, (C v2)_i).
 * Writes pos[2n] (float or double by precision 32/64) and, if eig is not NULL,
 * eig[4] (device, double): the two eigenvalues, the number of subspace
 * iterations used and the final relative residual max_j ||B v_j - l_j v_j|| / l_1.
 * 2 <= k <= 1024.
 * Device errors: SSM_E_NUMERIC (eigen-solve did not converge or zero layout).
 * ------------------------------------------------------------------- */
size_t ssm_pivotmds_workspace(int32_t n, int32_t k);
int ssm_pivotmds(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                 const uint16_t *dip, void *pos, int32_t precision, int32_t rescale,
                 double *eig, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * The dense contraction of PivotMDS (Algorithm 1 line 3): the integer Gram
 * matrix of the squared pivot distances,
 *   G[a][b] = sum_i d_ia^2 d_ib^2   (exact, 128-bit unsigned),
 * on which ssm_pivotmds applies the double centring at the k x k level.
 * Writes g_lo[k*k], g_hi[k*k] (device, uint64): entry a*k + b holds the low
 * and high 64 bits of G[a][b] for a <= b; entries with a > b are zero.  The
 * call zeroes both arrays itself.  Runs on the tensor cores (digit planes in
 * FP16 -- one 7-bit digit when every d^2 is below 128, 5-bit digits
 * otherwise -- with FP32 accumulation of exact integers).  1 <= k <= 1024.
 * Device errors: SSM_E_TIMEOUT (a tensor-core wait ran out).
 * ------------------------------------------------------------------- */
size_t ssm_gram_workspace(int32_t n, int32_t k);
int ssm_gram(int32_t n, int32_t k, const uint16_t *dip, uint64_t *g_lo, uint64_t *g_hi, int32_t *status,
             void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Stress majorization (Eq. 4; Algorithm 1 lines 5-10), Jacobi schedule:
 * each iteration computes every x_i^{t+1} from X^t,
 *   x_i^{t+1} = [ sum_{j in N(i)} (x_j + (x_i - x_j)/r_ij)
 *               + sum_{a: d_ia >= 2} w'_ia (x_pa + d_ia (x_i - x_pa)/r_ia) ]
 *             / [ deg(i) + sum_{a: d_ia >= 2} w'_ia ],
 *   w'_ia = cnt[cnt_off[a] + min(floor(d_ia/2), ecc_a)] / d_ia^2,
 * where r = ||x_i - x_j|| and a term with r == 0 contributes w * x_j only.
 * Runs `iters` iterations on pos in place (precision 32: float, 64: double).
 * After each iteration the relative change ||X^{t+1}-X^t||_F / ||X^t||_F is
 * reduced in FP64; if tol > 0 the remaining iterations are skipped on the
 * device once it falls below tol.  Writes *iters_done (device int32) and
 * *rel_change (device double, the last computed change).  cnt_off and cnt are
 * the tables of ssm_aggregate, cnt_len = cnt_off[k] (from ssm_aggregate_size);
 * m is the edge count (colidx has 2m entries).  1 <= iters, 1 <= k <= 4096.
 * Precision 32 chooses its form on the host from three numbers, hints[0] =
 * the largest d_ip entry, hints[1] / hints[2] = the rows with 33..1024 /
 * more than 1024 entries: when k * (max d + 1) weight pairs fit in shared
 * memory the sweep uses a full (w', w' d) table, otherwise a table of s
 * clamped at 2 ecc_a + 2; the neighbour sums of each iteration are taken by
 * one thread, warp or block per row by length.  hints (host int32[3]) come
 * from ssm_aggregate_size (dip_max) and ssm_build_graph (row_classes), both
 * synchronous anyway, or from ssm_iterate_hints (synchronous); with hints
 * the call is asynchronous, with hints == NULL it computes them and waits
 * once for `stream`.  Wrong hints give SSM_E_ARG where they are out of
 * range and wrong results otherwise. 
 * ------------------------------------------------------------------- */
size_t ssm_iterate_workspace(int32_t n, int64_t m, int32_t k, int64_t cnt_len, int32_t precision);
int ssm_iterate(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                const int32_t *pivots, const uint16_t *dip, const int32_t *cnt_off,
                const uint32_t *cnt, int64_t cnt_len, void *pos, int32_t precision, int32_t iters,
                double tol, int32_t *iters_done, double *rel_change, int32_t *status,
                const int32_t *hints, void *ws, size_t ws_bytes, cudaStream_t stream);
int ssm_iterate_hints(int32_t n, const int32_t *rowptr, int32_t k, const uint16_t *dip, int32_t *hints,
                      void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * The sparse model's update of Eq. 4 in the paper's own order (Algorithm 1
 * lines 6-10): nodes 0..n-1 in turn, each moved in place from the positions
 * already moved (Gauss-Seidel), in FP64 -- the order the paper uses, kept as
 * a quality reference beside the Jacobi schedule of ssm_iterate.  Arguments
 * as for ssm_iterate; pos is double[2n]; rel_change (device double) receives
 * the relative change of the last sweep.  One block of 1024 threads sums each
 * node's deg(i) + k terms (ascending per thread, then a fixed-order tree), so
 * a sweep takes about n block steps.  Workspace ssm_iterate_gs_workspace(n).
 * Device error SSM_E_ARG (a pivot id outside 0..n-1).  1 <= k <= 65535.
 * ------------------------------------------------------------------- */
size_t ssm_iterate_gs_workspace(int32_t n);
int ssm_iterate_gs(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, int32_t k,
                   const int32_t *pivots, const uint16_t *dip, const int32_t *cnt_off, const uint32_t *cnt,
                   double *pos, int32_t iters, double *rel_change, int32_t *status,
                   void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Full stress majorization (Section 3, the localized update before Eq. 4;
 * the sparse model with k = n reduces to it): every node moves to
 *   x_i = sum_{j != i} w_ij (x_j + d_ij (x_i - x_j)/r_ij) / sum_{j != i} w_ij,
 * w_ij = d_ij^-2 (a term with r_ij == 0 adds w_ij x_j), over the all-pairs
 * hop distances D[n*n] (uint16, D[i*n + j] = d_ij, symmetric; for example
 * ssm_pivot_bfs with every node as a source, n <= 65535).
 * order 0: Jacobi (every node from the previous iterate), precision 32 or 64
 * (FP64 rounds each operation as the oracle does: bit-identical results);
 * order 1: Gauss-Seidel (nodes 0..n-1 in turn, in place -- the order under
 * which full stress decreases monotonically), precision 64 only.
 * Runs `iters` sweeps on pos in place; rel_change (device double) receives
 * the relative change of the last sweep.  O(n^2) per sweep; meant for the
 * graph sizes of the paper's comparisons (about 1e3 to 2e4 nodes).
 * Workspace ssm_full_iterate_workspace(n, precision).
 * Device error SSM_E_DISCONNECTED (an entry 0xFFFF off the diagonal).
 * ------------------------------------------------------------------- */
size_t ssm_full_iterate_workspace(int32_t n, int32_t precision);
int ssm_full_iterate(int32_t n, const uint16_t *D, void *pos, int32_t precision, int32_t order, int32_t iters,
                     double *rel_change, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Batched sweeps: the Jacobi sweeps of Eq. 4 (Algorithm 1 lines 5-10) for G
 * independent small graphs in one CUDA-graph launch of one persistent kernel.
 * Each graph is prepared as for ssm_iterate (CSR, pivots, d_ip, cnt_off, cnt)
 * and packed into shared arrays; ssm_batch_graph gives, per graph, its sizes
 * and where its pieces start in the packed arrays (element offsets):
 *   rowptr[row_off .. row_off + n]   local row offsets (0 .. 2m, into colidx at col_off)
 *   colidx[col_off ..]               local node ids 0..n-1
 *   pivots[piv_off .. + k]           local node ids
 *   dip[dip_off .. + k n]            pivot-major uint16, as ssm_pivot_bfs writes it
 *   cnt_off[cnt_off_off .. + k + 1]  local offsets into cnt at cnt_base, cnt_len = cnt_off[k]
 *   pos[2 node_off .. + 2 n]         float (x, y) pairs, updated in place
 * Graphs have 1 <= n <= 12288 nodes and 1 <= k <= min(n, 1024) pivots.  Each
 * graph runs `iters` iterations (FP32, the clamped s-table form of the
 * single-graph sweep evaluated about x_i, neighbour terms in ascending column
 * order) in one block with its positions in shared memory; rel_change[g]
 * (device double) gets the relative change of graph g's last iteration.
 * Graphs fall into three size classes (n <= 1024, <= 4096, <= 12288), each
 * launched with its own shape: threads = 128, 256 or 512 fixes the block
 * size, nodes_per_lane = 2 or 4 the tile shape (64- or 128-node tiles); 0
 * tunes that parameter per class on this batch (a few iterations per
 * candidate on a scratch copy of the positions, timed with CUDA events) and
 * keeps the choice for the process, per class fingerprint (largest n,
 * largest k, table size, graph count, sum of n k), so a batch of the same
 * shape is not tuned again.  threads fixed and nodes_per_lane 0 means 2.
 * shape_used (host int32[2], may be NULL) gets the block size and nodes per
 * lane of the class with the most work.  Synchronous while it tunes, else
 * asynchronous on `stream` (the descriptors are copied before the call
 * returns).  Workspace: ssm_batch_iterate_workspace(G, graphs).
 * Device errors: SSM_E_NUMERIC (non-finite weights), SSM_E_GRAPH (a pivot or
 * column id outside its graph).
 * ------------------------------------------------------------------- */
typedef struct {
  int32_t n, k, cnt_len, reserved;
  int64_t node_off, row_off, col_off, piv_off, dip_off, cnt_off_off, cnt_base;
} ssm_batch_graph;
size_t ssm_batch_iterate_workspace(int32_t G, const ssm_batch_graph *graphs);
/* Batched preparation of the graphs above (Algorithm 1 lines 1-4 for G
 * small graphs in two launches, one block per graph): from edge lists to
 * the packed arrays ssm_batch_iterate reads.  Graph g has n nodes (1..12288),
 * k max/min-sp pivots (2 <= k <= min(n, 100); start node 0), and m_in edges
 * src/dst[edge_off .. edge_off + m_in) with local ids.
 * ssm_batch_pivots (synchronous): builds each CSR (rowptr / colidx with room
 * for 2 m_in entries per graph, packed as the out descriptors say), the k
 * pivots (ties to the lowest id), d_ip, regions (ties to the lowest pivot
 * index) and the eccentricities ecc[piv_off + a]; fills out[g] (offsets,
 * cnt_len and cnt_base, with the count tables packed in graph order) and
 * m_out[g] (host, edges after deduplication; may be NULL).  Device errors
 * are read back and returned: SSM_E_GRAPH, SSM_E_DISCONNECTED.
 * ssm_batch_layout_init (asynchronous): from those, cnt_off / cnt (as
 * ssm_aggregate), PivotMDS (exact integer Gram matrix, FP64 eigenpairs by a
 * parallel cyclic Jacobi method) and the rescale to unit mean edge length
 * into pos (float x, y pairs at 2 node_off); eig (device double [2G], may be
 * NULL) gets the two eigenvalues.  m[g] (host) = the edge counts.  Both use
 * a workspace of ssm_batch_prepare_workspace(G, in) bytes (the same one).
 */
typedef struct {
  int32_t n, k;
  int64_t m_in, edge_off;
} ssm_batch_input;
size_t ssm_batch_prepare_workspace(int32_t G, const ssm_batch_input *in);
int ssm_batch_pivots(int32_t G, const ssm_batch_input *in, const int32_t *src, const int32_t *dst,
                     ssm_batch_graph *out, int32_t *rowptr, int32_t *colidx, int32_t *pivots, uint16_t *dip,
                     int32_t *region, int32_t *ecc, int64_t *m_out, int32_t *status, void *ws, size_t ws_bytes,
                     cudaStream_t stream);
int ssm_batch_layout_init(int32_t G, const ssm_batch_graph *graphs, const int64_t *m, const int32_t *rowptr,
                          const int32_t *colidx, const uint16_t *dip, const int32_t *region, const int32_t *ecc,
                          int32_t *cnt_off, uint32_t *cnt, float *pos, double *eig, int32_t *status, void *ws,
                          size_t ws_bytes, cudaStream_t stream);

int ssm_batch_iterate(int32_t G, const ssm_batch_graph *graphs, const int32_t *rowptr, const int32_t *colidx,
                      const int32_t *pivots, const uint16_t *dip, const int32_t *cnt_off, const uint32_t *cnt,
                      float *pos, int32_t iters, double *rel_change, int32_t threads, int32_t nodes_per_lane,
                      int32_t *shape_used, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Layout quality measures (Section 4).
 * ssm_procrustes: the Procrustes statistic (Sibson 1978) of layouts X and Y
 * of the same n nodes (precision 32: float[2n], 64: double[2n]): both
 * centred, Y fitted by a uniform scale and a proper rotation (the paper
 * notes that its analysis cannot resolve reflections):
 *   P = 1 - T^2 / (||Xc||^2 ||Yc||^2),  T = sqrt((m11 + m22)^2 + (m12 - m21)^2),
 *   m_ab = sum_i xc_ia yc_ib;  P in [0, 1], 0 for a perfect match.
 * out[3] (device double) = {P, scale, angle} with Y ~ scale R(angle) X +
 * translation.  One block, FP64 sums in a fixed order; no workspace.
 * ssm_hull_error: the convex-hull error of Fig. 4 for hop radius kh: for
 * every node v, B = {w : d_vw <= kh} from the all-pairs table D[n*n], H the
 * convex hull of B's positions, err_v = |{u not in B : x_u inside or on H}|
 * / (n - |B|) (0 when B holds every node); per_node[n] (device double, may
 * be NULL) and *mean (device double, the mean in node order).  Hull and
 * inside tests use FP64 orientation tests.  A ball whose points outside the
 * quadrilateral of its four extreme points number above 4096 is reported
 * as SSM_E_ARG (err_v = -1).  Workspace ssm_hull_error_workspace(n).
 * ssm_gabriel_jaccard: the Gabriel-graph comparison of Section 4: the
 * Gabriel graphs of layouts A and B (u ~ v iff no third point lies strictly
 * inside the disc with diameter uv, tested as |2w - a - b|^2 < |a - b|^2 in
 * FP64 with a the lower id, so identical positions are adjacent), then for
 * every node v the Jaccard coefficient |N_A ^ N_B| / |N_A u N_B| of the
 * node sets within kh >= 1 hops of v in each graph (v excluded; 1 when both
 * are empty); per_node[n] (may be NULL) and *mean (device doubles, the mean
 * in node order).  Limits, reported as SSM_E_ARG in *status: 256 Gabriel
 * neighbours per node (identical positions form cliques), 512 points met
 * while bounding one node's neighbour region on the grid, 512 nodes in one
 * kh-neighbourhood.  Workspace ssm_gabriel_jaccard_workspace(n) (about 6 KB
 * per node).
 * ------------------------------------------------------------------- */
int ssm_procrustes(int32_t n, const void *X, const void *Y, int32_t precision, double *out, cudaStream_t stream);
size_t ssm_hull_error_workspace(int32_t n);
int ssm_hull_error(int32_t n, const uint16_t *D, const void *pos, int32_t precision, int32_t kh, double *per_node,
                   double *mean, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t ssm_gabriel_jaccard_workspace(int32_t n);
int ssm_gabriel_jaccard(int32_t n, const void *posA, const void *posB, int32_t precision, int32_t kh,
                        double *per_node, double *mean, int32_t *status, void *ws, size_t ws_bytes,
                        cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Weighted graphs (Algorithm 1 line 2: weighted MSSP; Section 3's weights
 * with general edge lengths).  Edge lengths are float32, finite, at least
 * FLT_MIN, with n * (largest length) < 1e37.  A distance d_ij is the least
 * float32 path sum: along a path walked from the source, each edge's length
 * is added to the running sum and rounded to float32; d_ij is the minimum
 * over paths (any correct search reaches this value, so it is exact and
 * reproducible).  Tables of distances are float32, pivot-major [k][n].
 *
 * ssm_edge_lengths: elen[2m] for the CSR (rowptr, colidx) that
 *   ssm_build_graph made from the same edge list src/dst[m_in] with lengths
 *   len[m_in]: elen[t] is the length of edge (i, colidx[t]); a repeated edge
 *   keeps its shortest length.  Bad lengths: SSM_E_ARG; an edge missing
 *   from the CSR: SSM_E_GRAPH (both in *status).  Workspace 256 bytes.
 * ssm_pivot_sssp: dist[a*n + v] = d(sources[a], v) for a < k (one
 *   label-correcting search per source, a block per source); an unreachable
 *   node gives SSM_E_DISCONNECTED.  Workspace ssm_pivot_sssp_workspace(n, k).
 * ssm_select_pivots_weighted: max/min sp (Section 4.1) on weighted
 *   distances: pivots[0] = start, then the node farthest from the pivots so
 *   far (ties to the lowest id), each search pruned to the nodes the new
 *   pivot is strictly closer to.  Workspace ..._workspace(n, k).
 * ssm_weighted_counts: region[i] = the lowest pivot index a minimising
 *   d_ia; s_tab[a*n + i] = |{j in R(a) : 2 d_ja <= d_ia}| (float32 test),
 *   0 where pivots[a] is i or a neighbour of i (the pivot sum of Eq. 4 runs
 *   over P \ N(i)).  The adapted weight is w'_ia = s / d_ia^2.  Workspace
 *   ssm_weighted_counts_workspace(n, k) (a sort of n 64-bit keys).
 * ssm_pivotmds_weighted: as ssm_pivotmds from the float32 table
 *   (delta = d^2 in FP64; C^T C from column-centred FP64 sums), rescaled so
 *   that sum_E ||x_i - x_j|| = sum_E l_ij when rescale != 0.
 * ssm_iterate_weighted: `iters` Jacobi updates of Eq. 4 with
 *   w_ij = l_ij^-2, d_ij = l_ij on the edges and w'_ia = s_ia / d_ia^2 on
 *   the pivots (skipped where s_ia = 0), in place on pos (float2 or
 *   double2 by precision; FP64 rounds every operation as written, in the
 *   order of the plain definition); *rel_change (device double) receives
 *   ||X^{t+1} - X^t||_F / ||X^t||_F of the last update.
 *   FP32 forms w' = s / d^2 once per call in the workspace and takes 1/r
 *   from rsqrt.  Workspace ssm_iterate_weighted_workspace(n, k, precision).
 * ssm_stress_weighted: ssm_stress with weighted distances (exhaustive when
 *   nsources == 0, else the same sampled pair list).
 * ------------------------------------------------------------------- */
int ssm_edge_lengths(int32_t n, int64_t m_in, const int32_t *src, const int32_t *dst, const float *len, int64_t m,
                     const int32_t *rowptr, const int32_t *colidx, float *elen, int32_t *status, void *ws,
                     size_t ws_bytes, cudaStream_t stream);
size_t ssm_pivot_sssp_workspace(int32_t n, int32_t k);
int ssm_pivot_sssp(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t k,
                   const int32_t *sources, float *dist, int32_t *status, void *ws, size_t ws_bytes,
                   cudaStream_t stream);
size_t ssm_select_pivots_weighted_workspace(int32_t n, int32_t k);
int ssm_select_pivots_weighted(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, const float *elen,
                               int32_t k, int32_t start, int32_t *pivots, int32_t *status, void *ws, size_t ws_bytes,
                               cudaStream_t stream);
size_t ssm_weighted_counts_workspace(int32_t n, int32_t k);
int ssm_weighted_counts(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t k, const int32_t *pivots,
                        const float *dist, int32_t *region, uint32_t *s_tab, int32_t *status, void *ws,
                        size_t ws_bytes, cudaStream_t stream);
size_t ssm_pivotmds_weighted_workspace(int32_t n, int32_t k);
int ssm_pivotmds_weighted(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t k,
                          const float *dist, void *pos, int32_t precision, int32_t rescale, double *eig,
                          int32_t *status, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t ssm_iterate_weighted_workspace(int32_t n, int32_t k, int32_t precision);
int ssm_iterate_weighted(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, int32_t k,
                         const int32_t *pivots, const float *dist, const uint32_t *s_tab, void *pos,
                         int32_t precision, int32_t iters, double *rel_change, int32_t *status, void *ws,
                         size_t ws_bytes, cudaStream_t stream);
size_t ssm_stress_weighted_workspace(int32_t n, int32_t nsources);
int ssm_stress_weighted(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *elen, const void *pos,
                        int32_t precision, int32_t nsources, int32_t ntargets, uint64_t seed, double *out,
                        double *sums, int32_t *status, void *ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------
 * Full stress of a layout (Eq. 1, w_ij = d_ij^-2) with optimal scaling
 * (Section 4: drawings are rescaled to their lowest stress).
 * nsources == 0: exhaustive over all pairs i < j (a BFS from every node).
 * nsources  > 0: nsources * ntargets sampled pairs: source j is node
 *   (hi32(u) * n) >> 32 for u = splitmix64 value j of stream `seed`, and
 *   target l of source j is t' + (t' >= source) with t' = (hi32(u) * (n-1)) >> 32
 *   for u = value nsources + j*ntargets + l (value c of the stream is the
 *   splitmix64 output for state seed + (c+1) * 0x9E3779B97F4A7C15).
 * Writes out[4] (device double): {raw, alpha*, scaled, normalized}, with
 *   raw = sum (r-d)^2/d^2, alpha* = S1/S2 (S1 = sum r/d, S2 = sum r^2/d^2),
 *   scaled = N - S1^2/S2 (N pairs), normalized = scaled / C(n,2);
 *   sampled sums are scaled by C(n,2)/N.  sums[4] (optional, device double)
 *   receives {sum (r-d)^2/d^2, S1, S2, N} before scaling.
 * All sums are FP64 in a fixed order.  Device errors: SSM_E_DISCONNECTED,
 * SSM_E_DIST_OVERFLOW, SSM_E_TIMEOUT.  2 <= n.
 * ------------------------------------------------------------------- */
size_t ssm_stress_workspace(int32_t n, int64_t m, int32_t nsources, int32_t ntargets);
int ssm_stress(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx, const void *pos,
               int32_t precision, int32_t nsources, int32_t ntargets, uint64_t seed,
               double *out, double *sums, int32_t *status,
               void *ws, size_t ws_bytes, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* SSM_H */
