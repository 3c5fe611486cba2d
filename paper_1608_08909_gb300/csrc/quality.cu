// Layout quality measures of Section 4, computed on the GPU:
//  * the Procrustes statistic of two layouts (Sibson 1978; the paper's
//    second measure after normalized stress): both centred, one fitted to
//    the other by a uniform scale and a proper rotation (the paper notes
//    that its analysis cannot resolve reflections),
//      P = 1 - T^2 / (||Xc||^2 ||Yc||^2),  T = sqrt((m11 + m22)^2 + (m12 - m21)^2),
//    m_ab = sum_i xc_ia yc_ib; one block, FP64 sums in a fixed order;
//  * the convex-hull error of Fig. 4: for node v the ball B = {w : d_vw <= kh}
//    of graph distances, H the convex hull of its positions, and
//    err_v = |{u not in B : x_u inside or on H}| / (n - |B|).  A block per
//    node: the ball is compacted from row v of the all-pairs table, thinned
//    (points strictly inside the quadrilateral of its four extreme points
//    cannot be hull vertices), sorted by (x, y, id) in shared memory, and the
//    hull built by Andrew's monotone chain in one thread; then the block
//    counts the other nodes inside or on the hull.  Every predicate is the
//    same FP64 expression as the oracle's, so the counts are exact matches.
#include <algorithm>

#include "common.cuh"

namespace ssm {

constexpr int kQThreads = 256;
constexpr int kHullCap = 4096;  // ball points a block sorts in shared memory (after thinning)

template <class T>
__device__ __forceinline__ T q_block_sum(T v, T *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = (T)0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];  // every thread, same order
  return s;
}

template <class V>
__global__ void __launch_bounds__(1024) k_procrustes(int32_t n, const V *__restrict__ X, const V *__restrict__ Y,
                                                     double *__restrict__ out) {
  __shared__ double red[32];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const V x = X[i], y = Y[i];
    s[0] += (double)x.x;
    s[1] += (double)x.y;
    s[2] += (double)y.x;
    s[3] += (double)y.y;
  }
  double mean[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) mean[q] = q_block_sum(s[q], red) / (double)n;
  double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const V x = X[i], y = Y[i];
    const double x0 = (double)x.x - mean[0], x1 = (double)x.y - mean[1];
    const double y0 = (double)y.x - mean[2], y1 = (double)y.y - mean[3];
    t[0] += x0 * y0;
    t[1] += x0 * y1;
    t[2] += x1 * y0;
    t[3] += x1 * y1;
    t[4] += x0 * x0 + x1 * x1;
    t[5] += y0 * y0 + y1 * y1;
  }
  double m[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) m[q] = q_block_sum(t[q], red);
  if (threadIdx.x == 0) {
    const double a = m[0] + m[3], b = m[1] - m[2];
    const double T = sqrt(a * a + b * b);
    if (!(m[4] > 0.0) || !(m[5] > 0.0)) {
      out[0] = 1.0;
      out[1] = 0.0;
      out[2] = 0.0;
    } else {
      out[0] = 1.0 - T * T / (m[4] * m[5]);
      out[1] = T / m[4];
      out[2] = atan2(b, a);
    }
  }
}

// (b - a) x (c - a) exactly as the oracle writes it (no contraction)
__device__ __forceinline__ double q_cross(double ax, double ay, double bx, double by, double cx, double cy) {
  const double ux = __dsub_rn(bx, ax), uy = __dsub_rn(by, ay), vx = __dsub_rn(cx, ax), vy = __dsub_rn(cy, ay);
  return __dsub_rn(__dmul_rn(ux, vy), __dmul_rn(uy, vx));
}

struct HullPt {
  double x, y;
  int id;
  int pad;
};

__device__ __forceinline__ bool q_less(const HullPt &a, const HullPt &b) {
  if (a.x != b.x) return a.x < b.x;
  if (a.y != b.y) return a.y < b.y;
  return a.id < b.id;
}

template <class V>
__device__ __forceinline__ void q_load(const V *pos, int i, double &x, double &y) {
  const V p = pos[i];
  x = (double)p.x;
  y = (double)p.y;
}

template <class V>
__global__ void __launch_bounds__(kQThreads) k_hull_error(int32_t n, const uint16_t *__restrict__ D,
                                                          const V *__restrict__ pos, int32_t kh,
                                                          int32_t *__restrict__ scratch, double *__restrict__ per,
                                                          int32_t *__restrict__ status) {
  extern __shared__ __align__(16) unsigned char q_smem[];
  HullPt *pts = reinterpret_cast<HullPt *>(q_smem);             // [kHullCap]
  int *hull = reinterpret_cast<int *>(pts + kHullCap);          // [kHullCap + 1]
  __shared__ int s_cnt, s_h;
  __shared__ unsigned long long s_in;
  __shared__ int s_ext[4];
  __shared__ double s_bb[4];
  int *ball = scratch + (size_t)blockIdx.x * n;
  for (int v = blockIdx.x; v < n; v += gridDim.x) {
    const uint16_t *row = D + (size_t)v * n;
    // 1. the ball, compacted (any order: it is sorted below)
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int w0 = 0; w0 < n; w0 += blockDim.x) {
      const int w = w0 + threadIdx.x;
      const bool in = w < n && (int)row[w] <= kh;
      const unsigned mask = __ballot_sync(0xffffffffu, in);
      int base = 0;
      if ((threadIdx.x & 31) == 0 && mask) base = atomicAdd(&s_cnt, __popc(mask));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (in) ball[base + __popc(mask & ((1u << (threadIdx.x & 31)) - 1u))] = w;
    }
    __syncthreads();
    const int m = s_cnt;
    if (m == n) {
      if (threadIdx.x == 0) per[v] = 0.0;
      __syncthreads();
      continue;
    }
    // 2. thin: the extreme points (least x, greatest x, least y, greatest y;
    // ties by the (x, y, id) order) span a quadrilateral; points strictly
    // inside it are not hull vertices
    int keep = m;
    if (m > kHullCap) {
      HullPt e[4];
      bool have = false;
      for (int t = threadIdx.x; t < m; t += blockDim.x) {
        HullPt p;
        q_load(pos, ball[t], p.x, p.y);
        p.id = ball[t];
        if (!have) {
          e[0] = e[1] = e[2] = e[3] = p;
          have = true;
        } else {
          if (q_less(p, e[0])) e[0] = p;
          if (q_less(e[1], p)) e[1] = p;
          if (p.y < e[2].y || (p.y == e[2].y && q_less(p, e[2]))) e[2] = p;
          if (p.y > e[3].y || (p.y == e[3].y && q_less(e[3], p))) e[3] = p;
        }
      }
      if (threadIdx.x == 0) s_ext[0] = s_ext[1] = s_ext[2] = s_ext[3] = -1;
      __syncthreads();
      // one thread folds the per-thread extremes in thread order (the result
      // is the unique extreme point under the order, whatever the folding)
      for (int t = 0; t < (int)blockDim.x; ++t) {
        if ((int)threadIdx.x == t && have) {
          for (int q = 0; q < 4; ++q) {
            HullPt cur;
            if (s_ext[q] < 0) {
              s_ext[q] = e[q].id;
              continue;
            }
            q_load(pos, s_ext[q], cur.x, cur.y);
            cur.id = s_ext[q];
            bool better;
            if (q == 0) better = q_less(e[q], cur);
            else if (q == 1) better = q_less(cur, e[q]);
            else if (q == 2) better = e[q].y < cur.y || (e[q].y == cur.y && q_less(e[q], cur));
            else better = e[q].y > cur.y || (e[q].y == cur.y && q_less(cur, e[q]));
            if (better) s_ext[q] = e[q].id;
          }
        }
        __syncthreads();
      }
      // quadrilateral in counter-clockwise order: least x, least y, greatest x, greatest y
      double qx[4], qy[4];
      const int ord[4] = {0, 2, 1, 3};
      for (int q = 0; q < 4; ++q) q_load(pos, s_ext[ord[q]], qx[q], qy[q]);
      if (threadIdx.x == 0) s_cnt = 0;
      __syncthreads();
      for (int t0 = 0; t0 < m; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        bool out = false;
        int id = 0;
        if (t < m) {
          id = ball[t];
          double x, y;
          q_load(pos, id, x, y);
          bool strict = true;
          for (int q = 0; q < 4; ++q)
            strict = strict && q_cross(qx[q], qy[q], qx[(q + 1) & 3], qy[(q + 1) & 3], x, y) > 0.0;
          out = !strict;
        }
        __syncthreads();  // every read of ball[t0 ..] is done before the rewrite below
        const unsigned mask = __ballot_sync(0xffffffffu, out);
        int base = 0;
        if ((threadIdx.x & 31) == 0 && mask) base = atomicAdd(&s_cnt, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (out) ball[base + __popc(mask & ((1u << (threadIdx.x & 31)) - 1u))] = id;
        __syncthreads();
      }
      keep = s_cnt;
      if (keep > kHullCap) {
        if (threadIdx.x == 0) {
          dev_fail(status, SSM_E_ARG);
          per[v] = -1.0;
        }
        __syncthreads();
        continue;
      }
    }
    // 3. sort by (x, y, id): bitonic over the next power of two
    int P = 1;
    while (P < keep) P <<= 1;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
      if (t < keep) {
        HullPt p;
        q_load(pos, ball[t], p.x, p.y);
        p.id = ball[t];
        pts[t] = p;
      } else {
        pts[t] = HullPt{__longlong_as_double(0x7ff0000000000000ll), __longlong_as_double(0x7ff0000000000000ll),
                        0x7fffffff, 0};
      }
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
          const int o = t ^ stride;
          if (o > t) {
            const bool up = (t & size) == 0;
            const HullPt a = pts[t], b = pts[o];
            if (q_less(b, a) == up) {
              pts[t] = b;
              pts[o] = a;
            }
          }
        }
        __syncthreads();
      }
    // 4. Andrew's monotone chain, one thread, the oracle's rule
    if (threadIdx.x == 0) {
      int h = 0;
      for (int t = 0; t < keep; ++t) {
        while (h >= 2 && q_cross(pts[hull[h - 2]].x, pts[hull[h - 2]].y, pts[hull[h - 1]].x, pts[hull[h - 1]].y,
                                 pts[t].x, pts[t].y) <= 0.0)
          --h;
        hull[h++] = t;
      }
      const int lo = h + 1;
      for (int t = keep - 2; t >= 0; --t) {
        while (h >= lo && q_cross(pts[hull[h - 2]].x, pts[hull[h - 2]].y, pts[hull[h - 1]].x, pts[hull[h - 1]].y,
                                  pts[t].x, pts[t].y) <= 0.0)
          --h;
        hull[h++] = t;
      }
      if (h > 1) --h;
      s_h = h;
      double x0 = pts[hull[0]].x, x1 = x0, y0 = pts[hull[0]].y, y1 = y0;
      for (int e = 1; e < h; ++e) {
        x0 = fmin(x0, pts[hull[e]].x);
        x1 = fmax(x1, pts[hull[e]].x);
        y0 = fmin(y0, pts[hull[e]].y);
        y1 = fmax(y1, pts[hull[e]].y);
      }
      s_bb[0] = x0;
      s_bb[1] = x1;
      s_bb[2] = y0;
      s_bb[3] = y1;
      s_in = 0ull;
    }
    __syncthreads();
    // 5. the other nodes inside or on the hull
    const int h = s_h;
    unsigned long long cnt = 0;
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
      if ((int)row[u] <= kh) continue;
      double x, y;
      q_load(pos, u, x, y);
      bool in;
      if (h == 1) {
        in = x == pts[hull[0]].x && y == pts[hull[0]].y;
      } else if (h == 2) {
        const HullPt a = pts[hull[0]], b = pts[hull[1]];
        in = q_cross(a.x, a.y, b.x, b.y, x, y) == 0.0 && x >= fmin(a.x, b.x) && x <= fmax(a.x, b.x) &&
             y >= fmin(a.y, b.y) && y <= fmax(a.y, b.y);
      } else {
        in = !(x < s_bb[0] || x > s_bb[1] || y < s_bb[2] || y > s_bb[3]);
        for (int e = 0; in && e < h; ++e) {
          const HullPt a = pts[hull[e]], b = pts[hull[e + 1 < h ? e + 1 : 0]];
          if (q_cross(a.x, a.y, b.x, b.y, x, y) < 0.0) in = false;
        }
      }
      cnt += in ? 1ull : 0ull;
    }
    cnt = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_in, cnt);
    __syncthreads();
    if (threadIdx.x == 0) per[v] = (double)s_in / (double)(n - m);
    __syncthreads();
  }
}

// mean of the per-node errors in node order (as the oracle adds them)
__global__ void k_mean_in_order(int32_t n, const double *__restrict__ per, double *__restrict__ mean) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += per[i];
  *mean = s / (double)n;
}

}  // namespace ssm

SSM_API int ssm_procrustes(int32_t n, const void *X, const void *Y, int32_t precision, double *out,
                           cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !X || !Y || !out) return fail(SSM_E_ARG, "ssm_procrustes: null pointer or bad size");
  if (precision == 64)
    note_launch(), k_procrustes<double2><<<1, 1024, 0, s>>>(n, (const double2 *)X, (const double2 *)Y, out);
  else if (precision == 32)
    note_launch(), k_procrustes<float2><<<1, 1024, 0, s>>>(n, (const float2 *)X, (const float2 *)Y, out);
  else
    return fail(SSM_E_ARG, "ssm_procrustes: precision must be 32 or 64");
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

static int hull_blocks(int32_t n) { return (int)std::min<int64_t>(n, (int64_t)ssm::num_sms() * 2); }

SSM_API size_t ssm_hull_error_workspace(int32_t n) {
  if (n < 1) return 0;
  ssm::Carver c(nullptr, 0);
  c.take<int32_t>((size_t)hull_blocks(n) * n);
  c.take<double>((size_t)n);
  return c.size();
}

SSM_API int ssm_hull_error(int32_t n, const uint16_t *D, const void *pos, int32_t precision, int32_t kh,
                           double *per_node, double *mean, int32_t *status, void *ws, size_t ws_bytes,
                           cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !D || !pos || !mean || !status || !ws || kh < 0) return fail(SSM_E_ARG, "ssm_hull_error: bad argument");
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_hull_error: precision must be 32 or 64");
  Carver c(ws, ws_bytes);
  const int blocks = hull_blocks(n);
  int32_t *scratch = c.take<int32_t>((size_t)blocks * n);
  double *per_ws = c.take<double>((size_t)n);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_hull_error: workspace %zu bytes, need %zu", ws_bytes, c.size());
  double *per = per_node ? per_node : per_ws;
  const size_t smem = kHullCap * sizeof(HullPt) + (kHullCap + 1) * sizeof(int);
  if (precision == 64) {
    SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_hull_error<double2>));
    note_launch(), k_hull_error<double2><<<blocks, kQThreads, smem, s>>>(n, D, (const double2 *)pos, kh, scratch, per, status);
  } else {
    SSM_TRY_CUDA(allow_dynamic_smem((const void *)k_hull_error<float2>));
    note_launch(), k_hull_error<float2><<<blocks, kQThreads, smem, s>>>(n, D, (const float2 *)pos, kh, scratch, per, status);
  }
  note_launch(), k_mean_in_order<<<1, 32, 0, s>>>(n, per, mean);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}

// ---------------------------------------------------------------- Gabriel graphs
// Gabriel graph of a layout (Section 4, after Fig. 4): u, v adjacent iff no
// other point lies inside the disc with diameter uv (the open disc, so
// identical positions are adjacent, as the paper adds them).  GPU form, one
// thread per node u:
//  * the points sit in a uniform grid (about two per cell);
//  * u visits the grid in rings of cells around its own; every point w met
//    clips u's region {x : (x - w) . (w - u) <= 0 for all w}, which holds
//    every Gabriel neighbour of u (a point x beyond that line through w sees
//    w inside the disc with diameter ux); the visit stops once the ring's
//    distance exceeds the farthest vertex of the clipped region;
//  * the visited points that pass the half-plane tests (with a relative
//    slack, so rounding in the clipping never drops a neighbour) are
//    candidates, and each candidate v is decided exactly: no point of the
//    cells that overlap the disc with diameter uv lies inside it, tested by
//    the oracle's expression |2w - a - b|^2 < |a - b|^2 (a the lower id).
namespace ssm {

constexpr int kGabVisit = 512;  // points one node may visit
constexpr int kGabPoly = 64;    // vertices of the clipped region
constexpr int kGabDeg = 256;    // Gabriel neighbours per node (coincident groups are cliques)

struct GridView {
  double x0, y0, cs;
  int side;
  const int *start;  // [side*side + 1]
  const int *pts;    // [n] point ids by cell
};

template <class V>
__device__ __forceinline__ int cell_of(const GridView &g, double x, double y, int *cx, int *cy) {
  int ix = (int)floor((x - g.x0) / g.cs), iy = (int)floor((y - g.y0) / g.cs);
  ix = min(max(ix, 0), g.side - 1);
  iy = min(max(iy, 0), g.side - 1);
  *cx = ix;
  *cy = iy;
  return iy * g.side + ix;
}

template <class V>
__global__ void k_bbox(int32_t n, const V *__restrict__ pos, double *__restrict__ bb) {
  __shared__ double red[4][32];
  double mn0 = INFINITY, mx0 = -INFINITY, mn1 = INFINITY, mx1 = -INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const V p = pos[i];
    mn0 = fmin(mn0, (double)p.x);
    mx0 = fmax(mx0, (double)p.x);
    mn1 = fmin(mn1, (double)p.y);
    mx1 = fmax(mx1, (double)p.y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn0 = fmin(mn0, __shfl_xor_sync(0xffffffffu, mn0, o));
    mx0 = fmax(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
    mn1 = fmin(mn1, __shfl_xor_sync(0xffffffffu, mn1, o));
    mx1 = fmax(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = mn0;
    red[1][warp] = mx0;
    red[2][warp] = mn1;
    red[3][warp] = mx1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      red[0][0] = fmin(red[0][0], red[0][w]);
      red[1][0] = fmax(red[1][0], red[1][w]);
      red[2][0] = fmin(red[2][0], red[2][w]);
      red[3][0] = fmax(red[3][0], red[3][w]);
    }
    for (int q = 0; q < 4; ++q) bb[q] = red[q][0];
  }
}

template <class V>
__global__ void k_grid_count(int32_t n, const V *__restrict__ pos, const double *__restrict__ bb, int side,
                             int *__restrict__ cellid, int *__restrict__ count) {
  const double ext = fmax(bb[1] - bb[0], bb[3] - bb[2]);
  GridView g{bb[0], bb[2], ext > 0.0 ? ext / side : 1.0, side, nullptr, nullptr};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const V p = pos[i];
    int cx, cy;
    const int c = cell_of<V>(g, (double)p.x, (double)p.y, &cx, &cy);
    cellid[i] = c;
    atomicAdd(count + c, 1);
  }
}

// exclusive scan of the cell counts, one block
__global__ void __launch_bounds__(1024) k_grid_scan(int cells, const int *__restrict__ count, int *__restrict__ start,
                                                    int *__restrict__ cursor) {
  __shared__ int part[1024];
  const int per = (cells + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per, e = min(cells, b + per);
  int s = 0;
  for (int c = b; c < e; ++c) s += count[c];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int v = part[t];
      part[t] = acc;
      acc += v;
    }
    start[cells] = acc;
  }
  __syncthreads();
  int acc = part[threadIdx.x];
  for (int c = b; c < e; ++c) {
    start[c] = acc;
    cursor[c] = acc;
    acc += count[c];
  }
}

__global__ void k_grid_fill(int32_t n, const int *__restrict__ cellid, int *__restrict__ cursor, int *__restrict__ pts) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    pts[atomicAdd(cursor + cellid[i], 1)] = i;
}

// w strictly inside the disc with diameter ab, the oracle's expression (a the lower id)
template <class V>
__device__ __forceinline__ bool q_in_disc(const V *pos, int a, int b, int w) {
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  double ax, ay, bx, by, wx, wy;
  q_load(pos, a, ax, ay);
  q_load(pos, b, bx, by);
  q_load(pos, w, wx, wy);
  const double tx = __dsub_rn(__dsub_rn(__dmul_rn(2.0, wx), ax), bx);
  const double ty = __dsub_rn(__dsub_rn(__dmul_rn(2.0, wy), ay), by);
  const double ex = __dsub_rn(ax, bx), ey = __dsub_rn(ay, by);
  return __dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)) < __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
}

template <class V>
__global__ void __launch_bounds__(128) k_gabriel(int32_t n, const V *__restrict__ pos, GridView g,
                                                 const double *__restrict__ bb, int *__restrict__ nbr,
                                                 int *__restrict__ deg, int *__restrict__ visit_ws,
                                                 int32_t *__restrict__ status) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  const double ext = fmax(bb[1] - bb[0], bb[3] - bb[2]);
  g.x0 = bb[0];
  g.y0 = bb[2];
  g.cs = ext > 0.0 ? ext / g.side : 1.0;
  double ux, uy;
  q_load(pos, u, ux, uy);
  int cx, cy;
  cell_of<V>(g, ux, uy, &cx, &cy);
  // the clipped region, starting from the points' bounding box (every
  // neighbour lies in it), widened a little so rounding keeps the box's own
  // points inside
  double px[kGabPoly], py[kGabPoly], qxs[kGabPoly], qys[kGabPoly];
  const double pad = ext > 0.0 ? 1e-6 * ext : 1.0;
  int np = 4;
  px[0] = bb[0] - pad; py[0] = bb[2] - pad;
  px[1] = bb[1] + pad; py[1] = bb[2] - pad;
  px[2] = bb[1] + pad; py[2] = bb[3] + pad;
  px[3] = bb[0] - pad; py[3] = bb[3] + pad;
  int *visit = visit_ws + (size_t)u * kGabVisit;
  int nv = 0;
  bool overflow = false;
  for (int r = 0;; ++r) {
    // ring r of cells around (cx, cy)
    for (int dy = -r; dy <= r; ++dy)
      for (int dx = -r; dx <= r; ++dx) {
        if (max(abs(dx), abs(dy)) != r) continue;
        const int ix = cx + dx, iy = cy + dy;
        if (ix < 0 || iy < 0 || ix >= g.side || iy >= g.side) continue;
        const int c = iy * g.side + ix;
        for (int t = g.start[c]; t < g.start[c + 1]; ++t) {
          const int w = g.pts[t];
          if (w == u) continue;
          if (nv < kGabVisit) visit[nv++] = w;
          else overflow = true;
          double wx, wy;
          q_load(pos, w, wx, wy);
          const double ax = wx - ux, ay = wy - uy;  // keep x with (x - w) . a <= 0
          const double lim = wx * ax + wy * ay;
          if (ax == 0.0 && ay == 0.0) continue;
          // a clip that would need more than kGabPoly vertices is skipped:
          // the region stays a superset, so the stopping radius stays safe
          int nq = 0;
          bool full = false;
          for (int e = 0; e < np && !full; ++e) {
            const int f = e + 1 < np ? e + 1 : 0;
            const double se = px[e] * ax + py[e] * ay - lim, sf = px[f] * ax + py[f] * ay - lim;
            if (se <= 0.0) {
              if (nq < kGabPoly) {
                qxs[nq] = px[e];
                qys[nq] = py[e];
                ++nq;
              } else {
                full = true;
              }
            }
            if ((se < 0.0 && sf > 0.0) || (se > 0.0 && sf < 0.0)) {
              const double tt = se / (se - sf);
              if (nq < kGabPoly) {
                qxs[nq] = px[e] + tt * (px[f] - px[e]);
                qys[nq] = py[e] + tt * (py[f] - py[e]);
                ++nq;
              } else {
                full = true;
              }
            }
          }
          if (full || nq < 3) continue;
          np = nq;
          for (int e = 0; e < np; ++e) {
            px[e] = qxs[e];
            py[e] = qys[e];
          }
        }
      }
    double rmax = 0.0;
    for (int e = 0; e < np; ++e) rmax = fmax(rmax, sqrt((px[e] - ux) * (px[e] - ux) + (py[e] - uy) * (py[e] - uy)));
    // every point of ring r + 1 or beyond is at least r cells away from u
    if ((double)r * g.cs > rmax * (1.0 + 1e-9) + 1e-12 * ext) break;
    if (r > 2 * g.side) break;
  }
  // candidates: visited points on the kept side of every visited point's line
  // (relative slack), each then decided exactly
  int d = 0;
  for (int a = 0; a < nv; ++a) {
    const int v = visit[a];
    double vx, vy;
    q_load(pos, v, vx, vy);
    bool cand = true;
    for (int b = 0; b < nv && cand; ++b) {
      const int w = visit[b];
      if (w == v) continue;
      double wx, wy;
      q_load(pos, w, wx, wy);
      const double ax = wx - ux, ay = wy - uy, bx = vx - wx, by = vy - wy;
      const double dot = bx * ax + by * ay;
      const double slack = 1e-9 * sqrt((bx * bx + by * by) * (ax * ax + ay * ay));
      if (dot > slack) cand = false;
    }
    if (!cand) continue;
    // exact: no point of the cells that overlap the disc's box inside the disc
    const double mx = 0.5 * (ux + vx), my = 0.5 * (uy + vy);
    const double rad = 0.5 * sqrt((ux - vx) * (ux - vx) + (uy - vy) * (uy - vy)) * (1.0 + 1e-9) + 1e-300;
    int c0x, c0y, c1x, c1y;
    cell_of<V>(g, mx - rad, my - rad, &c0x, &c0y);
    cell_of<V>(g, mx + rad, my + rad, &c1x, &c1y);
    bool blocked = false;
    for (int iy = c0y; iy <= c1y && !blocked; ++iy)
      for (int ix = c0x; ix <= c1x && !blocked; ++ix) {
        const int c = iy * g.side + ix;
        for (int t = g.start[c]; t < g.start[c + 1]; ++t) {
          const int w = g.pts[t];
          if (w != u && w != v && q_in_disc(pos, u, v, w)) {
            blocked = true;
            break;
          }
        }
      }
    if (blocked) continue;
    if (d < kGabDeg) nbr[(size_t)u * kGabDeg + d] = v;
    else overflow = true;
    ++d;
  }
  deg[u] = min(d, kGabDeg);
  if (overflow) dev_fail(status, SSM_E_ARG);
}

// Jaccard coefficient of the kh-neighbourhoods of every node in two graphs
// (fixed-width adjacency nbr[u*kGabDeg + t], t < deg[u]); one warp per node,
// both neighbourhoods grown level by level in shared memory
constexpr int kJacSet = 512;
__global__ void __launch_bounds__(256) k_gab_jaccard(int32_t n, int32_t kh, const int *__restrict__ nbrA,
                                                     const int *__restrict__ degA, const int *__restrict__ nbrB,
                                                     const int *__restrict__ degB, double *__restrict__ per,
                                                     int32_t *__restrict__ status) {
  __shared__ int sets[8][2][kJacSet];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * 8 + warp, nw = gridDim.x * 8;
  for (int v = gw; v < n; v += nw) {
    int size[2];
    bool over = false;
    for (int gsel = 0; gsel < 2; ++gsel) {
      const int *nbr = gsel ? nbrB : nbrA;
      const int *dg = gsel ? degB : degA;
      int *set = sets[warp][gsel];
      int sz = 0, lb = 0;
      // level 1 from v, then from each level's nodes in order
      for (int lev = 1; lev <= kh; ++lev) {
        const int le = sz;
        const int from_b = lev == 1 ? -1 : lb, from_e = lev == 1 ? 0 : le;
        for (int f = from_b; f < from_e; ++f) {
          const int x = f < 0 ? v : set[f];
          const int dx = dg[x];
          for (int base = 0; base < dx; base += 32) {
            const int t = base + lane;
            int y = -1;
            if (t < dx) y = nbr[(size_t)x * kGabDeg + t];
            bool add = y >= 0 && y != v;
            for (int q = 0; add && q < sz; ++q)
              if (set[q] == y) add = false;
            const unsigned m = __ballot_sync(0xffffffffu, add);
            const int pos = sz + __popc(m & ((1u << lane) - 1u));
            if (add && pos < kJacSet) set[pos] = y;
            sz += __popc(m);
            if (sz > kJacSet) {
              over = true;
              sz = kJacSet;
            }
            __syncwarp();
          }
        }
        lb = le;
      }
      size[gsel] = sz;
    }
    int both = 0;
    for (int a = lane; a < size[0]; a += 32) {
      const int y = sets[warp][0][a];
      bool in = false;
      for (int b = 0; b < size[1] && !in; ++b) in = sets[warp][1][b] == y;
      both += in ? 1 : 0;
    }
    both = __reduce_add_sync(0xffffffffu, both);
    if (lane == 0) {
      const int uni = size[0] + size[1] - both;
      per[v] = uni > 0 ? (double)both / (double)uni : 1.0;
      if (over) dev_fail(status, SSM_E_ARG);
    }
    __syncwarp();
  }
}

}  // namespace ssm

namespace ssm {
static int grid_side(int32_t n) {
  int s = (int)ceil(sqrt((double)n / 2.0));
  return s < 1 ? 1 : s;
}

struct GabWs {
  double *bb;
  int *cellid, *count, *start, *cursor, *pts, *visit, *nbr, *deg;
};

static void carve_gabriel(Carver &c, GabWs &w, int32_t n) {
  const int side = grid_side(n), cells = side * side;
  w.bb = c.take<double>(4);
  w.cellid = c.take<int>((size_t)n);
  w.count = c.take<int>((size_t)cells);
  w.start = c.take<int>((size_t)cells + 1);
  w.cursor = c.take<int>((size_t)cells);
  w.pts = c.take<int>((size_t)n);
  w.visit = c.take<int>((size_t)n * kGabVisit);
  w.nbr = c.take<int>((size_t)n * kGabDeg);
  w.deg = c.take<int>((size_t)n);
}

template <class V>
static int launch_gabriel(int32_t n, const V *pos, GabWs &w, int32_t *status, cudaStream_t s) {
  const int side = grid_side(n), cells = side * side;
  const int nb = std::max(1, std::min((n + 255) / 256, num_sms() * 8));
  SSM_TRY_CUDA(cudaMemsetAsync(w.count, 0, (size_t)cells * sizeof(int), s));
  note_launch(), k_bbox<V><<<1, 1024, 0, s>>>(n, pos, w.bb);
  note_launch(), k_grid_count<V><<<nb, 256, 0, s>>>(n, pos, w.bb, side, w.cellid, w.count);
  note_launch(), k_grid_scan<<<1, 1024, 0, s>>>(cells, w.count, w.start, w.cursor);
  note_launch(), k_grid_fill<<<nb, 256, 0, s>>>(n, w.cellid, w.cursor, w.pts);
  GridView g{0.0, 0.0, 0.0, side, w.start, w.pts};  // origin and cell size set on the device from the box
  note_launch(), k_gabriel<V><<<(n + 127) / 128, 128, 0, s>>>(n, pos, g, w.bb, w.nbr, w.deg, w.visit, status);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
}  // namespace ssm

SSM_API size_t ssm_gabriel_jaccard_workspace(int32_t n) {
  if (n < 1) return 0;
  ssm::Carver c(nullptr, 0);
  ssm::GabWs a, b;
  ssm::carve_gabriel(c, a, n);
  ssm::carve_gabriel(c, b, n);
  c.take<double>((size_t)n);
  return c.size();
}

SSM_API int ssm_gabriel_jaccard(int32_t n, const void *posA, const void *posB, int32_t precision, int32_t kh,
                                double *per_node, double *mean, int32_t *status, void *ws, size_t ws_bytes,
                                cudaStream_t s) {
  using namespace ssm;
  if (n < 1 || !posA || !posB || !mean || !status || !ws || kh < 1)
    return fail(SSM_E_ARG, "ssm_gabriel_jaccard: bad argument");
  if (precision != 32 && precision != 64) return fail(SSM_E_ARG, "ssm_gabriel_jaccard: precision must be 32 or 64");
  Carver c(ws, ws_bytes);
  GabWs a, b;
  carve_gabriel(c, a, n);
  carve_gabriel(c, b, n);
  double *per_ws = c.take<double>((size_t)n);
  if (!c.ok) return fail(SSM_E_NOMEM, "ssm_gabriel_jaccard: workspace %zu bytes, need %zu", ws_bytes, c.size());
  int rc;
  if (precision == 64) {
    if ((rc = launch_gabriel(n, (const double2 *)posA, a, status, s))) return rc;
    if ((rc = launch_gabriel(n, (const double2 *)posB, b, status, s))) return rc;
  } else {
    if ((rc = launch_gabriel(n, (const float2 *)posA, a, status, s))) return rc;
    if ((rc = launch_gabriel(n, (const float2 *)posB, b, status, s))) return rc;
  }
  double *per = per_node ? per_node : per_ws;
  const int jb = std::max(1, std::min((n + 7) / 8, num_sms() * 8));
  note_launch(), k_gab_jaccard<<<jb, 256, 0, s>>>(n, kh, a.nbr, a.deg, b.nbr, b.deg, per, status);
  note_launch(), k_mean_in_order<<<1, 32, 0, s>>>(n, per, mean);
  SSM_TRY_CUDA(cudaGetLastError());
  return SSM_OK;
}
