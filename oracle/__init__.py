"""ORACLE -- test infrastructure only.

Plain FP64 CPU restatement of "A Sparse Stress Model" (Ortmann, Klimenta,
Brandes; arxiv 1608.08909) in ``oracle.c``, wrapped with ctypes.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library.

Every function takes and returns numpy arrays; see ``oracle.c`` for the
paper passage each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", -1: "bad argument", -2: "bad graph", -3: "disconnected",
          -4: "distance above 65534", -5: "out of memory", -8: "numerical failure"}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: status {code} ({STATUS.get(code, '?')})")
        self.code = code


def build(force: bool = False) -> str:
    """Compile oracle.c (strict IEEE: no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            v, i32, i64, u64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            sig = {
                "orc_build_csr": [i32, i64, v, v, v, v, v],
                "orc_bfs": [i32, v, v, i32, v],
                "orc_maxmin": [i32, v, v, i32, i32, v],
                "orc_kmeans_sp": [i32, i32, v, v, i32, v, v, v],
                "orc_pivot_dist": [i32, v, v, i32, v, v],
                "orc_regions": [i32, i32, v, v],
                "orc_regions_smallest": [i32, i32, v, v],
                "orc_histograms": [i32, i32, v, v, v, v, v, i64],
                "orc_adapted_weights": [i32, i32, v, v, v],
                "orc_pivotmds": [i32, i32, v, v, v, v],
                "orc_rescale": [i32, v, v, v],
                "orc_sweep_jacobi": [i32, v, v, i32, v, v, v, v, v, v],
                "orc_sweep_jacobi_rows": [i32, v, v, i32, v, v, v, v, v, i32, i32],
                "orc_stress_sums_range": [i32, v, v, v, i32, i32, u64, i32, i32, v],
                "orc_sweep_gs": [i32, v, v, i32, v, v, v, v],
                "orc_full_sweep": [i32, v, v, v, i32, v],
                "orc_procrustes": [i32, v, v, v],
                "orc_hull_error": [i32, v, v, i32, v, v],
                "orc_gabriel": [i32, v, v],
                "orc_gabriel_jaccard": [i32, v, v, i32, v, v],
                "orc_splitmix64": [u64, i64, v],
                "orc_sample_pairs": [i32, i32, i32, u64, v, v],
                "orc_full_stress": [i32, v, v, v, i32, i32, u64, v, v],
                "orc_build_wcsr": [i32, i64, v, v, v, v, v, v, v],
                "orc_sssp": [i32, v, v, v, i32, v],
                "orc_wmaxmin": [i32, v, v, v, i32, i32, v],
                "orc_wpivot_dist": [i32, v, v, v, i32, v, v],
                "orc_wregions": [i32, i32, v, v],
                "orc_wcounts_rows": [i32, v, v, i32, v, v, v, v, i32, i32],
                "orc_wpivotmds": [i32, i32, v, v, v, v],
                "orc_wrescale": [i32, v, v, v, v],
                "orc_wsweep_jacobi_rows": [i32, v, v, v, i32, v, v, v, v, v, i32, i32],
                "orc_wfull_stress": [i32, v, v, v, v, i32, i32, u64, v, v],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.orc_relchange.argtypes = [i32, v, v]
            lib.orc_relchange.restype = d
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _chk(rc: int, what: str):
    if rc != 0:
        raise OracleError(rc, what)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Graph:
    """CSR of a simple undirected graph: rowptr[n+1], colidx[2m], sorted rows."""

    def __init__(self, n: int, rowptr: np.ndarray, colidx: np.ndarray, m: int):
        self.n, self.rowptr, self.colidx, self.m = n, rowptr, colidx, m


def build_csr(n: int, src, dst) -> Graph:
    src, dst = _i32(src), _i32(dst)
    rowptr = np.zeros(n + 1, np.int32)
    colidx = np.zeros(max(2 * len(src), 1), np.int32)
    m = ctypes.c_int64(0)
    _chk(_load().orc_build_csr(n, len(src), _p(src), _p(dst), _p(rowptr), _p(colidx), ctypes.byref(m)),
         "build_csr")
    return Graph(n, rowptr, colidx[: 2 * m.value].copy(), m.value)


def bfs(g: Graph, s: int) -> np.ndarray:
    dist = np.zeros(g.n, np.int32)
    _chk(_load().orc_bfs(g.n, _p(g.rowptr), _p(g.colidx), s, _p(dist)), "bfs")
    return dist


def maxmin(g: Graph, k: int, start: int = 0) -> np.ndarray:
    piv = np.zeros(k, np.int32)
    _chk(_load().orc_maxmin(g.n, _p(g.rowptr), _p(g.colidx), k, start, _p(piv)), "maxmin")
    return piv


def kmeans_sp(dip: np.ndarray, pivots, max_iter: int = 50):
    """k-means sp (Section 4.1) from the max/min-sp pivots and their d_ip table:
    returns (new pivots [k] int32, final cluster of every node [n] int32,
    assignment passes)."""
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    pivots = _i32(pivots)
    k, n = dip.shape
    out = np.zeros(k, np.int32)
    asg = np.zeros(n, np.int32)
    it = ctypes.c_int32(0)
    _chk(_load().orc_kmeans_sp(n, k, _p(dip), _p(pivots), max_iter, _p(out), _p(asg), ctypes.byref(it)), "kmeans_sp")
    return out, asg, it.value


def pivot_dist(g: Graph, pivots) -> np.ndarray:
    pivots = _i32(pivots)
    k = len(pivots)
    dip = np.zeros((k, g.n), np.uint16)
    _chk(_load().orc_pivot_dist(g.n, _p(g.rowptr), _p(g.colidx), k, _p(pivots), _p(dip)), "pivot_dist")
    return dip


def regions(dip: np.ndarray) -> np.ndarray:
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    k, n = dip.shape
    reg = np.zeros(n, np.int32)
    _chk(_load().orc_regions(n, k, _p(dip), _p(reg)), "regions")
    return reg


def regions_smallest(dip: np.ndarray) -> np.ndarray:
    """Regions with the paper's tie rule: ties to the region that is smallest at that moment,
    nodes taken by increasing distance to their nearest pivot, then by id."""
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    k, n = dip.shape
    reg = np.zeros(n, np.int32)
    _chk(_load().orc_regions_smallest(n, k, _p(dip), _p(reg)), "regions_smallest")
    return reg


def histograms(dip: np.ndarray, region: np.ndarray):
    """Returns (ecc[k], cnt_off[k+1] int64, cnt[cnt_off[k]] uint32)."""
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    region = _i32(region)
    k, n = dip.shape
    ecc = np.zeros(k, np.int32)
    lib = _load()
    _chk(lib.orc_histograms(n, k, _p(dip), _p(region), _p(ecc), None, None, 0), "histograms")
    cap = int((ecc.astype(np.int64) + 1).sum())
    off = np.zeros(k + 1, np.int64)
    cnt = np.zeros(max(cap, 1), np.uint32)
    _chk(lib.orc_histograms(n, k, _p(dip), _p(region), _p(ecc), _p(off), _p(cnt), cap), "histograms")
    return ecc, off, cnt[:cap]


def adapted_weights(dip: np.ndarray, region: np.ndarray) -> np.ndarray:
    """w[a][i] = s/d_ia^2 (0 where the pivot term is skipped), by direct count."""
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    region = _i32(region)
    k, n = dip.shape
    w = np.zeros((k, n), np.float64)
    _chk(_load().orc_adapted_weights(n, k, _p(dip), _p(region), _p(w)), "adapted_weights")
    return w


def gram(dip: np.ndarray) -> np.ndarray:
    """The dense contraction inside PivotMDS (Algorithm 1, line 3) before any
    centring: G[a][b] = sum_i d_ia^2 d_ib^2 over the pivot-major table, as
    exact Python integers (object array [k, k]).  Each squared distance is
    split into 16-bit halves, s = 2^16 h + l, so that every partial product
    sum h_a h_b, h_a l_b, l_a l_b is an integer below 2^53 and the float64
    matrix products are exact; the halves are recombined in integers."""
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    k, n = dip.shape
    if n >= (1 << 21):
        raise OracleError(-1, "gram: n too large for exact float64 partial sums")
    sq = dip.astype(np.uint64) ** 2
    h = (sq >> np.uint64(16)).astype(np.float64)
    l = (sq & np.uint64(0xFFFF)).astype(np.float64)
    hh, hl, lh, ll = h @ h.T, h @ l.T, l @ h.T, l @ l.T
    G = np.empty((k, k), dtype=object)
    for a in range(k):
        for b in range(k):
            G[a, b] = ((int(hh[a, b]) << 32) + ((int(hl[a, b]) + int(lh[a, b])) << 16) + int(ll[a, b]))
    return G


def pivotmds(dip: np.ndarray, return_b: bool = False):
    """PivotMDS layout [n][2] and the two eigenvalues (and B = C^T C if asked)."""
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    k, n = dip.shape
    pos = np.zeros((n, 2), np.float64)
    eig = np.zeros(2, np.float64)
    B = np.zeros((k, k), np.float64) if return_b else None
    _chk(_load().orc_pivotmds(n, k, _p(dip), _p(pos), _p(eig), _p(B) if return_b else None), "pivotmds")
    return (pos, eig, B) if return_b else (pos, eig)


def rescale(g: Graph, pos: np.ndarray) -> np.ndarray:
    pos = np.array(pos, dtype=np.float64, order="C", copy=True)
    _chk(_load().orc_rescale(g.n, _p(g.rowptr), _p(g.colidx), _p(pos)), "rescale")
    return pos


def sweep_jacobi(g: Graph, pivots, dip, w, pos):
    """One Jacobi update of Eq. 4; returns (new positions, relative change)."""
    pivots = _i32(pivots)
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    w = np.ascontiguousarray(w, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = np.zeros_like(pos)
    rel = ctypes.c_double(0.0)
    _chk(_load().orc_sweep_jacobi(g.n, _p(g.rowptr), _p(g.colidx), len(pivots), _p(pivots), _p(dip), _p(w),
                                  _p(pos), _p(out), ctypes.byref(rel)), "sweep_jacobi")
    return out, rel.value


def sweep_jacobi_threads(g: Graph, pivots, dip, w, pos, threads: int):
    """sweep_jacobi with the node loop cut into `threads` contiguous ranges run
    by host threads at once (ctypes releases the GIL during each C call).
    Every node's update is computed exactly as in sweep_jacobi, and the
    relative change is reduced afterwards in node order, so the result is
    identical to sweep_jacobi's."""
    import concurrent.futures as cf

    pivots = _i32(pivots)
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    w = np.ascontiguousarray(w, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = np.zeros_like(pos)
    n = g.n
    cuts = [n * t // threads for t in range(threads + 1)]
    lib = _load()

    def run(t):
        return lib.orc_sweep_jacobi_rows(n, _p(g.rowptr), _p(g.colidx), len(pivots), _p(pivots), _p(dip), _p(w),
                                         _p(pos), _p(out), cuts[t], cuts[t + 1])

    with cf.ThreadPoolExecutor(threads) as ex:
        for rc in ex.map(run, range(threads)):
            _chk(rc, "sweep_jacobi_rows")
    return out, lib.orc_relchange(n, _p(pos), _p(out))


def pivot_dist_threads(g: Graph, pivots, threads: int) -> np.ndarray:
    """pivot_dist with the pivots split over `threads` host threads; every row
    is one independent BFS, so the table is identical to pivot_dist's."""
    import concurrent.futures as cf

    pivots = _i32(pivots)
    parts = np.array_split(np.arange(len(pivots)), threads)
    with cf.ThreadPoolExecutor(threads) as ex:
        rows = list(ex.map(lambda idx: pivot_dist(g, pivots[idx]) if len(idx) else None, parts))
    return np.concatenate([r for r in rows if r is not None], axis=0)


def stress_sums_range(g: Graph, pos, S: int, T: int, seed: int, q0: int, q1: int) -> np.ndarray:
    """The pair sums {sum (r-d)^2/d^2, S1, S2, N} of full_stress's pair list
    restricted to its sources q0 <= q < q1."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    sums = np.zeros(4, np.float64)
    _chk(_load().orc_stress_sums_range(g.n, _p(g.rowptr), _p(g.colidx), _p(pos), S, T, ctypes.c_uint64(seed), q0, q1,
                                       _p(sums)), "stress_sums_range")
    return sums


def full_stress_threads(g: Graph, pos, S: int, T: int, seed: int, threads: int):
    """full_stress's sums over its sources split into `threads` ranges run at
    once and added in range order (the association of the sums differs from
    full_stress's by rounding only).  Returns (out[4], sums[4]) with out as in
    full_stress."""
    import concurrent.futures as cf

    nsrc = S if S > 0 else g.n
    cuts = [nsrc * t // threads for t in range(threads + 1)]
    with cf.ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda t: stress_sums_range(g, pos, S, T, seed, cuts[t], cuts[t + 1]), range(threads)))
    sums = np.zeros(4, np.float64)
    for p_ in parts:
        sums += p_
    raw, s1, s2, npairs = sums
    pairs = 0.5 * g.n * (g.n - 1)
    f = pairs / npairs if S > 0 else 1.0
    out = np.array([raw * f, s1 / s2 if s2 > 0 else 0.0, (npairs - s1 * s1 / s2 if s2 > 0 else npairs) * f, 0.0])
    out[3] = out[2] / pairs
    return out, sums


def sweep_gs(g: Graph, pivots, dip, w, pos):
    """One in-place (node by node, ascending) update of Eq. 4; returns new positions."""
    pivots = _i32(pivots)
    dip = np.ascontiguousarray(dip, dtype=np.uint16)
    w = np.ascontiguousarray(w, dtype=np.float64)
    pos = np.array(pos, dtype=np.float64, order="C", copy=True)
    _chk(_load().orc_sweep_gs(g.n, _p(g.rowptr), _p(g.colidx), len(pivots), _p(pivots), _p(dip), _p(w),
                              _p(pos)), "sweep_gs")
    return pos


def apsp(g: Graph) -> np.ndarray:
    """All-pairs hop distances [n][n] uint16, one BFS per node (row i = BFS from i)."""
    return pivot_dist(g, np.arange(g.n, dtype=np.int32))


def full_sweep(D: np.ndarray, pos, order: int = 0):
    """One sweep of full stress majorization over the all-pairs table D
    (order 0 Jacobi, 1 Gauss-Seidel); returns (positions, relative change)."""
    D = np.ascontiguousarray(D, dtype=np.uint16)
    n = D.shape[0]
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = np.zeros_like(pos)
    rel = ctypes.c_double(0.0)
    _chk(_load().orc_full_sweep(n, _p(D), _p(pos), _p(out), order, ctypes.byref(rel)), "full_sweep")
    return out, rel.value


def procrustes(X, Y):
    """Procrustes statistic of layouts X, Y [n][2] (rotation and uniform scale,
    no reflection): returns (P, scale, angle)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    out = np.zeros(3, np.float64)
    _chk(_load().orc_procrustes(len(X), _p(X), _p(Y), _p(out)), "procrustes")
    return tuple(out.tolist())


def hull_error(D: np.ndarray, pos, kh: int):
    """Convex-hull error of Fig. 4 for hop radius kh: returns (mean, per-node errors)."""
    D = np.ascontiguousarray(D, dtype=np.uint16)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = D.shape[0]
    per = np.zeros(n, np.float64)
    mean = ctypes.c_double(0.0)
    _chk(_load().orc_hull_error(n, _p(D), _p(pos), kh, _p(per), ctypes.byref(mean)), "hull_error")
    return mean.value, per


def gabriel(pos) -> np.ndarray:
    """Gabriel graph of a layout as an n x n 0/1 matrix (open-disc reading)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = len(pos)
    adj = np.zeros((n, n), np.uint8)
    _chk(_load().orc_gabriel(n, _p(pos), _p(adj)), "gabriel")
    return adj


def gabriel_jaccard(posA, posB, kh: int):
    """Gabriel-graph kh-neighbourhood Jaccard similarity of Fig. 3: (mean, per node)."""
    posA = np.ascontiguousarray(posA, dtype=np.float64)
    posB = np.ascontiguousarray(posB, dtype=np.float64)
    n = len(posA)
    per = np.zeros(n, np.float64)
    mean = ctypes.c_double(0.0)
    _chk(_load().orc_gabriel_jaccard(n, _p(posA), _p(posB), kh, _p(per), ctypes.byref(mean)), "gabriel_jaccard")
    return mean.value, per


def splitmix64(seed: int, count: int) -> np.ndarray:
    out = np.zeros(count, np.uint64)
    _chk(_load().orc_splitmix64(ctypes.c_uint64(seed), count, _p(out)), "splitmix64")
    return out


def sample_pairs(n: int, S: int, T: int, seed: int):
    srcs = np.zeros(S, np.int32)
    tgts = np.zeros((S, T), np.int32)
    _chk(_load().orc_sample_pairs(n, S, T, ctypes.c_uint64(seed), _p(srcs), _p(tgts)), "sample_pairs")
    return srcs, tgts


def full_stress(g: Graph, pos, S: int = 0, T: int = 0, seed: int = 0, return_sums: bool = False):
    """{raw, alpha*, scaled, normalized} of Eq. 1; S=0 exhaustive, else S*T sampled pairs."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = np.zeros(4, np.float64)
    sums = np.zeros(4, np.float64)
    _chk(_load().orc_full_stress(g.n, _p(g.rowptr), _p(g.colidx), _p(pos), S, T, ctypes.c_uint64(seed),
                                 _p(out), _p(sums)), "full_stress")
    return (out, sums) if return_sums else out


# ---------------------------------------------------------------------------
# Whole pipeline (Algorithm 1 with the Jacobi schedule), for tests and the
# CPU baseline.
# ---------------------------------------------------------------------------

class Prepared:
    """Everything Algorithm 1 lines 1-4 produce for one graph."""

    def __init__(self, g, pivots, dip, region, ecc, cnt_off, cnt, w, pos0, eig):
        self.g, self.pivots, self.dip, self.region = g, pivots, dip, region
        self.ecc, self.cnt_off, self.cnt, self.w, self.pos0, self.eig = ecc, cnt_off, cnt, w, pos0, eig


def prepare(n: int, src, dst, k: int, start: int = 0, sampler: str = "maxmin", kmeans_iters: int = 50,
            ties: str = "lowest") -> Prepared:
    g = build_csr(n, src, dst)
    piv = maxmin(g, k, start)
    dip = pivot_dist(g, piv)
    if sampler == "kmeans":
        piv, _, _ = kmeans_sp(dip, piv, kmeans_iters)
        dip = pivot_dist(g, piv)
    reg = regions(dip) if ties == "lowest" else regions_smallest(dip)
    ecc, off, cnt = histograms(dip, reg)
    w = adapted_weights(dip, reg)
    pos, eig = pivotmds(dip)
    pos = rescale(g, pos)
    return Prepared(g, piv, dip, reg, ecc, off, cnt, w, pos, eig)


def iterate(p: Prepared, pos, iters: int):
    """`iters` Jacobi updates from pos; returns (positions, last relative change)."""
    rel = 0.0
    for _ in range(iters):
        pos, rel = sweep_jacobi(p.g, p.pivots, p.dip, p.w, pos)
    return pos, rel


# ---------------------------------------------------------------- weighted graphs
class WGraph(Graph):
    """CSR of a weighted simple undirected graph: as Graph plus elen[2m]
    (float32, the length of the edge colidx[t])."""

    def __init__(self, n, rowptr, colidx, m, elen):
        super().__init__(n, rowptr, colidx, m)
        self.elen = elen


def build_wcsr(n: int, src, dst, lengths) -> WGraph:
    src, dst = _i32(src), _i32(dst)
    lengths = np.ascontiguousarray(lengths, dtype=np.float32)
    rowptr = np.zeros(n + 1, np.int32)
    colidx = np.zeros(max(2 * len(src), 1), np.int32)
    elen = np.zeros(max(2 * len(src), 1), np.float32)
    m = ctypes.c_int64(0)
    _chk(_load().orc_build_wcsr(n, len(src), _p(src), _p(dst), _p(lengths), _p(rowptr), _p(colidx), _p(elen),
                                ctypes.byref(m)), "build_wcsr")
    return WGraph(n, rowptr, colidx[: 2 * m.value].copy(), m.value, elen[: 2 * m.value].copy())


def sssp(g: WGraph, s: int) -> np.ndarray:
    dist = np.zeros(g.n, np.float32)
    _chk(_load().orc_sssp(g.n, _p(g.rowptr), _p(g.colidx), _p(g.elen), s, _p(dist)), "sssp")
    return dist


def wmaxmin(g: WGraph, k: int, start: int = 0) -> np.ndarray:
    piv = np.zeros(k, np.int32)
    _chk(_load().orc_wmaxmin(g.n, _p(g.rowptr), _p(g.colidx), _p(g.elen), k, start, _p(piv)), "wmaxmin")
    return piv


def wpivot_dist(g: WGraph, pivots) -> np.ndarray:
    pivots = _i32(pivots)
    dip = np.zeros((len(pivots), g.n), np.float32)
    _chk(_load().orc_wpivot_dist(g.n, _p(g.rowptr), _p(g.colidx), _p(g.elen), len(pivots), _p(pivots), _p(dip)),
         "wpivot_dist")
    return dip


def wregions(dip) -> np.ndarray:
    dip = np.ascontiguousarray(dip, dtype=np.float32)
    k, n = dip.shape
    reg = np.zeros(n, np.int32)
    _chk(_load().orc_wregions(n, k, _p(dip), _p(reg)), "wregions")
    return reg


def wcounts(g: WGraph, pivots, dip, region, i0: int = 0, i1: int | None = None, threads: int = 1) -> np.ndarray:
    """s[a][i] for the nodes i0 <= i < i1 (other columns 0), by direct count;
    the node range split over `threads` host threads."""
    import concurrent.futures as cf

    pivots, region = _i32(pivots), _i32(region)
    dip = np.ascontiguousarray(dip, dtype=np.float32)
    k, n = dip.shape
    i1 = n if i1 is None else i1
    s = np.zeros((k, n), np.uint32)
    lib = _load()
    cuts = [i0 + (i1 - i0) * t // threads for t in range(threads + 1)]

    def run(t):
        return lib.orc_wcounts_rows(n, _p(g.rowptr), _p(g.colidx), k, _p(pivots), _p(dip), _p(region), _p(s),
                                    cuts[t], cuts[t + 1])

    with cf.ThreadPoolExecutor(threads) as ex:
        for rc in ex.map(run, range(threads)):
            _chk(rc, "wcounts_rows")
    return s


def wpivotmds(dip):
    dip = np.ascontiguousarray(dip, dtype=np.float32)
    k, n = dip.shape
    pos = np.zeros((n, 2), np.float64)
    eig = np.zeros(2, np.float64)
    _chk(_load().orc_wpivotmds(n, k, _p(dip), _p(pos), _p(eig), None), "wpivotmds")
    return pos, eig


def wrescale(g: WGraph, pos) -> np.ndarray:
    pos = np.array(pos, dtype=np.float64, order="C")
    _chk(_load().orc_wrescale(g.n, _p(g.rowptr), _p(g.colidx), _p(g.elen), _p(pos)), "wrescale")
    return pos


def wsweep_jacobi(g: WGraph, pivots, dip, s, pos, threads: int = 1):
    """One Jacobi update of Eq. 4 on a weighted graph: (positions, relative change)."""
    import concurrent.futures as cf

    pivots = _i32(pivots)
    dip = np.ascontiguousarray(dip, dtype=np.float32)
    s = np.ascontiguousarray(s, dtype=np.uint32)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = np.zeros_like(pos)
    n = g.n
    lib = _load()
    cuts = [n * t // threads for t in range(threads + 1)]

    def run(t):
        return lib.orc_wsweep_jacobi_rows(n, _p(g.rowptr), _p(g.colidx), _p(g.elen), len(pivots), _p(pivots),
                                          _p(dip), _p(s), _p(pos), _p(out), cuts[t], cuts[t + 1])

    with cf.ThreadPoolExecutor(threads) as ex:
        for rc in ex.map(run, range(threads)):
            _chk(rc, "wsweep_jacobi_rows")
    return out, lib.orc_relchange(n, _p(pos), _p(out))


def wfull_stress(g: WGraph, pos, nsources: int = 0, ntargets: int = 0, seed: int = 0):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = np.zeros(4, np.float64)
    sums = np.zeros(4, np.float64)
    _chk(_load().orc_wfull_stress(g.n, _p(g.rowptr), _p(g.colidx), _p(g.elen), _p(pos), nsources, ntargets,
                                  ctypes.c_uint64(seed), _p(out), _p(sums)), "wfull_stress")
    return out, sums


class WPrepared:
    def __init__(self, g, pivots, dip, region, s, pos, eig):
        self.g, self.pivots, self.dip, self.region, self.s, self.pos, self.eig = g, pivots, dip, region, s, pos, eig


def wprepare(n: int, src, dst, lengths, k: int, start: int = 0, threads: int = 1) -> WPrepared:
    """Algorithm 1 lines 1-4 on a weighted graph."""
    g = build_wcsr(n, src, dst, lengths)
    piv = wmaxmin(g, k, start)
    dip = wpivot_dist(g, piv)
    reg = wregions(dip)
    s = wcounts(g, piv, dip, reg, threads=threads)
    pos, eig = wpivotmds(dip)
    pos = wrescale(g, pos)
    return WPrepared(g, piv, dip, reg, s, pos, eig)
