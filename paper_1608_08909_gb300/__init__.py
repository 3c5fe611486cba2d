"""GB300 sparse stress layout: Python binding of libssm (include/ssm.h).

Argument marshalling only.  Every step runs in the CUDA kernels of
``csrc/``; PyTorch provides device memory and streams.  There is no CPU
fallback: if the compiled library is missing or no CUDA device is present,
every call raises.

The functions mirror the C ABI names (``ssm_build_graph`` ... ``ssm_stress``)
and take / return torch tensors on the current CUDA device.  ``layout()`` runs
the whole Algorithm 1 pipeline.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

from . import _build

__all__ = [
    "SSMError", "lib", "ssm_build_graph", "ssm_select_pivots", "ssm_pivot_bfs", "ssm_aggregate_size",
    "ssm_aggregate", "ssm_aggregate_noalloc", "ssm_gram", "ssm_pivotmds", "ssm_batch_iterate",
    "ssm_batch_prepare", "ssm_batch_iterate_packed", "BatchPacked", "ssm_iterate", "ssm_stress", "ssm_check", "Graph", "Pivots", "layout",
    "ssm_set_wait_limit_ns", "ssm_last_sweep_config", "ssm_last_pivot_config", "ssm_kmeans_pivots", "ssm_iterate_gs", "ssm_apsp",
    "ssm_iterate_hints", "ssm_full_iterate", "ssm_regions_smallest", "ssm_aggregate_regions", "ssm_procrustes", "ssm_hull_error", "ssm_gabriel_jaccard",
    "WGraph", "ssm_build_wgraph", "ssm_pivot_sssp", "ssm_select_pivots_weighted", "ssm_weighted_counts",
    "ssm_pivotmds_weighted", "ssm_iterate_weighted", "ssm_stress_weighted", "layout_weighted",
]

STATUS = {0: "ok", -1: "invalid argument", -2: "edge endpoint out of range", -3: "graph is disconnected",
          -4: "hop distance above 65534", -5: "workspace too small", -6: "CUDA error", -7: "device wait timed out",
          -8: "numerical failure"}


class SSMError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        msg = f"{what}: status {code} ({STATUS.get(code, '?')})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """Load libssm.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            v, i32, i64, u64, d, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_double, ctypes.c_size_t)
            sig = {
                "ssm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
                "ssm_last_error": (ctypes.c_char_p, []),
                "ssm_kernel_launches": (ctypes.c_ulonglong, []),
                "ssm_set_wait_limit_ns": (ctypes.c_ulonglong, [ctypes.c_ulonglong]),
                "ssm_last_sweep_config": (None, [v]),
                "ssm_last_pivot_config": (None, [v]),
                "ssm_check": (ctypes.c_int, [v, v]),
                "ssm_build_graph_workspace": (sz, [i32, i64]),
                "ssm_build_graph": (ctypes.c_int, [i32, i64, v, v, v, v, v, v, v, sz, v]),
                "ssm_select_pivots_workspace": (sz, [i32, i64]),
                "ssm_select_pivots": (ctypes.c_int, [i32, i64, v, v, i32, i32, v, v, v, sz, v]),
                "ssm_kmeans_pivots_workspace": (sz, [i32, i32]),
                "ssm_kmeans_pivots": (ctypes.c_int, [i32, i32, v, v, i32, v, v, v, v, v, sz, v]),
                "ssm_pivot_bfs_workspace": (sz, [i32, i64, i32]),
                "ssm_pivot_bfs": (ctypes.c_int, [i32, i64, v, v, i32, v, v, v, v, sz, v]),
                "ssm_aggregate_workspace": (sz, [i32]),
                "ssm_aggregate_size": (ctypes.c_int, [i32, i32, v, v, v, v, sz, v]),
                "ssm_aggregate": (ctypes.c_int, [i32, i32, v, v, v, v, i64, v, v, sz, v]),
                "ssm_aggregate_noalloc": (ctypes.c_int, [i32, i32, v, v, v, v, i64, v, v, v]),
                "ssm_regions_smallest_workspace": (sz, [i32]),
                "ssm_regions_smallest": (ctypes.c_int, [i32, i32, v, v, v, v, sz, v]),
                "ssm_aggregate_regions": (ctypes.c_int, [i32, i32, v, v, v, v, i64, v, v, v, sz, v]),
                "ssm_gram_workspace": (sz, [i32, i32]),
                "ssm_gram": (ctypes.c_int, [i32, i32, v, v, v, v, v, sz, v]),
                "ssm_pivotmds_workspace": (sz, [i32, i32]),
                "ssm_batch_iterate_workspace": (sz, [i32, v]),
                "ssm_batch_iterate": (ctypes.c_int, [i32, v, v, v, v, v, v, v, v, i32, v, i32, i32, v, v, v, sz, v]),
                "ssm_pivotmds": (ctypes.c_int, [i32, v, v, i32, v, v, i32, i32, v, v, v, sz, v]),
                "ssm_iterate_workspace": (sz, [i32, i64, i32, i64, i32]),
                "ssm_iterate": (ctypes.c_int, [i32, i64, v, v, i32, v, v, v, v, i64, v, i32, i32, d, v, v, v, v, v, sz, v]),
                "ssm_iterate_hints": (ctypes.c_int, [i32, v, i32, v, v, v, sz, v]),
                "ssm_iterate_gs_workspace": (sz, [i32]),
                "ssm_iterate_gs": (ctypes.c_int, [i32, i64, v, v, i32, v, v, v, v, v, i32, v, v, v, sz, v]),
                "ssm_full_iterate_workspace": (sz, [i32, i32]),
                "ssm_full_iterate": (ctypes.c_int, [i32, v, v, i32, i32, i32, v, v, v, sz, v]),
                "ssm_procrustes": (ctypes.c_int, [i32, v, v, i32, v, v]),
                "ssm_hull_error_workspace": (sz, [i32]),
                "ssm_hull_error": (ctypes.c_int, [i32, v, v, i32, i32, v, v, v, v, sz, v]),
                "ssm_gabriel_jaccard_workspace": (sz, [i32]),
                "ssm_gabriel_jaccard": (ctypes.c_int, [i32, v, v, i32, i32, v, v, v, v, sz, v]),
                "ssm_edge_lengths": (ctypes.c_int, [i32, i64, v, v, v, i64, v, v, v, v, v, sz, v]),
                "ssm_pivot_sssp_workspace": (sz, [i32, i32]),
                "ssm_pivot_sssp": (ctypes.c_int, [i32, i64, v, v, v, i32, v, v, v, v, sz, v]),
                "ssm_select_pivots_weighted_workspace": (sz, [i32, i32]),
                "ssm_select_pivots_weighted": (ctypes.c_int, [i32, i64, v, v, v, i32, i32, v, v, v, sz, v]),
                "ssm_weighted_counts_workspace": (sz, [i32, i32]),
                "ssm_weighted_counts": (ctypes.c_int, [i32, v, v, i32, v, v, v, v, v, v, sz, v]),
                "ssm_pivotmds_weighted_workspace": (sz, [i32, i32]),
                "ssm_pivotmds_weighted": (ctypes.c_int, [i32, v, v, v, i32, v, v, i32, i32, v, v, v, sz, v]),
                "ssm_iterate_weighted_workspace": (sz, [i32, i32, i32]),
                "ssm_iterate_weighted": (ctypes.c_int, [i32, v, v, v, i32, v, v, v, v, i32, i32, v, v, v, sz, v]),
                "ssm_stress_weighted_workspace": (sz, [i32, i32]),
                "ssm_stress_weighted": (ctypes.c_int, [i32, v, v, v, v, i32, i32, i32, u64, v, v, v, v, sz, v]),
                "ssm_batch_prepare_workspace": (sz, [i32, v]),
                "ssm_batch_pivots": (ctypes.c_int, [i32, v, v, v, v, v, v, v, v, v, v, v, v, v, sz, v]),
                "ssm_batch_layout_init": (ctypes.c_int, [i32, v, v, v, v, v, v, v, v, v, v, v, v, v, sz, v]),
                "ssm_stress_workspace": (sz, [i32, i64, i32, i32]),
                "ssm_stress": (ctypes.c_int, [i32, i64, v, v, v, i32, i32, i32, u64, v, v, v, v, sz, v]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernels the library has enqueued since it was loaded (ssm_kernel_launches)."""
    return int(lib().ssm_kernel_launches())


def ssm_set_wait_limit_ns(ns: int) -> int:
    """Longest wait at a device-wide barrier before a kernel gives up with
    SSM_E_TIMEOUT (0: the default 2 s); returns the previous setting."""
    return int(lib().ssm_set_wait_limit_ns(int(ns)))


def ssm_last_sweep_config() -> dict:
    """What the last ssm_iterate on this thread chose (ssm_last_sweep_config)."""
    out = (ctypes.c_int32 * 4)()
    lib().ssm_last_sweep_config(ctypes.cast(out, ctypes.c_void_p))
    kinds = {-1: None, 0: "f32_clamped_smem", 1: "f32_clamped_global", 2: "f32_full_table", 3: "f64_counts_smem",
             4: "f64_counts_global"}
    return {"kernel": kinds.get(out[0], out[0]), "nsplit": out[1], "blocks": out[2], "dmax": out[3]}


def ssm_last_pivot_config() -> dict:
    """What the last max/min selection on this thread chose (ssm_last_pivot_config)."""
    out = (ctypes.c_int32 * 2)()
    lib().ssm_last_pivot_config(ctypes.cast(out, ctypes.c_void_p))
    return {"cluster": out[0], "mind_bytes": out[1]}


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("libssm needs a CUDA device; there is no CPU path")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _rc(code: int, what: str):
    if code != 0:
        raise SSMError(code, what, lib().ssm_last_error().decode(errors="replace"))


def _ws(nbytes: int, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _status(device):
    return torch.zeros(1, dtype=torch.int32, device=device)


def ssm_check(status: torch.Tensor, what: str = "device", stream=None):
    """Synchronise and raise SSMError if the device status word is set."""
    _rc(lib().ssm_check(_ptr(status), _stream(stream)), what)


@dataclass
class Graph:
    n: int
    m: int
    rowptr: torch.Tensor  # int32 [n+1]
    colidx: torch.Tensor  # int32 [2m]
    row_classes: tuple | None = None  # rows with 33..1024 and > 1024 entries (from ssm_build_graph)


@dataclass
class Pivots:
    k: int
    pivots: torch.Tensor   # int32 [k]
    dip: torch.Tensor      # uint16 [k, n]
    region: torch.Tensor   # int32 [n]
    cnt_off: torch.Tensor  # int32 [k+1]
    cnt: torch.Tensor      # uint32 [cnt_off[k]]
    dmax: int | None = None  # largest d_ip entry (from ssm_aggregate_size), a hint for ssm_iterate


def ssm_build_graph(n: int, src: torch.Tensor, dst: torch.Tensor, stream=None) -> Graph:
    """CSR of the simple undirected graph on the edge list (device int32 tensors)."""
    _require_cuda()
    L = lib()
    dev = src.device
    src = src.contiguous().to(torch.int32)
    dst = dst.contiguous().to(torch.int32)
    m_in = src.numel()
    rowptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
    colidx = torch.empty(max(2 * m_in, 1), dtype=torch.int32, device=dev)
    ws = _ws(L.ssm_build_graph_workspace(n, m_in), dev)
    m = ctypes.c_int64(0)
    rc_ = (ctypes.c_int32 * 2)()
    _rc(L.ssm_build_graph(n, m_in, _ptr(src), _ptr(dst), _ptr(rowptr), _ptr(colidx), ctypes.byref(m),
                          ctypes.cast(rc_, ctypes.c_void_p), _ptr(ws), ws.numel(), _stream(stream)), "ssm_build_graph")
    return Graph(n, int(m.value), rowptr, colidx[: 2 * m.value], row_classes=(int(rc_[0]), int(rc_[1])))


def ssm_select_pivots(g: Graph, k: int, start: int = 0, stream=None, check: bool = True) -> torch.Tensor:
    L = lib()
    dev = g.rowptr.device
    piv = torch.empty(k, dtype=torch.int32, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_select_pivots_workspace(g.n, g.m), dev)
    _rc(L.ssm_select_pivots(g.n, g.m, _ptr(g.rowptr), _ptr(g.colidx), k, start, _ptr(piv), _ptr(st), _ptr(ws), ws.numel(),
                            _stream(stream)), "ssm_select_pivots")
    if check:
        ssm_check(st, "ssm_select_pivots", stream)
    return piv


def ssm_kmeans_pivots(dip: torch.Tensor, pivots: torch.Tensor, max_iter: int = 50, stream=None, check: bool = True):
    """k-means sp (Section 4.1) from max/min-sp pivots and their d_ip table.
    Returns (new pivots [k] int32, cluster of every node [n] int32, passes run
    as a device int32 tensor)."""
    L = lib()
    k, n = dip.shape
    dev = dip.device
    out = torch.empty(k, dtype=torch.int32, device=dev)
    asg = torch.empty(n, dtype=torch.int32, device=dev)
    it = torch.zeros(1, dtype=torch.int32, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_kmeans_pivots_workspace(n, k), dev)
    _rc(L.ssm_kmeans_pivots(n, k, _ptr(dip), _ptr(pivots.contiguous()), max_iter, _ptr(out), _ptr(asg), _ptr(it),
                            _ptr(st), _ptr(ws), ws.numel(), _stream(stream)), "ssm_kmeans_pivots")
    if check:
        ssm_check(st, "ssm_kmeans_pivots", stream)
    return out, asg, it


def ssm_pivot_bfs(g: Graph, pivots: torch.Tensor, stream=None, check: bool = True) -> torch.Tensor:
    L = lib()
    dev = g.rowptr.device
    k = pivots.numel()
    dip = torch.empty((k, g.n), dtype=torch.uint16, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_pivot_bfs_workspace(g.n, g.m, k), dev)
    _rc(L.ssm_pivot_bfs(g.n, g.m, _ptr(g.rowptr), _ptr(g.colidx), k, _ptr(pivots.contiguous()), _ptr(dip), _ptr(st),
                        _ptr(ws), ws.numel(), _stream(stream)), "ssm_pivot_bfs")
    if check:
        ssm_check(st, "ssm_pivot_bfs", stream)
    return dip


def ssm_aggregate_size(dip: torch.Tensor, stream=None, with_dmax: bool = False):
    """Length of the count table (synchronous); with_dmax: (length, largest d_ip entry)."""
    L = lib()
    k, n = dip.shape
    ws = _ws(L.ssm_aggregate_workspace(k), dip.device)
    out = ctypes.c_int64(0)
    dm = ctypes.c_int32(0)
    _rc(L.ssm_aggregate_size(n, k, _ptr(dip), ctypes.byref(out), ctypes.byref(dm), _ptr(ws), ws.numel(),
                             _stream(stream)), "ssm_aggregate_size")
    return (int(out.value), int(dm.value)) if with_dmax else int(out.value)


def ssm_aggregate(dip: torch.Tensor, cnt_len: int | None = None, stream=None, check: bool = True):
    """Returns (region[n] int32, cnt_off[k+1] int32, cnt[cnt_len] uint32)."""
    L = lib()
    k, n = dip.shape
    dev = dip.device
    if cnt_len is None:
        cnt_len = ssm_aggregate_size(dip, stream)
    region = torch.empty(n, dtype=torch.int32, device=dev)
    off = torch.empty(k + 1, dtype=torch.int32, device=dev)
    cnt = torch.empty(cnt_len, dtype=torch.uint32, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_aggregate_workspace(k), dev)
    _rc(L.ssm_aggregate(n, k, _ptr(dip), _ptr(region), _ptr(off), _ptr(cnt), cnt_len, _ptr(st), _ptr(ws), ws.numel(),
                        _stream(stream)), "ssm_aggregate")
    if check:
        ssm_check(st, "ssm_aggregate", stream)
    return region, off, cnt


def ssm_regions_smallest(dip: torch.Tensor, stream=None, check: bool = True) -> torch.Tensor:
    """Regions with the paper's tie rule (ties to the region that is smallest at that moment)."""
    L = lib()
    k, n = dip.shape
    dev = dip.device
    region = torch.empty(n, dtype=torch.int32, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_regions_smallest_workspace(n), dev)
    _rc(L.ssm_regions_smallest(n, k, _ptr(dip), _ptr(region), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)),
        "ssm_regions_smallest")
    if check:
        ssm_check(st, "ssm_regions_smallest", stream)
    return region


def ssm_aggregate_regions(dip: torch.Tensor, region: torch.Tensor, stream=None, check: bool = True):
    """cnt_off and cnt (Section 3's counts) for given regions; returns (cnt_off, cnt)."""
    L = lib()
    k, n = dip.shape
    dev = dip.device
    off = torch.empty(k + 1, dtype=torch.int32, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_aggregate_workspace(k), dev)
    length = ctypes.c_int64(0)
    rc = L.ssm_aggregate_regions(n, k, _ptr(dip), _ptr(region), _ptr(off), None, 0, ctypes.byref(length), _ptr(st),
                                 _ptr(ws), ws.numel(), _stream(stream))
    if rc not in (0, -5):
        _rc(rc, "ssm_aggregate_regions")
    cnt = torch.empty(max(int(length.value), 1), dtype=torch.uint32, device=dev)
    _rc(L.ssm_aggregate_regions(n, k, _ptr(dip), _ptr(region), _ptr(off), _ptr(cnt), cnt.numel(), ctypes.byref(length),
                                _ptr(st), _ptr(ws), ws.numel(), _stream(stream)), "ssm_aggregate_regions")
    if check:
        ssm_check(st, "ssm_aggregate_regions", stream)
    return off, cnt[: int(length.value)]


def ssm_aggregate_noalloc(dip: torch.Tensor, region: torch.Tensor, cnt_off: torch.Tensor, cnt: torch.Tensor | None,
                          status: torch.Tensor, stream=None) -> int:
    """ssm_aggregate into caller buffers with no workspace (the library allocates
    nothing).  Returns the table length; raises SSMError (code -5) if cnt is
    missing or too small for it."""
    L = lib()
    k, n = dip.shape
    cap = 0 if cnt is None else cnt.numel()
    out = ctypes.c_int64(0)
    _rc(L.ssm_aggregate_noalloc(n, k, _ptr(dip), _ptr(region), _ptr(cnt_off), _ptr(cnt), cap, ctypes.byref(out),
                                _ptr(status), _stream(stream)), "ssm_aggregate_noalloc")
    return int(out.value)


def ssm_gram(dip: torch.Tensor, stream=None, check: bool = True):
    """Exact Gram matrix of the squared pivot distances, G[a][b] = sum_i d_ia^2 d_ib^2
    for a <= b, as two int64 tensors [k, k] holding the low and high 64 bits
    (reinterpret as unsigned); entries below the diagonal are zero."""
    L = lib()
    k, n = dip.shape
    dev = dip.device
    lo = torch.empty((k, k), dtype=torch.int64, device=dev)
    hi = torch.empty((k, k), dtype=torch.int64, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_gram_workspace(n, k), dev)
    _rc(L.ssm_gram(n, k, _ptr(dip), _ptr(lo), _ptr(hi), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)), "ssm_gram")
    if check:
        ssm_check(st, "ssm_gram", stream)
    return lo, hi


def ssm_pivotmds(g: Graph, dip: torch.Tensor, precision: int = 32, rescale: bool = True, stream=None,
                 check: bool = True):
    """Returns (pos [n,2] float32/float64, eig [4] float64: the two eigenvalues,
    subspace iterations used, final relative residual)."""
    L = lib()
    k, n = dip.shape
    dev = dip.device
    pos = torch.empty((n, 2), dtype=torch.float64 if precision == 64 else torch.float32, device=dev)
    eig = torch.empty(4, dtype=torch.float64, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_pivotmds_workspace(n, k), dev)
    _rc(L.ssm_pivotmds(n, _ptr(g.rowptr), _ptr(g.colidx), k, _ptr(dip), _ptr(pos), precision, int(bool(rescale)),
                       _ptr(eig), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)), "ssm_pivotmds")
    if check:
        ssm_check(st, "ssm_pivotmds", stream)
    return pos, eig


class IterateWorkspace:
    """Reusable device buffers for ssm_iterate (so timed loops allocate nothing)."""

    def __init__(self, n: int, m: int, k: int, cnt_len: int, precision: int, device):
        self.ws = _ws(lib().ssm_iterate_workspace(n, m, k, cnt_len, precision), device)
        self.iters_done = torch.zeros(1, dtype=torch.int32, device=device)
        self.rel = torch.zeros(1, dtype=torch.float64, device=device)
        self.status = _status(device)


def ssm_iterate(g: Graph, p: Pivots, pos: torch.Tensor, iters: int, tol: float = 0.0, stream=None,
                work: IterateWorkspace | None = None, check: bool = True):
    """Runs `iters` Jacobi sweeps of Eq. 4 on pos in place; returns (iters_done, rel_change) tensors."""
    L = lib()
    precision = 64 if pos.dtype == torch.float64 else 32
    if work is None:
        work = IterateWorkspace(g.n, g.m, p.k, p.cnt.numel(), precision, pos.device)
    hints = None
    if p.dmax is not None and g.row_classes is not None:  # no host wait inside the call
        hints = (ctypes.c_int32 * 3)(int(p.dmax), int(g.row_classes[0]), int(g.row_classes[1]))
    _rc(L.ssm_iterate(g.n, g.m, _ptr(g.rowptr), _ptr(g.colidx), p.k, _ptr(p.pivots), _ptr(p.dip), _ptr(p.cnt_off),
                      _ptr(p.cnt), p.cnt.numel(), _ptr(pos), precision, iters, float(tol), _ptr(work.iters_done), _ptr(work.rel),
                      _ptr(work.status), ctypes.cast(hints, ctypes.c_void_p) if hints is not None else None,
                      _ptr(work.ws), work.ws.numel(), _stream(stream)), "ssm_iterate")
    if check:
        ssm_check(work.status, "ssm_iterate", stream)
    return work.iters_done, work.rel


def ssm_iterate_hints(g: Graph, dip: torch.Tensor, stream=None) -> tuple:
    """(largest d_ip entry, rows with 33..1024 entries, rows with more): ssm_iterate's hints (synchronous)."""
    L = lib()
    k = dip.shape[0]
    ws = _ws(256, dip.device)
    h = (ctypes.c_int32 * 3)()
    _rc(L.ssm_iterate_hints(g.n, _ptr(g.rowptr), k, _ptr(dip), ctypes.cast(h, ctypes.c_void_p), _ptr(ws), ws.numel(),
                            _stream(stream)), "ssm_iterate_hints")
    return int(h[0]), int(h[1]), int(h[2])


def ssm_iterate_gs(g: Graph, p: Pivots, pos: torch.Tensor, iters: int, stream=None, check: bool = True):
    """`iters` in-place (Gauss-Seidel) sweeps of Eq. 4 in FP64 on pos (float64 [n, 2]);
    returns the relative change of the last sweep (device float64 tensor)."""
    L = lib()
    if pos.dtype != torch.float64:
        raise ValueError("ssm_iterate_gs runs in FP64: pos must be float64")
    dev = pos.device
    rel = torch.zeros(1, dtype=torch.float64, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_iterate_gs_workspace(g.n), dev)
    _rc(L.ssm_iterate_gs(g.n, g.m, _ptr(g.rowptr), _ptr(g.colidx), p.k, _ptr(p.pivots), _ptr(p.dip), _ptr(p.cnt_off),
                         _ptr(p.cnt), _ptr(pos), iters, _ptr(rel), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)),
        "ssm_iterate_gs")
    if check:
        ssm_check(st, "ssm_iterate_gs", stream)
    return rel


def ssm_apsp(g: Graph, stream=None, check: bool = True) -> torch.Tensor:
    """All-pairs hop distances [n, n] uint16: ssm_pivot_bfs with every node as a source."""
    return ssm_pivot_bfs(g, torch.arange(g.n, dtype=torch.int32, device=g.rowptr.device), stream, check)


def ssm_full_iterate(D: torch.Tensor, pos: torch.Tensor, iters: int, order: int = 0, stream=None, check: bool = True):
    """`iters` sweeps of full stress majorization over the all-pairs table D
    ([n, n] uint16) on pos in place (order 0 Jacobi FP32/FP64, order 1
    Gauss-Seidel FP64); returns the relative change of the last sweep."""
    L = lib()
    n = D.shape[0]
    precision = 64 if pos.dtype == torch.float64 else 32
    dev = pos.device
    rel = torch.zeros(1, dtype=torch.float64, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_full_iterate_workspace(n, precision), dev)
    _rc(L.ssm_full_iterate(n, _ptr(D), _ptr(pos), precision, order, iters, _ptr(rel), _ptr(st), _ptr(ws), ws.numel(),
                           _stream(stream)), "ssm_full_iterate")
    if check:
        ssm_check(st, "ssm_full_iterate", stream)
    return rel


def ssm_procrustes(X: torch.Tensor, Y: torch.Tensor, stream=None) -> torch.Tensor:
    """Procrustes statistic of two layouts [n, 2] (same dtype): device float64
    tensor {P, scale, angle}."""
    if X.dtype != Y.dtype or X.shape != Y.shape:
        raise ValueError("layouts must have the same shape and dtype")
    out = torch.zeros(3, dtype=torch.float64, device=X.device)
    precision = 64 if X.dtype == torch.float64 else 32
    _rc(lib().ssm_procrustes(X.shape[0], _ptr(X.contiguous()), _ptr(Y.contiguous()), precision, _ptr(out),
                             _stream(stream)), "ssm_procrustes")
    return out


def ssm_hull_error(D: torch.Tensor, pos: torch.Tensor, kh: int, stream=None, check: bool = True):
    """Convex-hull error of Fig. 4: returns (mean, per-node errors) as device float64 tensors."""
    L = lib()
    n = D.shape[0]
    dev = pos.device
    per = torch.empty(n, dtype=torch.float64, device=dev)
    mean = torch.zeros(1, dtype=torch.float64, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_hull_error_workspace(n), dev)
    precision = 64 if pos.dtype == torch.float64 else 32
    _rc(L.ssm_hull_error(n, _ptr(D), _ptr(pos.contiguous()), precision, kh, _ptr(per), _ptr(mean), _ptr(st), _ptr(ws),
                         ws.numel(), _stream(stream)), "ssm_hull_error")
    if check:
        ssm_check(st, "ssm_hull_error", stream)
    return mean, per


def ssm_gabriel_jaccard(posA: torch.Tensor, posB: torch.Tensor, kh: int, stream=None, check: bool = True):
    """Gabriel-graph Jaccard comparison of two layouts (Section 4): returns (mean, per-node) float64 tensors."""
    L = lib()
    n = posA.shape[0]
    if posB.shape != posA.shape or posB.dtype != posA.dtype:
        raise ValueError("ssm_gabriel_jaccard: layouts differ in shape or dtype")
    dev = posA.device
    per = torch.empty(n, dtype=torch.float64, device=dev)
    mean = torch.zeros(1, dtype=torch.float64, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_gabriel_jaccard_workspace(n), dev)
    precision = 64 if posA.dtype == torch.float64 else 32
    _rc(L.ssm_gabriel_jaccard(n, _ptr(posA.contiguous()), _ptr(posB.contiguous()), precision, kh, _ptr(per),
                              _ptr(mean), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)), "ssm_gabriel_jaccard")
    if check:
        ssm_check(st, "ssm_gabriel_jaccard", stream)
    return mean, per


class StressWorkspace:
    def __init__(self, n: int, m: int, nsources: int, ntargets: int, device):
        self.ws = _ws(lib().ssm_stress_workspace(n, m, nsources, ntargets), device)
        self.out = torch.zeros(4, dtype=torch.float64, device=device)
        self.sums = torch.zeros(4, dtype=torch.float64, device=device)
        self.status = _status(device)


def ssm_stress(g: Graph, pos: torch.Tensor, nsources: int = 0, ntargets: int = 0, seed: int = 0, stream=None,
               work: StressWorkspace | None = None, check: bool = True):
    """Returns (out[4], sums[4]) float64 device tensors: {raw, alpha*, scaled, normalized}."""
    L = lib()
    precision = 64 if pos.dtype == torch.float64 else 32
    if work is None:
        work = StressWorkspace(g.n, g.m, nsources, ntargets, pos.device)
    _rc(L.ssm_stress(g.n, g.m, _ptr(g.rowptr), _ptr(g.colidx), _ptr(pos), precision, nsources, ntargets,
                     ctypes.c_uint64(seed), _ptr(work.out), _ptr(work.sums), _ptr(work.status), _ptr(work.ws),
                     work.ws.numel(), _stream(stream)), "ssm_stress")
    if check:
        ssm_check(work.status, "ssm_stress", stream)
    return work.out, work.sums


_BATCH_DTYPE = None


def _batch_dtype():
    """numpy layout of ssm_batch_graph (include/ssm.h)."""
    import numpy as np
    global _BATCH_DTYPE
    if _BATCH_DTYPE is None:
        _BATCH_DTYPE = np.dtype([("n", "<i4"), ("k", "<i4"), ("cnt_len", "<i4"), ("reserved", "<i4"),
                                 ("node_off", "<i8"), ("row_off", "<i8"), ("col_off", "<i8"), ("piv_off", "<i8"),
                                 ("dip_off", "<i8"), ("cnt_off_off", "<i8"), ("cnt_base", "<i8")])
        assert _BATCH_DTYPE.itemsize == 72
    return _BATCH_DTYPE


def ssm_batch_iterate(items, iters: int, threads: int = 0, nodes_per_lane: int = 0, stream=None, check: bool = True):
    """Jacobi sweeps for a batch of small graphs in one launch (ssm_batch_iterate).

    items: list of (Graph, Pivots, pos float32 [n, 2]) on one device; every
    pos is updated in place.  threads / nodes_per_lane: 0 tunes (and caches)
    the block size / tile shape per size class.  Returns (rel_change float64
    [G] device tensor, (block size, nodes per lane) of the heaviest class)."""
    import numpy as np
    L = lib()
    G = len(items)
    dev = items[0][2].device
    desc = np.zeros(G, dtype=_batch_dtype())
    node = row = col = piv = dipo = offo = cbase = 0
    for i, (g, p, pos) in enumerate(items):
        if pos.dtype != torch.float32 or pos.shape != (g.n, 2):
            raise ValueError("batch positions must be float32 [n, 2]")
        desc[i] = (g.n, p.k, p.cnt.numel(), 0, node, row, col, piv, dipo, offo, cbase)
        node += g.n
        row += g.n + 1
        col += g.colidx.numel()
        piv += p.k
        dipo += p.k * g.n
        offo += p.k + 1
        cbase += p.cnt.numel()
    import contextlib
    ctx = torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()
    with ctx:
        return _batch_call(L, items, desc, col, iters, threads, nodes_per_lane, stream, check, dev)


def _batch_call(L, items, desc, col, iters, threads, nodes_per_lane, stream, check, dev):
    G = len(items)
    rowptr = torch.cat([g.rowptr for g, _, _ in items])
    colidx = torch.cat([g.colidx for g, _, _ in items]) if col else torch.zeros(1, dtype=torch.int32, device=dev)
    pivots = torch.cat([p.pivots for _, p, _ in items])
    dip = torch.cat([p.dip.view(torch.int16).reshape(-1) for _, p, _ in items])
    cnt_off = torch.cat([p.cnt_off for _, p, _ in items])
    cnt = torch.cat([p.cnt.view(torch.int32) for _, p, _ in items])
    pos_all = torch.cat([pos for _, _, pos in items])
    rel = torch.zeros(G, dtype=torch.float64, device=dev)
    st = _status(dev)
    dp = desc.ctypes.data_as(ctypes.c_void_p)
    ws = _ws(L.ssm_batch_iterate_workspace(G, dp), dev)
    used = (ctypes.c_int32 * 2)()
    _rc(L.ssm_batch_iterate(G, dp, _ptr(rowptr), _ptr(colidx), _ptr(pivots), _ptr(dip), _ptr(cnt_off), _ptr(cnt),
                            _ptr(pos_all), iters, _ptr(rel), threads, nodes_per_lane, used, _ptr(st), _ptr(ws),
                            ws.numel(), _stream(stream)), "ssm_batch_iterate")
    if check:
        ssm_check(st, "ssm_batch_iterate", stream)
    o = 0
    for g, _, pos in items:
        pos.copy_(pos_all[o:o + g.n])
        o += g.n
    return rel, (int(used[0]), int(used[1]))


class BatchPacked:
    """A batch prepared on the GPU (ssm_batch_pivots + ssm_batch_layout_init):
    the packed arrays ssm_batch_iterate reads, with their descriptors."""

    def __init__(self, desc, m, rowptr, colidx, pivots, dip, region, ecc, cnt_off, cnt, pos, eig):
        self.desc, self.m = desc, m
        self.rowptr, self.colidx, self.pivots, self.dip = rowptr, colidx, pivots, dip
        self.region, self.ecc, self.cnt_off, self.cnt, self.pos, self.eig = region, ecc, cnt_off, cnt, pos, eig

    def __len__(self):
        return len(self.desc)

    def graph(self, g: int) -> dict:
        """Views of graph g's pieces (local ids), for inspection and tests."""
        d = self.desc[g]
        n, k = int(d["n"]), int(d["k"])
        ro, co, po, do = int(d["row_off"]), int(d["col_off"]), int(d["piv_off"]), int(d["dip_off"])
        rowptr = self.rowptr[ro:ro + n + 1]
        m2 = 2 * int(self.m[g])
        oo, cb = int(d["cnt_off_off"]), int(d["cnt_base"])
        no = int(d["node_off"])
        return {"n": n, "k": k, "m": int(self.m[g]), "rowptr": rowptr, "colidx": self.colidx[co:co + m2],
                "pivots": self.pivots[po:po + k], "dip": self.dip[do:do + k * n].view(k, n),
                "region": self.region[no:no + n], "cnt_off": self.cnt_off[oo:oo + k + 1],
                "cnt": self.cnt[cb:cb + int(d["cnt_len"])], "pos": self.pos[no:no + n],
                "eig": self.eig[2 * g:2 * g + 2] if self.eig is not None else None}


def _batch_input_dtype():
    import numpy as np
    return np.dtype([("n", "<i4"), ("k", "<i4"), ("m_in", "<i8"), ("edge_off", "<i8")])


def ssm_batch_prepare(graphs, device="cuda", stream=None, check: bool = True) -> BatchPacked:
    """Algorithm 1 lines 1-4 for a batch of small graphs in two launches.
    graphs: list of (n, src, dst, k) with host edge arrays (local ids)."""
    import numpy as np
    _require_cuda()
    L = lib()
    G = len(graphs)
    inp = np.zeros(G, dtype=_batch_input_dtype())
    eo = 0
    for i, (n, s_, d_, k) in enumerate(graphs):
        inp[i] = (n, k, len(s_), eo)
        eo += len(s_)
    src = torch.from_numpy(np.concatenate([np.asarray(g[1], np.int32) for g in graphs]) if eo else
                           np.zeros(1, np.int32)).to(device)
    dst = torch.from_numpy(np.concatenate([np.asarray(g[2], np.int32) for g in graphs]) if eo else
                           np.zeros(1, np.int32)).to(device)
    ns = inp["n"].astype(np.int64)
    ks = inp["k"].astype(np.int64)
    nodes, rows, cols = int(ns.sum()), int((ns + 1).sum()), max(1, int(2 * inp["m_in"].sum()))
    pivs, dips, offs = int(ks.sum()), int((ks * ns).sum()), int((ks + 1).sum())
    rowptr = torch.empty(rows, dtype=torch.int32, device=device)
    colidx = torch.empty(cols, dtype=torch.int32, device=device)
    pivots = torch.empty(pivs, dtype=torch.int32, device=device)
    dip = torch.empty(dips, dtype=torch.uint16, device=device)
    region = torch.empty(nodes, dtype=torch.int32, device=device)
    ecc = torch.empty(pivs, dtype=torch.int32, device=device)
    desc = np.zeros(G, dtype=_batch_dtype())
    m = np.zeros(G, np.int64)
    st = _status(device)
    ip = inp.ctypes.data_as(ctypes.c_void_p)
    ws = _ws(L.ssm_batch_prepare_workspace(G, ip), device)
    _rc(L.ssm_batch_pivots(G, ip, _ptr(src), _ptr(dst), desc.ctypes.data_as(ctypes.c_void_p), _ptr(rowptr),
                           _ptr(colidx), _ptr(pivots), _ptr(dip), _ptr(region), _ptr(ecc),
                           m.ctypes.data_as(ctypes.c_void_p), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)),
        "ssm_batch_pivots")
    cnt_off = torch.empty(offs, dtype=torch.int32, device=device)
    cnt = torch.empty(max(1, int(desc["cnt_len"].astype(np.int64).sum())), dtype=torch.uint32, device=device)
    pos = torch.empty((nodes, 2), dtype=torch.float32, device=device)
    eig = torch.zeros(2 * G, dtype=torch.float64, device=device)
    _rc(L.ssm_batch_layout_init(G, desc.ctypes.data_as(ctypes.c_void_p), m.ctypes.data_as(ctypes.c_void_p),
                                _ptr(rowptr), _ptr(colidx), _ptr(dip), _ptr(region), _ptr(ecc), _ptr(cnt_off),
                                _ptr(cnt), _ptr(pos), _ptr(eig), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)),
        "ssm_batch_layout_init")
    if check:
        ssm_check(st, "ssm_batch_layout_init", stream)
    return BatchPacked(desc, m, rowptr, colidx, pivots, dip, region, ecc, cnt_off, cnt, pos, eig)


def ssm_batch_iterate_packed(bp: BatchPacked, iters: int, threads: int = 0, nodes_per_lane: int = 0, stream=None,
                             check: bool = True):
    """ssm_batch_iterate on a prepared batch, positions updated in place in bp.pos;
    returns (rel_change float64 [G], (block size, nodes per lane) of the heaviest class)."""
    L = lib()
    G = len(bp)
    dev = bp.pos.device
    rel = torch.zeros(G, dtype=torch.float64, device=dev)
    st = _status(dev)
    dp = bp.desc.ctypes.data_as(ctypes.c_void_p)
    ws = _ws(L.ssm_batch_iterate_workspace(G, dp), dev)
    used = (ctypes.c_int32 * 2)()
    _rc(L.ssm_batch_iterate(G, dp, _ptr(bp.rowptr), _ptr(bp.colidx), _ptr(bp.pivots), _ptr(bp.dip), _ptr(bp.cnt_off),
                            _ptr(bp.cnt), _ptr(bp.pos), iters, _ptr(rel), threads, nodes_per_lane, used, _ptr(st),
                            _ptr(ws), ws.numel(), _stream(stream)), "ssm_batch_iterate")
    if check:
        ssm_check(st, "ssm_batch_iterate", stream)
    return rel, (int(used[0]), int(used[1]))


def prepare(n: int, src, dst, k: int, start: int = 0, precision: int = 32, device="cuda", stream=None,
            sampler: str = "maxmin", kmeans_iters: int = 50):
    """Algorithm 1 lines 1-4 on the GPU: returns (Graph, Pivots, initial positions, eigenvalues).
    sampler: "maxmin" (max/min sp) or "kmeans" (k-means sp: max/min sp refined
    by k-means over the pivots' distances, then d_ip of the new pivots)."""
    _require_cuda()
    if sampler not in ("maxmin", "kmeans"):
        raise ValueError("sampler must be 'maxmin' or 'kmeans'")
    src = torch.as_tensor(src, dtype=torch.int32).to(device, non_blocking=True)
    dst = torch.as_tensor(dst, dtype=torch.int32).to(device, non_blocking=True)
    g = ssm_build_graph(n, src, dst, stream)
    piv = ssm_select_pivots(g, k, start, stream)
    dip = ssm_pivot_bfs(g, piv, stream)
    if sampler == "kmeans":
        piv, _, _ = ssm_kmeans_pivots(dip, piv, kmeans_iters, stream)
        dip = ssm_pivot_bfs(g, piv, stream)
    cnt_len, dmax = ssm_aggregate_size(dip, stream, with_dmax=True)
    region, off, cnt = ssm_aggregate(dip, cnt_len, stream=stream)
    pos, eig = ssm_pivotmds(g, dip, precision, True, stream)
    return g, Pivots(k, piv, dip, region, off, cnt, dmax), pos, eig


def layout(n: int, src, dst, k: int = 200, iters: int = 100, tol: float = 0.0, start: int = 0,
           precision: int = 32, device="cuda"):
    """Whole pipeline (Algorithm 1, Jacobi schedule); returns positions [n,2] on the device."""
    g, p, pos, _ = prepare(n, src, dst, k, start, precision, device)
    ssm_iterate(g, p, pos, iters, tol)
    return pos


# ---------------------------------------------------------------- weighted graphs
@dataclass
class WGraph(Graph):
    elen: torch.Tensor = None  # float32 [2m], the length of edge colidx[t]


def ssm_build_wgraph(n: int, src: torch.Tensor, dst: torch.Tensor, lengths: torch.Tensor, stream=None,
                     check: bool = True) -> WGraph:
    """CSR of the weighted simple undirected graph (a repeated edge keeps its
    shortest length): ssm_build_graph, then ssm_edge_lengths."""
    g = ssm_build_graph(n, src, dst, stream)
    L = lib()
    dev = src.device
    src = src.contiguous().to(torch.int32)
    dst = dst.contiguous().to(torch.int32)
    lengths = lengths.contiguous().to(torch.float32)
    elen = torch.empty(max(2 * g.m, 1), dtype=torch.float32, device=dev)
    st = _status(dev)
    ws = _ws(256, dev)
    _rc(L.ssm_edge_lengths(n, src.numel(), _ptr(src), _ptr(dst), _ptr(lengths), g.m, _ptr(g.rowptr), _ptr(g.colidx),
                           _ptr(elen), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)), "ssm_edge_lengths")
    if check:
        ssm_check(st, "ssm_edge_lengths", stream)
    return WGraph(g.n, g.m, g.rowptr, g.colidx, row_classes=g.row_classes, elen=elen[: 2 * g.m])


def ssm_pivot_sssp(g: WGraph, sources: torch.Tensor, stream=None, check: bool = True) -> torch.Tensor:
    """Weighted distances [k, n] float32 from each source (least float32 path sums)."""
    L = lib()
    dev = g.rowptr.device
    k = sources.numel()
    dist = torch.empty((k, g.n), dtype=torch.float32, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_pivot_sssp_workspace(g.n, k), dev)
    _rc(L.ssm_pivot_sssp(g.n, g.m, _ptr(g.rowptr), _ptr(g.colidx), _ptr(g.elen), k, _ptr(sources.contiguous()),
                         _ptr(dist), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)), "ssm_pivot_sssp")
    if check:
        ssm_check(st, "ssm_pivot_sssp", stream)
    return dist


def ssm_select_pivots_weighted(g: WGraph, k: int, start: int = 0, stream=None, check: bool = True) -> torch.Tensor:
    L = lib()
    dev = g.rowptr.device
    piv = torch.empty(k, dtype=torch.int32, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_select_pivots_weighted_workspace(g.n, k), dev)
    _rc(L.ssm_select_pivots_weighted(g.n, g.m, _ptr(g.rowptr), _ptr(g.colidx), _ptr(g.elen), k, start, _ptr(piv),
                                     _ptr(st), _ptr(ws), ws.numel(), _stream(stream)), "ssm_select_pivots_weighted")
    if check:
        ssm_check(st, "ssm_select_pivots_weighted", stream)
    return piv


def ssm_weighted_counts(g: WGraph, pivots: torch.Tensor, dist: torch.Tensor, stream=None, check: bool = True):
    """Returns (region[n] int32, s[k, n] uint32) of Section 3 on weighted distances."""
    L = lib()
    k, n = dist.shape
    dev = dist.device
    region = torch.empty(n, dtype=torch.int32, device=dev)
    s_tab = torch.empty((k, n), dtype=torch.uint32, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_weighted_counts_workspace(n, k), dev)
    _rc(L.ssm_weighted_counts(n, _ptr(g.rowptr), _ptr(g.colidx), k, _ptr(pivots.contiguous()), _ptr(dist),
                              _ptr(region), _ptr(s_tab), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)),
        "ssm_weighted_counts")
    if check:
        ssm_check(st, "ssm_weighted_counts", stream)
    return region, s_tab


def ssm_pivotmds_weighted(g: WGraph, dist: torch.Tensor, precision: int = 32, rescale: bool = True, stream=None,
                          check: bool = True):
    """PivotMDS from the weighted distance table: returns (pos [n, 2], eig [4] float64)."""
    L = lib()
    k, n = dist.shape
    dev = dist.device
    pos = torch.empty((n, 2), dtype=torch.float64 if precision == 64 else torch.float32, device=dev)
    eig = torch.zeros(4, dtype=torch.float64, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_pivotmds_weighted_workspace(n, k), dev)
    _rc(L.ssm_pivotmds_weighted(n, _ptr(g.rowptr), _ptr(g.colidx), _ptr(g.elen), k, _ptr(dist), _ptr(pos), precision,
                                int(rescale), _ptr(eig), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)),
        "ssm_pivotmds_weighted")
    if check:
        ssm_check(st, "ssm_pivotmds_weighted", stream)
    return pos, eig


def ssm_iterate_weighted(g: WGraph, pivots: torch.Tensor, dist: torch.Tensor, s_tab: torch.Tensor,
                         pos: torch.Tensor, iters: int, stream=None, check: bool = True) -> torch.Tensor:
    """`iters` Jacobi updates of Eq. 4 on a weighted graph, in place on pos;
    returns the last relative change (device float64 [1])."""
    L = lib()
    k, n = dist.shape
    dev = pos.device
    precision = 64 if pos.dtype == torch.float64 else 32
    rel = torch.zeros(1, dtype=torch.float64, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_iterate_weighted_workspace(n, k, precision), dev)
    _rc(L.ssm_iterate_weighted(n, _ptr(g.rowptr), _ptr(g.colidx), _ptr(g.elen), k, _ptr(pivots.contiguous()),
                               _ptr(dist), _ptr(s_tab), _ptr(pos), precision, iters, _ptr(rel), _ptr(st), _ptr(ws),
                               ws.numel(), _stream(stream)), "ssm_iterate_weighted")
    if check:
        ssm_check(st, "ssm_iterate_weighted", stream)
    return rel


def ssm_stress_weighted(g: WGraph, pos: torch.Tensor, nsources: int = 0, ntargets: int = 0, seed: int = 0,
                        stream=None, check: bool = True):
    """{raw, alpha*, scaled, normalized} and the four pair sums (float64 device tensors)."""
    L = lib()
    dev = pos.device
    precision = 64 if pos.dtype == torch.float64 else 32
    out = torch.zeros(4, dtype=torch.float64, device=dev)
    sums = torch.zeros(4, dtype=torch.float64, device=dev)
    st = _status(dev)
    ws = _ws(L.ssm_stress_weighted_workspace(g.n, nsources), dev)
    _rc(L.ssm_stress_weighted(g.n, _ptr(g.rowptr), _ptr(g.colidx), _ptr(g.elen), _ptr(pos.contiguous()), precision,
                              nsources, ntargets, ctypes.c_uint64(seed), _ptr(out), _ptr(sums), _ptr(st), _ptr(ws),
                              ws.numel(), _stream(stream)), "ssm_stress_weighted")
    if check:
        ssm_check(st, "ssm_stress_weighted", stream)
    return out, sums


def layout_weighted(n: int, src, dst, lengths, k: int, iters: int, start: int = 0, device="cuda"):
    """Algorithm 1 on a weighted graph, every step on the GPU: returns
    (graph, pivots, dist, region, s, positions float32 [n, 2], eigenvalues)."""
    _require_cuda()
    src = torch.as_tensor(src, dtype=torch.int32).to(device)
    dst = torch.as_tensor(dst, dtype=torch.int32).to(device)
    lengths = torch.as_tensor(lengths, dtype=torch.float32).to(device)
    g = ssm_build_wgraph(n, src, dst, lengths)
    piv = ssm_select_pivots_weighted(g, k, start)
    dist = ssm_pivot_sssp(g, piv)
    region, s_tab = ssm_weighted_counts(g, piv, dist)
    pos, eig = ssm_pivotmds_weighted(g, dist, 32, True)
    ssm_iterate_weighted(g, piv, dist, s_tab, pos, iters)
    return g, piv, dist, region, s_tab, pos, eig
