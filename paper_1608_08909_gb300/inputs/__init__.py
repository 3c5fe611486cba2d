"""Seeded synthetic graphs shaped like the paper's workloads (Section 4, Table 1).

The paper evaluates on SuiteSparse meshes, power grids, heavy-tailed networks
and a complete binary tree; those files are not available, so seeded
generators stand in for them:

* ``grid(rows, cols)``        -- 4-neighbour grid (mesh-like, like 3elt/bodyy5)
* ``path(n)``                 -- path graph (closed-form distances)
* ``complete_btree(depth)``   -- the paper's "btree" for depth 9 (n=1023)
* ``random_btree(n, seed)``   -- random binary tree
* ``rgg(n, mean_deg, seed)``  -- random geometric graph, largest component kept
* ``ba(n, attach, seed)``     -- Barabasi-Albert preferential attachment
* ``induced_prefix(...)``     -- the subgraph induced by nodes 0..n_keep-1
* ``distance_table(k, n, dmax, seed)`` -- a uniform random k x n uint16 table
  (values 0..dmax, dmax present) for exactness tests of the dense contraction
* ``mixed_graph(family, n, seed)`` / ``request_stream(count, seed, ...)`` -- the
  mixed families (near-square grid, random binary tree, RGG of mean degree 6)
  and a seeded stream of layout requests (log-uniform sizes, unit-rate
  exponential inter-arrival gaps) for the serving and batching workloads

Each returns ``(n, src, dst)`` with int32 numpy edge arrays.  This module holds
none of the layout method's arithmetic; it is the one piece both the CUDA path
and the CPU oracle consume.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_OUT = os.path.join(_HERE, "_build", "libssmgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library next to it (gcc, portable flags)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            i32p = P(ctypes.c_int32)
            i32pp = P(i32p)
            i64p = P(ctypes.c_int64)
            lib.gen_free.argtypes = [ctypes.c_void_p]
            lib.gen_grid.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i64p, i32pp, i32pp]
            lib.gen_path.argtypes = [ctypes.c_int32, i32p, i64p, i32pp, i32pp]
            lib.gen_complete_btree.argtypes = [ctypes.c_int32, i32p, i64p, i32pp, i32pp]
            lib.gen_random_btree.argtypes = [ctypes.c_int32, ctypes.c_uint64, i32p, i64p, i32pp, i32pp]
            lib.gen_rgg.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                    i32p, i64p, i32pp, i32pp]
            lib.gen_rgg_lengths.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                            i32p, i64p, i32pp, i32pp,
                                            ctypes.POINTER(ctypes.POINTER(ctypes.c_float))]
            lib.gen_ba.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p, i64p, i32pp, i32pp]
            lib.gen_induced_prefix.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i64p, i32pp, i32pp]
            _lib = lib
    return _lib


def _call(fn, *args):
    n = ctypes.c_int32(0)
    m = ctypes.c_int64(0)
    s = ctypes.POINTER(ctypes.c_int32)()
    d = ctypes.POINTER(ctypes.c_int32)()
    rc = fn(*args, ctypes.byref(n), ctypes.byref(m), ctypes.byref(s), ctypes.byref(d))
    if rc != 0:
        raise ValueError(f"generator failed with status {rc}")
    lib = _load()
    try:
        src = np.ctypeslib.as_array(s, shape=(max(m.value, 1),))[: m.value].copy()
        dst = np.ctypeslib.as_array(d, shape=(max(m.value, 1),))[: m.value].copy()
    finally:
        lib.gen_free(ctypes.cast(s, ctypes.c_void_p))
        lib.gen_free(ctypes.cast(d, ctypes.c_void_p))
    return int(n.value), src, dst


def grid(rows: int, cols: int):
    return _call(_load().gen_grid, rows, cols)


def path(n: int):
    return _call(_load().gen_path, n)


def complete_btree(depth: int):
    return _call(_load().gen_complete_btree, depth)


def random_btree(n: int, seed: int):
    return _call(_load().gen_random_btree, n, ctypes.c_uint64(seed))


def rgg(n: int, mean_deg: float, seed: int, radius: float = 0.0):
    return _call(_load().gen_rgg, n, mean_deg, radius, ctypes.c_uint64(seed))


def rgg_lengths(n: int, mean_deg: float, seed: int, radius: float = 0.0):
    """The graph of rgg(n, mean_deg, seed, radius) with float32 edge lengths
    (Euclidean length / radius): returns (n, src, dst, len)."""
    lib = _load()
    nn = ctypes.c_int32(0)
    m = ctypes.c_int64(0)
    s = ctypes.POINTER(ctypes.c_int32)()
    d = ctypes.POINTER(ctypes.c_int32)()
    ln = ctypes.POINTER(ctypes.c_float)()
    rc = lib.gen_rgg_lengths(n, mean_deg, radius, ctypes.c_uint64(seed), ctypes.byref(nn), ctypes.byref(m),
                             ctypes.byref(s), ctypes.byref(d), ctypes.byref(ln))
    if rc != 0:
        raise ValueError(f"generator failed with status {rc}")
    try:
        mm = max(m.value, 1)
        src = np.ctypeslib.as_array(s, shape=(mm,))[: m.value].copy()
        dst = np.ctypeslib.as_array(d, shape=(mm,))[: m.value].copy()
        lens = np.ctypeslib.as_array(ln, shape=(mm,))[: m.value].copy()
    finally:
        for ptr in (s, d, ln):
            lib.gen_free(ctypes.cast(ptr, ctypes.c_void_p))
    return int(nn.value), src, dst, lens


def random_lengths(m: int, seed: int, kind: str = "uniform", lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Seeded float32 edge lengths: "uniform" in [lo, hi), or "integer" in
    {1, ..., int(hi)} (sums stay exact in float32 on small graphs)."""
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.uniform(lo, hi, size=m).astype(np.float32)
    if kind == "integer":
        return rng.integers(1, int(hi) + 1, size=m).astype(np.float32)
    raise ValueError(f"unknown length kind {kind!r}")


def ba(n: int, attach: int, seed: int):
    return _call(_load().gen_ba, n, attach, ctypes.c_uint64(seed))


def induced_prefix(n_keep: int, src: np.ndarray, dst: np.ndarray):
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = ctypes.c_int64(0)
    s = ctypes.POINTER(ctypes.c_int32)()
    d = ctypes.POINTER(ctypes.c_int32)()
    i32p = ctypes.POINTER(ctypes.c_int32)
    rc = lib.gen_induced_prefix(n_keep, len(src), src.ctypes.data_as(i32p), dst.ctypes.data_as(i32p),
                                ctypes.byref(m), ctypes.byref(s), ctypes.byref(d))
    if rc != 0:
        raise ValueError(f"induced_prefix failed with status {rc}")
    try:
        a = np.ctypeslib.as_array(s, shape=(max(m.value, 1),))[: m.value].copy()
        b = np.ctypeslib.as_array(d, shape=(max(m.value, 1),))[: m.value].copy()
    finally:
        lib.gen_free(ctypes.cast(s, ctypes.c_void_p))
        lib.gen_free(ctypes.cast(d, ctypes.c_void_p))
    return n_keep, a, b


def distance_table(k: int, n: int, dmax: int, seed: int) -> np.ndarray:
    """Uniform random pivot-major uint16 table [k, n] with entries in 0..dmax
    and dmax itself at one seeded position (not a metric; it exercises every
    bit of every squared entry)."""
    rng = np.random.default_rng(seed)
    t = rng.integers(0, dmax + 1, size=(k, n), dtype=np.int64)
    t[rng.integers(0, k), rng.integers(0, n)] = dmax
    return t.astype(np.uint16)


FAMILIES = ("grid", "btree", "rgg")


def mixed_graph(family: str, n: int, seed: int):
    """One graph of the mixed serving / batching families, about n nodes:
    a near-square grid (rows = floor(sqrt(n))), a random binary tree (node i
    hangs below a uniformly chosen earlier node with fewer than two children),
    or the largest component of an RGG of mean degree 6."""
    if family == "grid":
        r = max(1, int(np.floor(np.sqrt(n))))
        return grid(r, max(1, n // r))
    if family == "btree":
        return random_btree(n, seed)
    if family == "rgg":
        return rgg(n, 6.0, seed)
    raise KeyError(family)


def request_stream(count: int, seed: int, n_min: int = 1000, n_max: int = 200000):
    """Seeded layout requests: a list of dicts (family, n, seed, gap) with n
    log-uniform in [n_min, n_max], the family drawn uniformly from FAMILIES and
    gap an exponential inter-arrival time of unit rate (scale by 1/rate)."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        out.append(dict(family=FAMILIES[int(rng.integers(0, len(FAMILIES)))], n=n,
                        seed=int(rng.integers(1, 2 ** 62)), gap=float(rng.exponential(1.0))))
    return out


# Named workloads (the sizes of the configurations this library is measured on)
def workload(name: str, seed: int = 1):
    """Edge list of a named synthetic workload: returns (n, src, dst, k, iters).

    * ``grid32``  : 32x32 grid, k=50, 200 iterations (exhaustive stress)
    * ``rgg256k`` : RGG n=262144, mean degree 8, LCC, k=200, 100 iterations
    * ``ba1m``    : Barabasi-Albert n=2^20, 4 edges per new node, k=200, 100 iterations
    * ``ba64k``   : nodes 0..65535 of ``ba1m`` (the induced prefix subgraph), k=200
    """
    if name == "grid32":
        n, s, d = grid(32, 32)
        return n, s, d, 50, 200
    if name == "rgg256k":
        n, s, d = rgg(262144, 8.0, seed)
        return n, s, d, 200, 100
    if name == "ba1m":
        n, s, d = ba(1 << 20, 4, seed)
        return n, s, d, 200, 100
    if name == "ba64k":
        n, s, d = ba(1 << 20, 4, seed)
        n, s, d = induced_prefix(65536, s, d)
        return n, s, d, 200, 100
    raise KeyError(name)
