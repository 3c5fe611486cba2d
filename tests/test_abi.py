"""The C ABI: the library builds, loads and exports every function that
include/ssm.h declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1608_08909_gb300 as ssm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ssm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_pipeline():
    names = declared_functions()
    for fn in ("ssm_build_graph", "ssm_select_pivots", "ssm_pivot_bfs", "ssm_aggregate", "ssm_pivotmds",
               "ssm_iterate", "ssm_stress"):
        assert fn in names


def test_library_exports_every_declared_symbol():
    L = ssm.lib()
    missing = [f for f in declared_functions() if not hasattr(L, f)]
    assert not missing, missing


def test_status_strings_and_workspace_queries():
    L = ssm.lib()
    assert L.ssm_status_string(0) == b"ok"
    assert L.ssm_status_string(-3) == b"graph is disconnected"
    assert L.ssm_iterate_workspace(1000, 2000, 50, 600, 32) > 8000
    assert L.ssm_iterate_workspace(1000, 2000, 50, 600, 64) > 8000
    assert L.ssm_pivot_bfs_workspace(1000, 2000, 64) >= L.ssm_pivot_bfs_workspace(1000, 2000, 32) > 0
    assert L.ssm_build_graph_workspace(0, 5) == 0


@pytest.mark.parametrize("call", [
    lambda L: L.ssm_select_pivots(10, 9, None, None, 3, 0, None, None, None, 0, None),
    lambda L: L.ssm_pivot_bfs(10, 9, None, None, 3, None, None, None, None, 0, None),
    lambda L: L.ssm_iterate(10, 9, None, None, 3, None, None, None, None, 3, None, 32, 1, 0.0, None, None, None,
                            None, None, 0, None),
    lambda L: L.ssm_iterate_hints(10, None, 3, None, None, None, 0, None),
    lambda L: L.ssm_build_graph(0, 5, None, None, None, None, None, None, None, 0, None),
    lambda L: L.ssm_stress(1, 0, None, None, None, 32, 0, 0, 0, None, None, None, None, 0, None),
    lambda L: L.ssm_pivotmds(10, None, None, 1, None, None, 32, 0, None, None, None, 0, None),
])
def test_bad_arguments_rejected_on_host(call):
    L = ssm.lib()
    assert call(L) == -1
    assert len(L.ssm_last_error()) > 0


def _batch_desc(specs):
    desc = np.zeros(len(specs), dtype=ssm._batch_dtype())
    for i, (n, k, cnt_len) in enumerate(specs):
        desc[i] = (n, k, cnt_len, 0, 0, 0, 0, 0, 0, 0, 0)
    return desc


@pytest.mark.parametrize("specs,threads,npl,what", [
    ([(12289, 10, 20)], 0, 0, "n = 12289"),     # above the shared-memory positions limit
    ([(100, 0, 20)], 0, 0, "k = 0"),
    ([(100, 101, 200)], 0, 0, "k = 101"),       # more pivots than nodes
    ([(100, 10, 5)], 0, 0, "cnt_len < k"),
    ([(100, 10, 20)], 192, 0, "threads"),       # not a tuned block size
    ([(100, 10, 20)], 256, 3, "nodes per lane"),  # not a tile shape
])
def test_batch_arguments_rejected_on_host(specs, threads, npl, what):
    """ssm_batch_iterate checks every descriptor before touching the device
    (the dummy device pointers below are never dereferenced)."""
    L = ssm.lib()
    desc = _batch_desc(specs)
    dp = desc.ctypes.data_as(ctypes.c_void_p)
    fake = ctypes.c_void_p(256)
    rc = L.ssm_batch_iterate(len(specs), dp, fake, fake, fake, fake, fake, fake, fake, 1, fake, threads, npl, None,
                             fake, fake, 1 << 20, None)
    assert rc == -1
    assert len(L.ssm_last_error()) > 0


def test_batch_workspace_grows_with_the_batch():
    L = ssm.lib()
    one = _batch_desc([(1000, 50, 1100)])
    two = _batch_desc([(1000, 50, 1100), (4000, 100, 4200)])
    w1 = L.ssm_batch_iterate_workspace(1, one.ctypes.data_as(ctypes.c_void_p))
    w2 = L.ssm_batch_iterate_workspace(2, two.ctypes.data_as(ctypes.c_void_p))
    # the tiled d_ip copy alone: 2 k n (rounded up to 128-node tiles, room for either tile shape) per graph
    assert w1 >= 2 * 50 * 1024 and w2 >= w1 + 2 * 100 * 4096


def test_gram_arguments_rejected_on_host():
    L = ssm.lib()
    fake = ctypes.c_void_p(256)
    assert L.ssm_gram(10, 0, fake, fake, fake, fake, fake, 256, None) == -1
    assert L.ssm_gram(10, 1025, fake, fake, fake, fake, fake, 256, None) == -1
    assert L.ssm_gram(10, 5, fake, fake, fake, fake, fake, 16, None) == -5  # workspace too small
