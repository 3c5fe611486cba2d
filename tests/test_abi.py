"""The C ABI: the library builds, loads and exports every function that
include/ssm.h declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

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
                            None, 0, None),
    lambda L: L.ssm_stress(1, 0, None, None, None, 32, 0, 0, 0, None, None, None, None, 0, None),
    lambda L: L.ssm_pivotmds(10, None, None, 1, None, None, 32, 0, None, None, None, 0, None),
])
def test_bad_arguments_rejected_on_host(call):
    L = ssm.lib()
    assert call(L) == -1
    assert len(L.ssm_last_error()) > 0
