"""ssm_aggregate_noalloc: the variant of ssm_aggregate that takes no workspace.

It serves callers that cannot allocate device memory (for example a server
that reserved its whole memory budget up front); its scratch is a fixed device
array inside the library.  Its outputs must equal those of ssm_aggregate, bit
for bit (they are integers), on consecutive calls that reuse that array.
This file is collected last so that a run stopping at the first failure has
run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _dip(n, s, d, k):
    g = ssm.ssm_build_graph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV))
    piv = ssm.ssm_select_pivots(g, k)
    return ssm.ssm_pivot_bfs(g, piv)


@pytest.mark.parametrize("name,k", [("grid", 50), ("rgg", 100), ("ba", 64)])
def test_noalloc_equals_aggregate_on_repeated_calls(name, k):
    n, s, d = {"grid": lambda: I.grid(32, 32), "rgg": lambda: I.rgg(6000, 8.0, 7),
               "ba": lambda: I.ba(20000, 4, 3)}[name]()
    dip = _dip(n, s, d, k)
    region, off, cnt = ssm.ssm_aggregate(dip)
    torch.cuda.synchronize()
    # caller-owned outputs, allocated once by the caller
    r2 = torch.empty_like(region)
    o2 = torch.empty_like(off)
    c2 = torch.empty(cnt.numel() + 7, dtype=torch.uint32, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    for _ in range(2):
        r2.fill_(-1)
        o2.fill_(-1)
        c2.fill_(12345)
        length = ssm.ssm_aggregate_noalloc(dip, r2, o2, c2, st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert length == cnt.numel()
        assert torch.equal(r2, region)
        assert torch.equal(o2, off)
        assert torch.equal(c2[:length], cnt)


def test_noalloc_size_query_and_limits():
    n, s, d = I.grid(20, 30)
    dip = _dip(n, s, d, 12)
    _, off, cnt = ssm.ssm_aggregate(dip)
    L = ssm.lib()
    region = torch.empty(n, dtype=torch.int32, device=DEV)
    o2 = torch.empty(13, dtype=torch.int32, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    length = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    # no table buffer: the call reports the length it needs and leaves cnt alone
    rc = L.ssm_aggregate_noalloc(n, 12, p(dip), p(region), p(o2), None, 0, ctypes.byref(length), p(st), stream)
    assert rc == -5
    assert length.value == cnt.numel()
    # more pivots than the fixed scratch holds: rejected on the host
    big = torch.zeros((4097, 2), dtype=torch.uint16, device=DEV)
    rc = L.ssm_aggregate_noalloc(2, 4097, p(big), p(region), p(o2), None, 0, ctypes.byref(length), p(st), stream)
    assert rc == -1
    assert b"4096" in L.ssm_last_error()
