"""The timeout path of the device-wide barriers, made to run out on purpose.

ssm_set_wait_limit_ns sets the longest wait at a barrier of the persistent
kernels; with a limit of one nanosecond the first block that has to wait for
another gives up, records SSM_E_TIMEOUT in the status word, raises the abort
flag that releases every other block, and the kernel returns.  The test then
checks that the call reports SSM_E_TIMEOUT (-7), and that with the default
limit restored the same calls on the same context give the oracle's results.
No kernel is left waiting: every wait ends by the limit or by the abort flag.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture
def short_waits():
    prev = ssm.ssm_set_wait_limit_ns(1)
    yield
    ssm.ssm_set_wait_limit_ns(prev)
    assert ssm.ssm_set_wait_limit_ns(prev) == prev


def _graph(n, s, d):
    return ssm.ssm_build_graph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV))


def test_pulled_bfs_barrier_times_out(short_waits):
    """ssm_pivot_bfs on a small-diameter graph runs the cooperative pulled
    bitset BFS, whose levels end at a grid barrier."""
    n, s, d = I.ba(20000, 4, 3)
    g = _graph(n, s, d)
    og = O.build_csr(n, s, d)
    piv = O.maxmin(og, 64, 0)
    with pytest.raises(ssm.SSMError) as e:
        ssm.ssm_pivot_bfs(g, torch.from_numpy(piv).to(DEV))
    assert e.value.code == -7
    ssm.ssm_set_wait_limit_ns(0)
    dip = ssm.ssm_pivot_bfs(g, torch.from_numpy(piv).to(DEV)).cpu().numpy()
    assert np.array_equal(dip, O.pivot_dist(og, piv))


def test_eigen_solver_barrier_times_out(short_waits):
    """ssm_pivotmds's FP64 subspace iteration runs on a cooperative grid whose
    steps end at grid barriers."""
    n, s, d = I.grid(32, 32)
    og = O.build_csr(n, s, d)
    dip = O.pivot_dist(og, O.maxmin(og, 50, 0))
    g = _graph(n, s, d)
    with pytest.raises(ssm.SSMError) as e:
        ssm.ssm_pivotmds(g, torch.from_numpy(dip).to(DEV), precision=64, rescale=False)
    assert e.value.code == -7
    ssm.ssm_set_wait_limit_ns(0)
    pos, eig = ssm.ssm_pivotmds(g, torch.from_numpy(dip).to(DEV), precision=64, rescale=False)
    _, oeig = O.pivotmds(dip)
    np.testing.assert_allclose(eig.cpu().numpy()[:2], oeig, rtol=1e-10)
