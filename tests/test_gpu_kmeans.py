"""k-means sp pivot sampling (Section 4.1) on the GPU against the oracle:
new pivots, the final cluster of every node and the number of passes must
match exactly (integers; the one floating-point decision per (node, cluster)
is taken by both sides in the same FP64 operations on exact integers)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"

GRAPHS = {
    "path7": (lambda: I.path(7), 2),
    "grid": (lambda: I.grid(32, 32), 50),
    "grid_ragged": (lambda: I.grid(17, 45), 33),
    "rgg": (lambda: I.rgg(6000, 8.0, 7), 100),
    "rbtree": (lambda: I.random_btree(3001, 4), 64),
    "ba": (lambda: I.ba(20000, 4, 3), 70),
    "btree": (lambda: I.complete_btree(9), 40),
}


def _gpu_graph(n, s, d):
    return ssm.ssm_build_graph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_kmeans_sp_bit_exact(name):
    make, k = GRAPHS[name]
    n, s, d = make()
    og = O.build_csr(n, s, d)
    piv = O.maxmin(og, k, 0)
    dip = O.pivot_dist(og, piv)
    want_p, want_a, want_it = O.kmeans_sp(dip, piv)
    got_p, got_a, got_it = ssm.ssm_kmeans_pivots(torch.from_numpy(dip).to(DEV), torch.from_numpy(piv).to(DEV))
    assert int(got_it.item()) == want_it
    assert np.array_equal(got_a.cpu().numpy(), want_a)
    assert np.array_equal(got_p.cpu().numpy(), want_p)


@pytest.mark.parametrize("max_iter", [1, 2, 3])
def test_kmeans_sp_pass_cap(max_iter):
    """The pass cap: the centres after the last allowed pass decide the pivots."""
    n, s, d = I.rgg(6000, 8.0, 9)
    og = O.build_csr(n, s, d)
    piv = O.maxmin(og, 80, 0)
    dip = O.pivot_dist(og, piv)
    want_p, want_a, want_it = O.kmeans_sp(dip, piv, max_iter)
    got_p, got_a, got_it = ssm.ssm_kmeans_pivots(torch.from_numpy(dip).to(DEV), torch.from_numpy(piv).to(DEV), max_iter)
    assert want_it == max_iter == int(got_it.item())
    assert np.array_equal(got_a.cpu().numpy(), want_a)
    assert np.array_equal(got_p.cpu().numpy(), want_p)


def test_kmeans_sp_many_clusters_and_ragged_tiles():
    """k above one 64-cluster chunk and one 64-pivot chunk, n not a multiple of
    the 64-node tile, on a mid-size RGG."""
    n, s, d = I.rgg(20011, 8.0, 13)
    og = O.build_csr(n, s, d)
    k = 150
    piv = O.maxmin(og, k, 0)
    dip = O.pivot_dist(og, piv)
    want_p, want_a, want_it = O.kmeans_sp(dip, piv)
    got_p, got_a, got_it = ssm.ssm_kmeans_pivots(torch.from_numpy(dip).to(DEV), torch.from_numpy(piv).to(DEV))
    assert int(got_it.item()) == want_it
    assert np.array_equal(got_a.cpu().numpy(), want_a)
    assert np.array_equal(got_p.cpu().numpy(), want_p)


def test_pipeline_with_kmeans_sampler():
    """Algorithm 1 with the paper's recommended sampler: pivots and d_ip of the
    k-means-sp pivots bit-exact, PivotMDS start within FP32 rounding."""
    n, s, d = I.rgg(6000, 8.0, 7)
    k = 60
    prep = O.prepare(n, s, d, k, sampler="kmeans")
    g, P, pos, eig = ssm.prepare(n, s, d, k, sampler="kmeans")
    assert np.array_equal(P.pivots.cpu().numpy(), prep.pivots)
    assert np.array_equal(P.dip.cpu().numpy(), prep.dip)
    assert np.array_equal(P.cnt.cpu().numpy(), prep.cnt)


def test_kmeans_sp_rejects_sizes_beyond_exact_arithmetic():
    """n * max(d) >= 2^32: the 32-bit centre sums could overflow, so the call
    reports SSM_E_ARG on the device and keeps the input pivots."""
    n, k = 70000, 2
    dip = torch.from_numpy(np.full((k, n), 65534, np.uint16)).to(DEV)
    piv = torch.tensor([0, 1], dtype=torch.int32, device=DEV)
    with pytest.raises(ssm.SSMError) as e:
        ssm.ssm_kmeans_pivots(dip, piv)
    assert e.value.code == -1
