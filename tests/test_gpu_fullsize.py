"""Parity at full size, in the launch configuration bench.py times.

Workload: the random geometric graph with 262144 points (largest component
261828 nodes), k = 200 max/min-sp pivots, FP32 positions, stress on 1024 x
1024 sampled pairs.  The oracle computes every integer stage in full (about
8 s of CPU), one Jacobi sweep from the same state, and the stress on the
identical pair list.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgg():
    n, s, d, k, iters = I.workload("rgg256k", 1)
    og = O.build_csr(n, s, d)
    g, P, pos, eig = ssm.prepare(n, s, d, k, precision=32)
    return n, s, d, k, og, g, P, pos


def test_fullsize_integer_stages_bit_exact(rgg):
    n, s, d, k, og, g, P, pos = rgg
    assert g.m == og.m
    assert np.array_equal(g.colidx.cpu().numpy(), og.colidx)
    piv = O.maxmin(og, k, 0)
    assert np.array_equal(P.pivots.cpu().numpy(), piv)
    dip = O.pivot_dist(og, piv)
    assert np.array_equal(P.dip.cpu().numpy(), dip)
    reg = O.regions(dip)
    ecc, off, cnt = O.histograms(dip, reg)
    assert np.array_equal(P.region.cpu().numpy(), reg)
    assert np.array_equal(P.cnt.cpu().numpy(), cnt)


def test_fullsize_pivotmds_properties(rgg):
    """x = C v with orthogonal axes: ||x_c||^2 / ||y_c||^2 equals lambda_1/lambda_2
    and x_c . y_c = 0 (before the uniform rescale both hold exactly)."""
    n, s, d, k, og, g, P, pos = rgg
    p, eig = ssm.ssm_pivotmds(g, P.dip, precision=64, rescale=False)
    p = p.cpu().numpy()
    eig = eig.cpu().numpy()
    x = p[:, 0] - p[:, 0].mean()
    y = p[:, 1] - p[:, 1].mean()
    assert np.dot(x, x) == pytest.approx(eig[0], rel=1e-8)
    assert np.dot(y, y) == pytest.approx(eig[1], rel=1e-8)
    assert abs(np.dot(x, y)) <= 1e-8 * np.sqrt(eig[0] * eig[1])


def test_fullsize_one_sweep(rgg):
    n, s, d, k, og, g, P, pos = rgg
    x0 = pos.cpu().numpy().astype(np.float64)
    dip = P.dip.cpu().numpy()
    w = O.adapted_weights(dip, P.region.cpu().numpy())
    want, orel = O.sweep_jacobi(og, P.pivots.cpu().numpy(), dip, w, x0)
    p = pos.clone()
    _, rel = ssm.ssm_iterate(g, P, p, 1)
    got = p.cpu().numpy().astype(np.float64)
    c = want - want.mean(0)
    err = np.sqrt(((got - want) ** 2).sum(1)).max() / np.sqrt((c ** 2).sum(1).mean())
    assert err < 1e-5
    assert rel.item() == pytest.approx(orel, rel=1e-4)


def test_fullsize_sampled_stress(rgg):
    n, s, d, k, og, g, P, pos = rgg
    out, sums = ssm.ssm_stress(g, pos, 1024, 1024, 1)
    want, wsums = O.full_stress(og, pos.cpu().numpy().astype(np.float64), 1024, 1024, 1, return_sums=True)
    np.testing.assert_allclose(sums.cpu().numpy(), wsums, rtol=1e-9)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-9)


@pytest.mark.parametrize("family", ["ba", "grid"])
def test_one_sweep_many_tiles(family):
    """Graphs with more than two 128-node tiles per resident warp, where every
    warp takes whole tiles (full-table mode on the Barabasi-Albert graph,
    clamped mode on the 800 x 800 grid)."""
    if family == "ba":
        n, s, d = I.ba(700000, 4, 3)
    else:
        n, s, d = I.grid(800, 800)
    k = 32
    og = O.build_csr(n, s, d)
    g, P, pos, eig = ssm.prepare(n, s, d, k, precision=32)
    x0 = pos.cpu().numpy().astype(np.float64)
    dip = P.dip.cpu().numpy()
    w = O.adapted_weights(dip, P.region.cpu().numpy())
    want, orel = O.sweep_jacobi(og, P.pivots.cpu().numpy(), dip, w, x0)
    p = pos.clone()
    _, rel = ssm.ssm_iterate(g, P, p, 1)
    got = p.cpu().numpy().astype(np.float64)
    c = want - want.mean(0)
    err = np.sqrt(((got - want) ** 2).sum(1)).max() / np.sqrt((c ** 2).sum(1).mean())
    assert err < 1e-5
    assert rel.item() == pytest.approx(orel, rel=1e-4)
