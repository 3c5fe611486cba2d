"""Parity at full size on the Barabasi-Albert graph of 2^20 nodes (4 edges per
new node, seed 1), k = 200 max/min-sp pivots, in the launch configuration
bench.py times by default: the sweep runs in full-table mode (largest d_ip 8,
a 200 x 9 table of (w', w' d)) with whole 128-node tiles per warp, and the
sampled stress takes 1024 sources x 1024 targets through the pulled bitset BFS
in four passes of 256 sources.

The oracle computes every integer stage in full (max/min pivots, d_ip,
regions, counts), one Jacobi sweep from the GPU's PivotMDS start and the
stress sums over the identical pair list; the independent BFS runs and node
ranges are spread over host threads (results identical to the serial calls).
"""
import os

import numpy as np
import pytest

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def ba1m():
    n, s, d, k, iters = I.workload("ba1m", 1)
    og = O.build_csr(n, s, d)
    g, P, pos, eig = ssm.prepare(n, s, d, k, precision=32)
    piv = O.maxmin(og, k, 0)
    dip = O.pivot_dist_threads(og, piv, THREADS)
    return dict(n=n, k=k, og=og, g=g, P=P, pos=pos, piv=piv, dip=dip)


def test_ba1m_integer_stages_bit_exact(ba1m):
    og, g, P = ba1m["og"], ba1m["g"], ba1m["P"]
    assert g.m == og.m == 4194294
    assert np.array_equal(g.rowptr.cpu().numpy(), og.rowptr)
    assert np.array_equal(g.colidx.cpu().numpy(), og.colidx)
    assert np.array_equal(P.pivots.cpu().numpy(), ba1m["piv"])
    assert np.array_equal(P.dip.cpu().numpy(), ba1m["dip"])
    reg = O.regions(ba1m["dip"])
    ecc, off, cnt = O.histograms(ba1m["dip"], reg)
    assert np.array_equal(P.region.cpu().numpy(), reg)
    assert np.array_equal(P.cnt_off.cpu().numpy().astype(np.int64), off)
    assert np.array_equal(P.cnt.cpu().numpy(), cnt)


def test_ba1m_full_table_mode_applies(ba1m):
    """The configuration the bench times: k (max d + 1) weight pairs fit the
    full table (6112 pairs)."""
    dmax = int(ba1m["dip"].max())
    assert ba1m["k"] * (dmax + 1) <= 6112


def test_ba1m_one_sweep(ba1m):
    og, g, P, pos = ba1m["og"], ba1m["g"], ba1m["P"], ba1m["pos"]
    dip = ba1m["dip"]
    w = O.adapted_weights(dip, O.regions(dip))
    x0 = pos.cpu().numpy().astype(np.float64)
    want, orel = O.sweep_jacobi_threads(og, ba1m["piv"], dip, w, x0, THREADS)
    p = pos.clone()
    _, rel = ssm.ssm_iterate(g, P, p, 1)
    got = p.cpu().numpy().astype(np.float64)
    c = want - want.mean(0)
    err = np.sqrt(((got - want) ** 2).sum(1)).max() / np.sqrt((c ** 2).sum(1).mean())
    assert err < 1e-5
    assert rel.item() == pytest.approx(orel, rel=1e-4)


def test_ba1m_sampled_stress(ba1m):
    og, g, pos = ba1m["og"], ba1m["g"], ba1m["pos"]
    out, sums = ssm.ssm_stress(g, pos, 1024, 1024, 1)
    want, wsums = O.full_stress_threads(og, pos.cpu().numpy().astype(np.float64), 1024, 1024, 1, THREADS)
    np.testing.assert_allclose(sums.cpu().numpy(), wsums, rtol=1e-9)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-9)
