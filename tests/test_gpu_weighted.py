"""Weighted graphs on the GPU against the oracle (Algorithm 1 line 2's
weighted MSSP, Section 3's weights with edge lengths): the CSR lengths,
distances, max/min pivots, regions and counts bit-exact (least float32 path
sums are unique, whatever the search order); PivotMDS to 1e-10 in the
eigenvalues; the FP64 sweep bit-identical, the FP32 sweep within 1e-5 per
step; stress to 1e-9."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _mixed_lengths(m, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.1, 1.0, m) * 10.0 ** rng.integers(-2, 3, m)).astype(np.float32)


WGRAPHS = {
    "rgg": lambda: I.rgg_lengths(3000, 7.0, 3),
    "rgg_large": lambda: I.rgg_lengths(40000, 8.0, 5),
    "grid_int": lambda: (lambda n, s, d: (n, s, d, I.random_lengths(len(s), 4, "integer", hi=9)))(*I.grid(40, 37)),
    "ba_uniform": lambda: (lambda n, s, d: (n, s, d, I.random_lengths(len(s), 5, "uniform", 0.25, 4.0)))(
        *I.ba(5000, 3, 5)),
    "path_mixed": lambda: (lambda n, s, d: (n, s, d, _mixed_lengths(len(s), 6)))(*I.path(3000)),
    "btree_mixed": lambda: (lambda n, s, d: (n, s, d, _mixed_lengths(len(s), 7)))(*I.random_btree(2000, 7)),
}
K = {"rgg": 40, "rgg_large": 100, "grid_int": 50, "ba_uniform": 64, "path_mixed": 9, "btree_mixed": 33}

_cache = {}


def _case(name):
    if name not in _cache:
        n, s, d, l = WGRAPHS[name]()
        og = O.build_wcsr(n, s, d, l)
        k = K[name]
        piv = O.wmaxmin(og, k)
        dip = O.wpivot_dist(og, piv)
        reg = O.wregions(dip)
        cnt = O.wcounts(og, piv, dip, reg, threads=8)
        _cache[name] = (n, s, d, l, og, piv, dip, reg, cnt)
    return _cache[name]


def _gpu_wgraph(n, s, d, l):
    return ssm.ssm_build_wgraph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV),
                                torch.from_numpy(np.ascontiguousarray(l, np.float32)).to(DEV))


def _norm_err(a, b):
    b = np.asarray(b, np.float64)
    a = np.asarray(a, np.float64)
    c = b - b.mean(0)
    rms = np.sqrt((c ** 2).sum(1).mean())
    return np.sqrt(((a - b) ** 2).sum(1)).max() / rms


@pytest.mark.parametrize("name", list(WGRAPHS))
def test_weighted_preprocessing_bit_exact(name):
    n, s, d, l, og, piv, dip, reg, cnt = _case(name)
    g = _gpu_wgraph(n, s, d, l)
    assert np.array_equal(g.rowptr.cpu().numpy(), og.rowptr)
    assert np.array_equal(g.colidx.cpu().numpy(), og.colidx)
    assert np.array_equal(g.elen.cpu().numpy(), og.elen)
    gp = ssm.ssm_select_pivots_weighted(g, len(piv))
    assert np.array_equal(gp.cpu().numpy(), piv)
    gd = ssm.ssm_pivot_sssp(g, gp)
    assert np.array_equal(gd.cpu().numpy(), dip)
    greg, gs = ssm.ssm_weighted_counts(g, gp, gd)
    assert np.array_equal(greg.cpu().numpy(), reg)
    assert np.array_equal(gs.cpu().numpy(), cnt)


def test_repeated_edges_keep_the_shortest_length():
    src = np.array([0, 1, 1, 2, 2, 3, 0, 3], np.int32)
    dst = np.array([1, 0, 2, 1, 2, 0, 1, 2], np.int32)
    ln = np.array([3.0, 2.0, 1.5, 4.0, 9.0, 0.5, 7.0, 1.0], np.float32)
    g = _gpu_wgraph(4, src, dst, ln)
    og = O.build_wcsr(4, src, dst, ln)
    assert np.array_equal(g.elen.cpu().numpy(), og.elen)


def test_bad_lengths_and_disconnected_graphs_are_errors():
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 2], np.int32)
    for bad in (0.0, -1.0, np.inf, np.nan):
        with pytest.raises(ssm.SSMError) as e:
            _gpu_wgraph(3, src, dst, np.array([1.0, bad], np.float32))
        assert e.value.code == -1
    with pytest.raises(ssm.SSMError) as e:  # node 3 isolated: the graph builder refuses it
        _gpu_wgraph(4, src, dst, np.array([1.0, 2.0], np.float32))
    assert e.value.code == -3
    # the searches detect it too, on a CSR made by hand
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=DEV)
    g = ssm.WGraph(4, 2, t([0, 1, 3, 4, 4], torch.int32), t([1, 0, 2, 1], torch.int32),
                   elen=t([1.0, 1.0, 2.0, 2.0], torch.float32))
    with pytest.raises(ssm.SSMError) as e:
        ssm.ssm_pivot_sssp(g, torch.tensor([0], dtype=torch.int32, device=DEV))
    assert e.value.code == -3
    with pytest.raises(ssm.SSMError) as e:
        ssm.ssm_select_pivots_weighted(g, 2)
    assert e.value.code == -3


def test_unit_lengths_match_the_unweighted_gpu_path():
    n, s, d = I.rgg(6000, 7.0, 9)
    g = _gpu_wgraph(n, s, d, np.ones(len(s), np.float32))
    ug = ssm.ssm_build_graph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV))
    k = 50
    piv = ssm.ssm_select_pivots_weighted(g, k)
    assert torch.equal(piv, ssm.ssm_select_pivots(ug, k))
    dist = ssm.ssm_pivot_sssp(g, piv)
    dip = ssm.ssm_pivot_bfs(ug, piv)
    assert torch.equal(dist, dip.to(torch.int32).to(torch.float32))


@pytest.mark.parametrize("name", ["rgg", "grid_int", "ba_uniform", "path_mixed"])
def test_weighted_pivotmds_matches_oracle(name):
    n, s, d, l, og, piv, dip, reg, cnt = _case(name)
    opos, oeig = O.wpivotmds(dip)
    g = _gpu_wgraph(n, s, d, l)
    gd = torch.from_numpy(dip).to(DEV)
    for prec in (32, 64):
        pos, eig = ssm.ssm_pivotmds_weighted(g, gd, precision=prec, rescale=False)
        eig = eig.cpu().numpy()
        np.testing.assert_allclose(eig[0], oeig[0], rtol=1e-10)
        if oeig[1] > 1e-9 * oeig[0]:
            np.testing.assert_allclose(eig[1], oeig[1], rtol=1e-10)
        tol = 2e-6 if prec == 32 else 1e-9
        if oeig[1] > 1e-6 * oeig[0]:
            assert _norm_err(pos.cpu().numpy(), opos) < tol
        else:
            assert _norm_err(pos.cpu().numpy()[:, :1], opos[:, :1]) < tol
    pos, _ = ssm.ssm_pivotmds_weighted(g, gd, precision=64, rescale=True)
    if oeig[1] > 1e-6 * oeig[0]:
        assert _norm_err(pos.cpu().numpy(), O.wrescale(og, opos)) < 1e-9


@pytest.mark.parametrize("name", ["rgg", "grid_int", "ba_uniform", "btree_mixed"])
def test_weighted_sweep_fp64_bit_identical(name):
    n, s, d, l, og, piv, dip, reg, cnt = _case(name)
    x0 = O.wrescale(og, O.wpivotmds(dip)[0])
    g = _gpu_wgraph(n, s, d, l)
    pos = torch.from_numpy(x0.copy()).to(DEV)
    rel = ssm.ssm_iterate_weighted(g, torch.from_numpy(piv).to(DEV), torch.from_numpy(dip).to(DEV),
                                   torch.from_numpy(cnt).to(DEV), pos, 5)
    x, r = x0, 0.0
    for _ in range(5):
        x, r = O.wsweep_jacobi(og, piv, dip, cnt, x, threads=8)
    assert np.array_equal(pos.cpu().numpy(), x)
    assert rel.item() == pytest.approx(r, rel=1e-12)


@pytest.mark.parametrize("name", list(WGRAPHS))
def test_weighted_sweep_fp32_single_steps(name):
    n, s, d, l, og, piv, dip, reg, cnt = _case(name)
    x = O.wrescale(og, O.wpivotmds(dip)[0])
    g = _gpu_wgraph(n, s, d, l)
    gp, gd, gs = (torch.from_numpy(a).to(DEV) for a in (piv, dip, cnt))
    for step in range(3):
        x32 = x.astype(np.float32)
        pos = torch.from_numpy(x32.copy()).to(DEV)
        rel = ssm.ssm_iterate_weighted(g, gp, gd, gs, pos, 1)
        ox, orel = O.wsweep_jacobi(og, piv, dip, cnt, x32.astype(np.float64), threads=8)
        assert _norm_err(pos.cpu().numpy(), ox) < 1e-5, step
        # the FP32 output's own rounding (about 6e-8 of |x|) bounds how well a
        # small relative change can be resolved
        assert abs(rel.item() - orel) <= 1e-3 * orel + 2e-7
        x = ox


def test_weighted_sweep_coincident_positions():
    """r = 0 (coincident nodes): the term contributes w * x_j only, on both sides."""
    n, s, d, l, og, piv, dip, reg, cnt = _case("grid_int")
    x = O.wrescale(og, O.wpivotmds(dip)[0])
    x[5] = x[6]
    x[100] = x[piv[3]]
    g = _gpu_wgraph(n, s, d, l)
    pos = torch.from_numpy(x.copy()).to(DEV)
    ssm.ssm_iterate_weighted(g, torch.from_numpy(piv).to(DEV), torch.from_numpy(dip).to(DEV),
                             torch.from_numpy(cnt).to(DEV), pos, 1)
    ox, _ = O.wsweep_jacobi(og, piv, dip, cnt, x)
    assert np.array_equal(pos.cpu().numpy(), ox)


@pytest.mark.parametrize("name", ["rgg", "ba_uniform", "grid_int"])
def test_weighted_stress_matches_oracle(name):
    n, s, d, l, og, piv, dip, reg, cnt = _case(name)
    x = O.wrescale(og, O.wpivotmds(dip)[0])
    g = _gpu_wgraph(n, s, d, l)
    for prec in (64, 32):
        xx = x if prec == 64 else x.astype(np.float32)
        pos = torch.from_numpy(np.ascontiguousarray(xx)).to(DEV)
        for S, T in ((0, 0), (64, 128)):
            out, sums = ssm.ssm_stress_weighted(g, pos, S, T, 11)
            oout, osums = O.wfull_stress(og, xx.astype(np.float64), S, T, 11)
            np.testing.assert_allclose(sums.cpu().numpy(), osums, rtol=1e-9)
            np.testing.assert_allclose(out.cpu().numpy(), oout, rtol=1e-9)


def test_layout_weighted_end_to_end_lowers_stress():
    n, s, d, l = I.rgg_lengths(20000, 8.0, 12)
    g, piv, dist, region, s_tab, pos, eig = ssm.layout_weighted(n, s, d, l, 64, 0)
    before, _ = ssm.ssm_stress_weighted(g, pos, 256, 256, 3)
    ssm.ssm_iterate_weighted(g, piv, dist, s_tab, pos, 60)
    after, _ = ssm.ssm_stress_weighted(g, pos, 256, 256, 3)
    assert torch.isfinite(pos).all()
    assert after[3].item() < before[3].item()
