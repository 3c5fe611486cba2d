"""Pins of the oracle's weighted-graph functions (Algorithm 1 line 2's
weighted MSSP, Section 3's weights on weighted graphs).

Each test checks them against something other than themselves: scipy's
Dijkstra (a library routine), brute force over all simple paths of tiny
graphs, the unweighted oracle functions (pinned on their own) for unit
lengths, the full-stress update of Section 3 on trees (k = n), exact scaling
by a power of two, and closed forms.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle as O
from paper_1608_08909_gb300 import inputs as I


def _wgraph(kind, seed):
    if kind == "rgg":
        n, s, d, l = I.rgg_lengths(500, 7.0, seed)
    elif kind == "grid_int":
        n, s, d = I.grid(12, 15)
        l = I.random_lengths(len(s), seed, "integer", hi=9)
    elif kind == "ba_uniform":
        n, s, d = I.ba(400, 3, seed)
        l = I.random_lengths(len(s), seed, "uniform", 0.25, 4.0)
    else:
        n, s, d = I.random_btree(300, seed)
        l = I.random_lengths(len(s), seed, "integer", hi=7)
    return n, s, d, l


def _scipy_dist(g):
    A = sp.csr_matrix((g.elen.astype(np.float64), g.colidx, g.rowptr), shape=(g.n, g.n))
    return csg.dijkstra(A, directed=True)


def test_build_wcsr_structure_and_shortest_duplicate():
    src = [0, 1, 1, 2, 2, 3, 0]
    dst = [1, 0, 2, 1, 2, 0, 1]
    ln = [3.0, 2.0, 1.5, 4.0, 9.0, 0.5, 7.0]
    g = O.build_wcsr(4, src, dst, ln)
    assert g.m == 3
    assert list(g.rowptr) == [0, 2, 4, 5, 6]
    assert list(g.colidx) == [1, 3, 0, 2, 1, 0]
    # (0,1) given as 3, 2 and 7: the shortest, 2, in both rows; the self-loop is dropped
    assert list(g.elen) == [2.0, 0.5, 2.0, 1.5, 1.5, 0.5]
    with pytest.raises(O.OracleError):
        O.build_wcsr(2, [0], [1], [0.0])
    with pytest.raises(O.OracleError):
        O.build_wcsr(2, [0], [1], [np.inf])


@pytest.mark.parametrize("kind", ["grid_int", "btree_int"])
def test_sssp_equals_scipy_dijkstra_on_integer_lengths(kind):
    """Integer lengths keep every path sum exact in float32 here, so the
    float32 search must equal scipy's FP64 Dijkstra exactly."""
    n, s, d, l = _wgraph(kind, 3)
    g = O.build_wcsr(n, s, d, l)
    D = _scipy_dist(g)
    for src in (0, n // 3, n - 1):
        assert np.array_equal(O.sssp(g, src).astype(np.float64), D[src])


@pytest.mark.parametrize("kind", ["rgg", "ba_uniform"])
def test_sssp_close_to_scipy_dijkstra_on_real_lengths(kind):
    n, s, d, l = _wgraph(kind, 5)
    g = O.build_wcsr(n, s, d, l)
    D = _scipy_dist(g)
    for src in (0, n - 1):
        np.testing.assert_allclose(O.sssp(g, src), D[src], rtol=2e-6 * 40, atol=0)


def test_sssp_is_the_least_float32_path_sum_brute_force():
    """Tiny graphs with lengths of mixed magnitudes, where float32 rounding
    matters: the distance equals the minimum over all simple paths of the sum
    rounded to float32 after each edge, walked from the source."""
    rng = np.random.default_rng(9)
    for trial in range(30):
        n = 7
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.5]
        edges += [(i, i + 1) for i in range(n - 1)]
        s = [e[0] for e in edges]
        d = [e[1] for e in edges]
        ln = (rng.uniform(0.1, 1.0, len(edges)) * 10.0 ** rng.integers(-3, 4, len(edges))).astype(np.float32)
        g = O.build_wcsr(n, s, d, ln)
        adj = {u: {} for u in range(n)}
        for u in range(n):
            for t in range(g.rowptr[u], g.rowptr[u + 1]):
                adj[u][int(g.colidx[t])] = np.float32(g.elen[t])
        src = int(rng.integers(0, n))
        best = np.full(n, np.inf, np.float32)
        best[src] = 0

        def walk(u, acc, seen):
            for v, lv in adj[u].items():
                if v in seen:
                    continue
                nv = np.float32(acc + lv)
                best[v] = min(best[v], nv)
                walk(v, nv, seen | {v})

        walk(src, np.float32(0), {src})
        assert np.array_equal(O.sssp(g, src), best), trial


@pytest.mark.parametrize("kind", ["grid", "rgg", "btree"])
def test_unit_lengths_reduce_to_the_unweighted_oracle(kind):
    """With every length 1 each weighted step is the unweighted one: pivots,
    distances, regions, s (0 for d <= 1), PivotMDS, rescale, the sweep and
    the stress, bit for bit."""
    n, s, d = {"grid": lambda: I.grid(14, 17), "rgg": lambda: I.rgg(600, 7.0, 2),
               "btree": lambda: I.complete_btree(7)}[kind]()
    k = 15
    g = O.build_csr(n, s, d)
    wg = O.build_wcsr(n, s, d, np.ones(len(s), np.float32))
    assert np.array_equal(wg.rowptr, g.rowptr) and np.array_equal(wg.colidx, g.colidx)
    piv = O.maxmin(g, k)
    assert np.array_equal(O.wmaxmin(wg, k), piv)
    dip = O.pivot_dist(g, piv)
    wdip = O.wpivot_dist(wg, piv)
    assert np.array_equal(wdip, dip.astype(np.float32))
    reg = O.regions(dip)
    assert np.array_equal(O.wregions(wdip), reg)
    w = O.adapted_weights(dip, reg)
    ws = O.wcounts(wg, piv, wdip, reg)
    d64 = dip.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        assert np.array_equal(np.where(dip >= 2, ws / (d64 * d64), 0.0), w)
    assert np.all(ws[dip <= 1] == 0)
    pos, eig = O.pivotmds(dip)
    wpos, weig = O.wpivotmds(wdip)
    assert np.array_equal(wpos, pos) and np.array_equal(weig, eig)
    pos = O.rescale(g, pos)
    assert np.array_equal(O.wrescale(wg, wpos), pos)
    x1, r1 = O.sweep_jacobi(g, piv, dip, w, pos)
    wx1, wr1 = O.wsweep_jacobi(wg, piv, wdip, ws, pos)
    assert np.array_equal(wx1, x1) and wr1 == r1
    assert np.array_equal(O.wfull_stress(wg, x1)[0], O.full_stress(g, x1))
    assert np.array_equal(O.wfull_stress(wg, x1, 16, 32, 5)[0], O.full_stress(g, x1, 16, 32, 5))


def test_scaling_lengths_by_two_scales_everything_exactly():
    """Lengths times 2 (exact in binary): distances double exactly, pivots,
    regions and s are unchanged, and rescaled layouts and sweeps double."""
    n, s, d, l = _wgraph("ba_uniform", 4)
    g1 = O.build_wcsr(n, s, d, l)
    g2 = O.build_wcsr(n, s, d, 2 * l)
    k = 12
    p1, p2 = O.wmaxmin(g1, k), O.wmaxmin(g2, k)
    assert np.array_equal(p1, p2)
    d1, d2 = O.wpivot_dist(g1, p1), O.wpivot_dist(g2, p2)
    assert np.array_equal(d2, 2 * d1)
    r1, r2 = O.wregions(d1), O.wregions(d2)
    assert np.array_equal(r1, r2)
    s1 = O.wcounts(g1, p1, d1, r1)
    assert np.array_equal(O.wcounts(g2, p2, d2, r2), s1)
    x1 = O.wrescale(g1, O.wpivotmds(d1)[0])
    x2 = O.wrescale(g2, O.wpivotmds(d2)[0])
    np.testing.assert_allclose(x2, 2 * x1, rtol=1e-12, atol=1e-12 * np.abs(x1).max())
    y1, _ = O.wsweep_jacobi(g1, p1, d1, s1, x1)
    y2, _ = O.wsweep_jacobi(g2, p2, d2, s1, 2 * x1)
    assert np.array_equal(y2, 2 * y1)


def test_every_node_a_pivot_on_a_tree_is_the_full_stress_update():
    """Section 3: with k = n the sparse model is full stress.  On a tree with
    integer lengths every edge is the only path between its ends, so
    l_ij = d_ij, every region is its pivot alone (s = 1) and the weighted
    sweep must equal the full-stress update over the weighted all-pairs
    distances (orc_full_sweep, summed in another order)."""
    n, s, d = I.random_btree(120, 8)
    l = I.random_lengths(len(s), 8, "integer", hi=5)
    g = O.build_wcsr(n, s, d, l)
    piv = np.arange(n, dtype=np.int32)
    dip = O.wpivot_dist(g, piv)
    reg = O.wregions(dip)
    assert np.array_equal(reg, piv)
    cnt = O.wcounts(g, piv, dip, reg)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(n, 2)) * 5
    y, _ = O.wsweep_jacobi(g, piv, dip, cnt, x)
    yf, _ = O.full_sweep(dip.astype(np.uint16), x, 0)
    np.testing.assert_allclose(y, yf, rtol=1e-12, atol=1e-12 * np.abs(yf).max())


def test_wcounts_small_hand_case():
    """Path 0-1-2-3-4 with lengths 1, 3, 1, 1 and pivots (0, 4): d to 0 is
    (0, 1, 4, 5, 6) and to 4 is (6, 5, 2, 1, 0); regions {0, 1} and {2, 3, 4}.
    s(i, a=0) counts j in {0, 1} with 2 d_j0 <= d_i0: node 2 (d 4): 2 (0 and
    2*1 <= 4); node 3 (5): 2; node 4 (6): 2; node 1 is adjacent, node 0 the
    pivot: 0.  s(i, a=1) over {2, 3, 4} (d 2, 1, 0): node 0 (6): 3; node 1
    (5): 3; node 2 (2): 2 (0 and 2*1 <= 2); node 3 adjacent, node 4 the
    pivot: 0."""
    g = O.build_wcsr(5, [0, 1, 2, 3], [1, 2, 3, 4], [1.0, 3.0, 1.0, 1.0])
    piv = np.array([0, 4], np.int32)
    dip = O.wpivot_dist(g, piv)
    assert list(dip[0]) == [0, 1, 4, 5, 6] and list(dip[1]) == [6, 5, 2, 1, 0]
    reg = O.wregions(dip)
    assert list(reg) == [0, 0, 1, 1, 1]
    cnt = O.wcounts(g, piv, dip, reg)
    assert list(cnt[0]) == [0, 0, 2, 2, 2]
    assert list(cnt[1]) == [3, 3, 2, 0, 0]


def test_weighted_path_pivotmds_is_exact_1d_and_stress_vanishes():
    """A path whose nodes sit at cumulative lengths is exactly 1-D
    Euclidean: PivotMDS recovers the positions up to sign and scale (second
    eigenvalue zero), and that layout has zero stress after optimal scaling."""
    n, s, d = I.path(50)
    l = I.random_lengths(len(s), 2, "integer", hi=6)
    g = O.build_wcsr(n, s, d, l)
    coord = np.concatenate([[0.0], np.cumsum(l.astype(np.float64))])
    dip = O.wpivot_dist(g, O.wmaxmin(g, 6))
    pos, eig = O.wpivotmds(dip)
    assert eig[1] <= 1e-9 * eig[0]
    c = coord - coord.mean()
    f = np.dot(pos[:, 0], c) / np.dot(c, c)
    np.testing.assert_allclose(pos[:, 0], f * c, atol=1e-9 * abs(f) * np.abs(c).max())
    x = np.stack([coord, np.zeros(n)], 1)
    out, _ = O.wfull_stress(g, x)
    assert out[0] < 1e-20 and out[2] < 1e-9


def test_wrescale_matches_total_edge_length():
    n, s, d, l = _wgraph("rgg", 6)
    g = O.build_wcsr(n, s, d, l)
    x = O.wrescale(g, np.random.default_rng(0).normal(size=(n, 2)))
    e = [(i, g.colidx[t], g.elen[t]) for i in range(n) for t in range(g.rowptr[i], g.rowptr[i + 1])
         if g.colidx[t] > i]
    tot = sum(np.hypot(*(x[i] - x[j])) for i, j, _ in e)
    assert tot == pytest.approx(sum(float(w) for _, _, w in e), rel=1e-12)


def test_wmaxmin_matches_definition_on_library_distances():
    n, s, d, l = _wgraph("rgg", 7)
    g = O.build_wcsr(n, s, d, l)
    piv = O.wmaxmin(g, 10)
    mind = np.full(n, np.inf)
    for a, p in enumerate(piv):
        if a > 0:
            m = mind.max()
            assert p == int(np.flatnonzero(mind == m)[0])
        mind = np.minimum(mind, O.sssp(g, int(p)))
    assert len(set(piv.tolist())) == 10


def test_weighted_sampled_stress_is_unbiased():
    n, s, d, l = _wgraph("grid_int", 2)
    g = O.build_wcsr(n, s, d, l)
    x = np.random.default_rng(4).normal(size=(n, 2)) * 10
    full, _ = O.wfull_stress(g, x)
    est = np.mean([O.wfull_stress(g, x, 64, 64, seed)[0][0] for seed in range(20)])
    assert est == pytest.approx(full[0], rel=0.05)
