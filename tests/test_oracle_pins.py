"""Pins of the CPU oracle to what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (scipy shortest paths, numpy eigh), a closed form, an exact special
case, a hand derivation stored under tests/golden/, or an invariant the paper
states.  A plausible slip in the oracle (a dropped term, a wrong index or
sign, a transposed operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
from scipy.optimize import minimize_scalar

import oracle as O
from paper_1608_08909_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _apsp(g):
    A = sp.csr_matrix((np.ones(len(g.colidx)), g.colidx, g.rowptr), shape=(g.n, g.n))
    D = csg.shortest_path(A, method="D", unweighted=True)
    return D


def _rand_graph(rng, n, p):
    # connected: random spanning tree plus random extra edges
    src, dst = [], []
    for v in range(1, n):
        src.append(int(rng.integers(0, v)))
        dst.append(v)
    extra = rng.random((n, n)) < p
    for i, j in zip(*np.nonzero(np.triu(extra, 1))):
        src.append(int(i))
        dst.append(int(j))
    return n, np.array(src, np.int32), np.array(dst, np.int32)


# ---------------------------------------------------------------- graph / BFS

def test_build_csr_matches_scipy_structure():
    rng = np.random.default_rng(3)
    n = 37
    src = rng.integers(0, n, 300).astype(np.int32)
    dst = rng.integers(0, n, 300).astype(np.int32)
    g = O.build_csr(n, src, dst)
    keep = src != dst
    A = sp.coo_matrix((np.ones(keep.sum()), (src[keep], dst[keep])), shape=(n, n)).tocsr()
    A = ((A + A.T) > 0).astype(np.int8).tocsr()
    A.sort_indices()
    assert np.array_equal(g.rowptr, A.indptr)
    assert np.array_equal(g.colidx, A.indices)
    assert g.m == A.nnz // 2


def test_build_csr_rejects_out_of_range():
    with pytest.raises(O.OracleError) as e:
        O.build_csr(3, [0, 1], [1, 3])
    assert e.value.code == -2


@pytest.mark.parametrize("seed", range(6))
def test_bfs_matches_library_apsp(seed):
    rng = np.random.default_rng(seed)
    n, s, d = _rand_graph(rng, int(rng.integers(2, 40)), 0.08)
    g = O.build_csr(n, s, d)
    D = _apsp(g)
    for v in range(n):
        assert np.array_equal(O.bfs(g, v), D[v].astype(np.int32))


def test_bfs_closed_forms():
    n, s, d = I.grid(7, 9)
    g = O.build_csr(n, s, d)
    for v in (0, 13, 62):
        r, c = divmod(np.arange(n), 9)
        rv, cv = divmod(v, 9)
        assert np.array_equal(O.bfs(g, v), np.abs(r - rv) + np.abs(c - cv))
    n, s, d = I.path(50)
    g = O.build_csr(n, s, d)
    assert np.array_equal(O.bfs(g, 17), np.abs(np.arange(50) - 17))
    n, s, d = I.complete_btree(6)
    g = O.build_csr(n, s, d)

    def depth(i):
        return int(math.floor(math.log2(i + 1)))

    def lca_dist(i, j):
        di, dj = depth(i), depth(j)
        a, b = i, j
        while a != b:
            if a > b:
                a = (a - 1) // 2
            else:
                b = (b - 1) // 2
        return di + dj - 2 * depth(a)

    for v in (0, 5, 100):
        assert np.array_equal(O.bfs(g, v), [lca_dist(v, j) for j in range(n)])


# ---------------------------------------------------------------- pivots

def test_maxmin_grid_golden():
    want = [int(x) for x in open(os.path.join(GOLD, "grid32_maxmin.txt")) if x.strip() and x[0] != "#"]
    n, s, d = I.grid(32, 32)
    g = O.build_csr(n, s, d)
    assert O.maxmin(g, 5).tolist() == want


@pytest.mark.parametrize("seed", range(5))
def test_maxmin_matches_definition_on_library_apsp(seed):
    rng = np.random.default_rng(100 + seed)
    n, s, d = _rand_graph(rng, int(rng.integers(5, 60)), 0.05)
    g = O.build_csr(n, s, d)
    D = _apsp(g)
    k = int(rng.integers(1, n + 1))
    start = int(rng.integers(0, n))
    P = [start]
    while len(P) < k:
        mind = D[P].min(axis=0)
        P.append(int(np.argmax(mind)))  # first maximum = lowest node id
    assert O.maxmin(g, k, start).tolist() == P


def test_maxmin_rejects_disconnected():
    with pytest.raises(O.OracleError) as e:
        g = O.build_csr(4, [0, 2], [1, 3])
        O.maxmin(g, 2)
    assert e.value.code == -3


@pytest.mark.parametrize("seed", range(4))
def test_pivot_dist_regions_histograms(seed):
    rng = np.random.default_rng(200 + seed)
    n, s, d = _rand_graph(rng, int(rng.integers(10, 80)), 0.04)
    g = O.build_csr(n, s, d)
    D = _apsp(g)
    k = int(rng.integers(1, min(n, 12) + 1))
    piv = rng.choice(n, k, replace=False).astype(np.int32)
    dip = O.pivot_dist(g, piv)
    assert np.array_equal(dip, D[piv].astype(np.uint16))
    reg = O.regions(dip)
    assert np.array_equal(reg, np.argmin(D[piv], axis=0))  # first minimum = lowest pivot index
    # R is a partition with p in R(p) (Section 3)
    assert np.array_equal(reg[piv], np.arange(k))
    ecc, off, cnt = O.histograms(dip, reg)
    for a in range(k):
        members = np.nonzero(reg == a)[0]
        dm = dip[a, members].astype(int)
        assert ecc[a] == dm.max()
        row = cnt[off[a]:off[a + 1]]
        assert len(row) == ecc[a] + 1
        assert np.array_equal(row, [(dm <= t).sum() for t in range(ecc[a] + 1)])
    assert sum(cnt[off[a + 1] - 1] for a in range(k)) == n


# ---------------------------------------------------------------- adapted weights

def test_adapted_weights_path_golden():
    n, s, d = I.path(7)
    g = O.build_csr(n, s, d)
    dip = O.pivot_dist(g, [0, 6])
    reg = O.regions(dip)
    assert reg.tolist() == [0, 0, 0, 0, 1, 1, 1]
    w = O.adapted_weights(dip, reg)
    for line in open(os.path.join(GOLD, "path7_weights.txt")):
        if not line.strip() or line[0] == "#":
            continue
        f = line.split()
        a, i = int(f[0]), int(f[1])
        want = 0.0 if f[2] == "skip" else int(f[2]) / int(f[3])
        assert w[a, i] == pytest.approx(want, rel=0, abs=0), (a, i)
    # asymmetry (Section 3): w'(0 -> 6) != w'(6 -> 0)
    assert w[1, 0] != w[0, 6]


@pytest.mark.parametrize("seed", range(4))
def test_adapted_weights_match_histogram_route(seed):
    """Direct count (sorted region lists) against the cumulative counts."""
    rng = np.random.default_rng(300 + seed)
    n, s, d = _rand_graph(rng, int(rng.integers(20, 120)), 0.02)
    g = O.build_csr(n, s, d)
    k = int(rng.integers(2, 16))
    piv = O.maxmin(g, k, int(rng.integers(0, n)))
    dip = O.pivot_dist(g, piv)
    reg = O.regions(dip)
    ecc, off, cnt = O.histograms(dip, reg)
    w = O.adapted_weights(dip, reg)
    for a in range(k):
        for i in range(n):
            dd = int(dip[a, i])
            if dd < 2:
                assert w[a, i] == 0.0
                continue
            s_ = int(cnt[off[a] + min(dd // 2, ecc[a])])
            assert s_ >= 1
            assert w[a, i] == s_ / (dd * dd)


def test_weights_reduce_to_full_stress_when_k_equals_n():
    """k = n: every node is its own region, s = 1, w' = 1/d^2 (Section 3)."""
    n, s, d = I.grid(5, 6)
    g = O.build_csr(n, s, d)
    piv = np.arange(n, dtype=np.int32)
    dip = O.pivot_dist(g, piv)
    w = O.adapted_weights(dip, O.regions(dip))
    D = _apsp(g)
    want = np.where(D >= 2, 1.0 / np.maximum(D, 1) ** 2, 0.0)
    assert np.array_equal(w, want)


# ---------------------------------------------------------------- sweep

def _full_stress_jacobi_update(D, X):
    """GKN localized update (Section 3, the full-stress update before Eq. 4), all i from X."""
    n = len(X)
    out = np.zeros_like(X)
    for i in range(n):
        num = np.zeros(2)
        den = 0.0
        for j in range(n):
            if j == i:
                continue
            w = 1.0 / D[i, j] ** 2
            diff = X[i] - X[j]
            r = np.hypot(*diff)
            num += w * (X[j] + D[i, j] * diff / r)
            den += w
        out[i] = num / den
    return out


def test_sweep_k_equals_n_is_full_stress_update():
    n, s, d = I.grid(4, 5)
    g = O.build_csr(n, s, d)
    D = _apsp(g)
    piv = np.arange(n, dtype=np.int32)
    dip = O.pivot_dist(g, piv)
    w = O.adapted_weights(dip, O.regions(dip))
    X = np.random.default_rng(0).normal(size=(n, 2))
    got, _ = O.sweep_jacobi(g, piv, dip, w, X)
    np.testing.assert_allclose(got, _full_stress_jacobi_update(D, X), rtol=1e-13, atol=1e-13)


def _stress_eq1(D, X):
    n = len(X)
    iu = np.triu_indices(n, 1)
    r = np.hypot(*(X[iu[0]] - X[iu[1]]).T)
    dd = D[iu]
    return np.sum((r - dd) ** 2 / dd ** 2)


def test_gauss_seidel_full_stress_is_monotone():
    """Node-at-a-time majorization of full stress never increases it (Section 3, [gkn-sm-04])."""
    n, s, d = I.random_btree(40, 5)
    g = O.build_csr(n, s, d)
    D = _apsp(g)
    piv = np.arange(n, dtype=np.int32)
    dip = O.pivot_dist(g, piv)
    w = O.adapted_weights(dip, O.regions(dip))
    X = np.random.default_rng(1).normal(size=(n, 2)) * 3
    prev = _stress_eq1(D, X)
    for _ in range(30):
        X = O.sweep_gs(g, piv, dip, w, X)
        cur = _stress_eq1(D, X)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_sweep_equivariance():
    """Eq. 4 commutes with rotations, reflections and translations of the layout."""
    n, s, d = I.rgg(300, 7.0, 11)
    p = O.prepare(n, s, d, 12)
    X = p.pos0
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]]) @ np.diag([1, -1])
    t = np.array([3.5, -1.25])
    a, _ = O.sweep_jacobi(p.g, p.pivots, p.dip, p.w, X)
    b, _ = O.sweep_jacobi(p.g, p.pivots, p.dip, p.w, X @ R.T + t)
    np.testing.assert_allclose(b, a @ R.T + t, rtol=0, atol=1e-10 * np.abs(a).max())


def test_two_node_jacobi_oscillation():
    """Two nodes at distance r (edge, d=1): Eq. 4 moves each to x_j + (x_i - x_j)/r,
    so from r = 0.4 Jacobi maps the distance to 1 exactly (both move)."""
    g = O.build_csr(2, [0], [1])
    X = np.array([[0.0, 0.0], [0.4, 0.0]])
    piv = np.array([0], np.int32)
    dip = O.pivot_dist(g, piv)
    w = O.adapted_weights(dip, O.regions(dip))
    Y, rel = O.sweep_jacobi(g, piv, dip, w, X)
    # node 0 -> x1 + (x0-x1)/0.4 = 0.4 - 1 = -0.6 ; node 1 -> x0 + (x1-x0)/0.4 = 1.0
    np.testing.assert_allclose(Y, [[-0.6, 0.0], [1.0, 0.0]], rtol=0, atol=1e-15)
    assert rel == pytest.approx(math.hypot(0.6, 0.6) / 0.4)


def test_coincident_nodes_rule():
    """r = 0: the term contributes w * x_j only."""
    g = O.build_csr(2, [0], [1])
    X = np.array([[1.0, 2.0], [1.0, 2.0]])
    piv = np.array([0], np.int32)
    dip = O.pivot_dist(g, piv)
    w = O.adapted_weights(dip, O.regions(dip))
    Y, _ = O.sweep_jacobi(g, piv, dip, w, X)
    np.testing.assert_array_equal(Y, X)


# ---------------------------------------------------------------- PivotMDS

def test_pivotmds_eigs_match_library():
    n, s, d = I.rgg(400, 8.0, 3)
    g = O.build_csr(n, s, d)
    piv = O.maxmin(g, 20)
    dip = O.pivot_dist(g, piv)
    pos, eig, B = O.pivotmds(dip, return_b=True)
    # B = C^T C with C the double-centred -1/2 d^2 (numpy route)
    Dl = dip.T.astype(np.float64) ** 2
    C = -0.5 * (Dl - Dl.mean(1, keepdims=True) - Dl.mean(0, keepdims=True) + Dl.mean())
    np.testing.assert_allclose(B, C.T @ C, rtol=1e-12, atol=1e-9 * np.abs(B).max())
    lam, V = np.linalg.eigh(C.T @ C)
    np.testing.assert_allclose(eig, lam[::-1][:2], rtol=1e-10)
    for r in range(2):
        v = V[:, -1 - r]
        v = v * np.sign(v[np.argmax(np.abs(v))])
        np.testing.assert_allclose(pos[:, r], C @ v, rtol=1e-8, atol=1e-8 * np.abs(pos).max())


def test_gram_brute_force_integers():
    """The exact Gram matrix against Python-integer loops, on values that fill
    all 32 bits of d^2 (where float64 sums of the full products would round)."""
    dip = I.distance_table(4, 11, 65534, 7)
    G = O.gram(dip)
    for a in range(4):
        for b in range(4):
            assert G[a, b] == sum(int(dip[a, i]) ** 2 * int(dip[b, i]) ** 2 for i in range(11))
    assert G[0, 0] > 2 ** 64  # the 128-bit range is reached


def test_gram_centres_to_pivotmds_b():
    """Double centring commutes with the contraction: C^T C = 1/4 J (G - s s^T / n) J
    with s_a = sum_i d_ia^2 and J the k x k centring matrix, against the B
    that the oracle's PivotMDS forms from the centred C."""
    n, s, d = I.rgg(400, 8.0, 3)
    g = O.build_csr(n, s, d)
    dip = O.pivot_dist(g, O.maxmin(g, 20))
    _, _, B = O.pivotmds(dip, return_b=True)
    G = O.gram(dip).astype(np.float64)
    sa = (dip.astype(np.float64) ** 2).sum(1)
    k = dip.shape[0]
    J = np.eye(k) - 1.0 / k
    np.testing.assert_allclose(0.25 * J @ (G - np.outer(sa, sa) / n) @ J, B, rtol=1e-9, atol=1e-9 * np.abs(B).max())


def test_pivotmds_path_is_exact_1d():
    """On a path d_ij = |i-j| is Euclidean in 1-D, so classical MDS is exact:
    x_i is proportional to i - mean(i) and the second eigenvalue vanishes."""
    n, s, d = I.path(60)
    g = O.build_csr(n, s, d)
    dip = O.pivot_dist(g, O.maxmin(g, 7))
    pos, eig = O.pivotmds(dip)
    assert eig[1] <= 1e-9 * eig[0]
    i = np.arange(n) - (n - 1) / 2
    c = np.dot(pos[:, 0], i) / np.dot(i, i)
    np.testing.assert_allclose(pos[:, 0], c * i, rtol=0, atol=1e-9 * abs(c) * n)
    assert np.abs(pos[:, 1]).max() <= 1e-6 * np.abs(pos[:, 0]).max()


def test_rescale_sets_mean_edge_length_one():
    n, s, d = I.grid(9, 11)
    p = O.prepare(n, s, d, 8)
    X = p.pos0
    e = [(i, j) for i in range(n) for j in p.g.colidx[p.g.rowptr[i]:p.g.rowptr[i + 1]] if j > i]
    tot = sum(np.hypot(*(X[i] - X[j])) for i, j in e)
    assert tot == pytest.approx(p.g.m, rel=1e-12)


# ---------------------------------------------------------------- stress

def test_stress_unit_square_closed_form():
    """4-cycle on the unit square: edges r=d=1, diagonals r=sqrt2, d=2."""
    g = O.build_csr(4, [0, 1, 2, 3], [1, 2, 3, 0])
    X = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64)
    out = O.full_stress(g, X)
    r2 = math.sqrt(2.0)
    assert out[0] == pytest.approx(3 - 2 * r2, rel=1e-14)
    assert out[1] == pytest.approx((4 + r2) / 5, rel=1e-14)
    assert out[2] == pytest.approx((12 - 8 * r2) / 5, rel=1e-13)
    assert out[3] == pytest.approx((12 - 8 * r2) / 5 / 6, rel=1e-13)


def test_stress_zero_for_exact_path_layout():
    n, s, d = I.path(25)
    g = O.build_csr(n, s, d)
    X = np.stack([np.arange(n) * 2.0, np.zeros(n)], 1)  # twice the right scale
    out = O.full_stress(g, X)
    assert out[0] > 0
    assert out[1] == pytest.approx(0.5, rel=1e-14)
    assert abs(out[2]) < 1e-9


def test_optimal_scale_against_numerical_minimum():
    n, s, d = I.random_btree(30, 2)
    g = O.build_csr(n, s, d)
    D = _apsp(g)
    X = np.random.default_rng(4).normal(size=(n, 2))
    out = O.full_stress(g, X)
    f = lambda a: _stress_eq1(D, a * X)  # noqa: E731
    res = minimize_scalar(f, bracket=(0.1, 10.0), tol=1e-12)
    assert out[1] == pytest.approx(res.x, rel=1e-6)
    assert out[2] == pytest.approx(res.fun, rel=1e-9)
    assert out[0] == pytest.approx(f(1.0), rel=1e-12)


def test_splitmix64_reference_values():
    want = [int(x, 16) for x in open(os.path.join(GOLD, "splitmix64_seed0.txt")) if x.startswith("0x")]
    assert O.splitmix64(0, 3).tolist() == want


def test_sample_pairs_valid_and_uniform():
    n, S, T = 50, 64, 512
    srcs, tgts = O.sample_pairs(n, S, T, 9)
    assert srcs.min() >= 0 and srcs.max() < n
    assert tgts.min() >= 0 and tgts.max() < n
    assert not np.any(tgts == srcs[:, None])
    counts = np.bincount(tgts.ravel(), minlength=n)
    exp = S * T / n
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 2 * n  # loose: mean n-1, sd ~ sqrt(2n)


def test_sampled_stress_unbiased():
    """The sampled estimator averages to the exhaustive stress."""
    n, s, d = I.rgg(120, 7.0, 5)
    p = O.prepare(n, s, d, 10)
    ex = O.full_stress(p.g, p.pos0)
    est = np.mean([O.full_stress(p.g, p.pos0, 16, 64, seed)[0] for seed in range(60)])
    assert est == pytest.approx(ex[0], rel=0.03)


def test_sample_pairs_first_pairs_hand_derived():
    """The index mapping of the sampled pair list (source, then targets with the
    skip over the source) against pairs derived by hand from the published
    splitmix64 outputs (tests/golden/sample_pairs_seed0.txt); the second case
    starts the stream so that the first source is node 0 and every target
    takes the skip."""
    rows = [ln.split() for ln in open(os.path.join(GOLD, "sample_pairs_seed0.txt")) if ln.startswith("0x")]
    assert len(rows) == 2
    for r in rows:
        seed, n, S, T = int(r[0], 16), int(r[1]), int(r[2]), int(r[3])
        srcs, tgts = O.sample_pairs(n, S, T, seed)
        assert srcs.tolist() == [int(r[4])]
        assert tgts.reshape(-1).tolist() == [int(x) for x in r[5:]]


def test_gauss_seidel_uses_updated_positions():
    """One in-place sweep on the path 0-1-2 with the single pivot 0, from
    x = (0,0), (3,0), (3,4), derived by hand from Eq. 4:
      node 0: neighbour 1 at r = 3 -> (3,0) + (-3,0)/3 = (2,0);
      node 1: neighbours 0 (already moved to (2,0), r = 1) and 2 (r = 4):
              (2,0) + (1,0)/1 = (3,0) and (3,4) + (0,-4)/4 = (3,3) -> (3, 1.5)
              (the Jacobi order, which reads the old (0,0), gives (2, 1.5));
      node 2: neighbour 1 at (3,1.5), r = 2.5 -> (3,1.5) + (0,2.5)/2.5 = (3,2.5);
              pivot 0 at (2,0), d = 2, R(0) = {0,1,2}, s = |{j: d_j0 <= 1}| = 2,
              w' = 2/4 = 1/2, r = sqrt(17): w'((2,0) + 2 (1,4)/sqrt(17));
              x_2 = [(3,2.5) + w'(...)] / (1 + 1/2)."""
    n, s, d = 3, np.array([0, 1], np.int32), np.array([1, 2], np.int32)
    g = O.build_csr(n, s, d)
    piv = np.array([0], np.int32)
    dip = O.pivot_dist(g, piv)
    w = O.adapted_weights(dip, O.regions(dip))
    x = np.array([[0.0, 0.0], [3.0, 0.0], [3.0, 4.0]])
    r17 = math.sqrt(17.0)
    want = np.array([[2.0, 0.0], [3.0, 1.5],
                     [(3.0 + 0.5 * (2.0 + 2.0 / r17)) / 1.5, (2.5 + 0.5 * (8.0 / r17)) / 1.5]])
    got = O.sweep_gs(g, piv, dip, w, x)
    np.testing.assert_allclose(got, want, rtol=1e-15, atol=1e-15)
    jac, _ = O.sweep_jacobi(g, piv, dip, w, x)
    np.testing.assert_allclose(jac[1], [2.0, 1.5], rtol=1e-15)


def test_node_range_and_source_range_pieces_add_up():
    """The range forms used to spread the oracle over host threads: node ranges
    of the Jacobi sweep reproduce the whole sweep exactly, source ranges of the
    stress sums add up to the whole list's sums, and pivot subsets give the
    same d_ip rows."""
    n, s, d = I.rgg(2500, 8.0, 4)
    p = O.prepare(n, s, d, 24)
    a, ra = O.sweep_jacobi(p.g, p.pivots, p.dip, p.w, p.pos0)
    b, rb = O.sweep_jacobi_threads(p.g, p.pivots, p.dip, p.w, p.pos0, 3)
    assert np.array_equal(a, b) and ra == rb
    out, sums = O.full_stress(p.g, p.pos0, 40, 33, 5, return_sums=True)
    out2, sums2 = O.full_stress_threads(p.g, p.pos0, 40, 33, 5, 4)
    np.testing.assert_allclose(sums2, sums, rtol=1e-13)
    np.testing.assert_allclose(out2, out, rtol=1e-12)
    ex, exs = O.full_stress(p.g, p.pos0, return_sums=True)
    ex2, exs2 = O.full_stress_threads(p.g, p.pos0, 0, 0, 0, 3)
    np.testing.assert_allclose(exs2, exs, rtol=1e-13)
    assert np.array_equal(O.pivot_dist_threads(p.g, p.pivots, 5), p.dip)


# ---------------------------------------------------------------- k-means sp (Section 4.1)

def test_kmeans_sp_hand_derived_path():
    """Path 0..6, max/min-sp pivots (0, 6): y_i = (i, 6 - i).  First pass: the
    squared distances to y_0 and y_6 are 2 i^2 and 2 (6 - i)^2, node 3 ties and
    joins cluster 0, so the clusters are {0,1,2,3} and {4,5,6} with means
    (1.5, 4.5) and (5, 1).  Second pass: node 3 is at 4.5 from the first mean
    and 8 from the second, node 4 at 6.5 and 2: nothing changes, stop after 2
    passes.  New pivots: nodes 1 and 2 are both at 0.5 from (1.5, 4.5) -> the
    lower id, 1; node 5 is the second mean itself -> 5."""
    n, s, d = I.path(7)
    g = O.build_csr(n, s, d)
    piv = O.maxmin(g, 2)
    assert piv.tolist() == [0, 6]
    newp, asg, it = O.kmeans_sp(O.pivot_dist(g, piv), piv)
    assert newp.tolist() == [1, 5]
    assert asg.tolist() == [0, 0, 0, 0, 1, 1, 1]
    assert it == 2


@pytest.mark.parametrize("name", ["rgg", "grid", "rbtree"])
def test_kmeans_sp_matches_library_lloyd(name):
    """scikit-learn's Lloyd iterations from the same initial centres (the
    max/min pivots' distance vectors) reach the same clusters in the same
    number of passes on graphs without exact ties."""
    KMeans = pytest.importorskip("sklearn.cluster").KMeans
    n, s, d = {"rgg": lambda: I.rgg(400, 8.0, 3), "grid": lambda: I.grid(13, 17),
               "rbtree": lambda: I.random_btree(300, 5)}[name]()
    k = {"rgg": 12, "grid": 10, "rbtree": 9}[name]
    g = O.build_csr(n, s, d)
    piv = O.maxmin(g, k)
    dip = O.pivot_dist(g, piv)
    _, asg, it = O.kmeans_sp(dip, piv)
    Y = dip.T.astype(np.float64)
    km = KMeans(n_clusters=k, init=Y[piv], n_init=1, max_iter=50, tol=0.0, algorithm="lloyd").fit(Y)
    assert np.array_equal(km.labels_, asg)
    assert km.n_iter_ == it


@pytest.mark.parametrize("seed", [2, 7])
def test_kmeans_sp_is_an_exact_fixed_point(seed):
    """In exact rational arithmetic: every node sits at a nearest centre of
    the final clustering, every centre is its members' mean, and every new
    pivot is the member nearest its centre with ties to the lowest id."""
    from fractions import Fraction

    n, s, d = I.ba(300, 3, seed)
    k = 12
    g = O.build_csr(n, s, d)
    piv = O.maxmin(g, k)
    dip = O.pivot_dist(g, piv)
    newp, asg, it = O.kmeans_sp(dip, piv)
    assert 1 <= it <= 50
    Y = dip.T.astype(np.int64)
    cent = []
    for a in range(k):
        mem = np.nonzero(asg == a)[0]
        cent.append((Y[mem].sum(0), len(mem)) if len(mem) else None)
    def dist(i, a):
        S, c = cent[a]
        return sum(Fraction(int(Y[i, b]) * c - int(S[b]), c) ** 2 for b in range(k))
    for i in range(n):
        dd = [dist(i, a) for a in range(k) if cent[a] is not None]
        assert dist(i, asg[i]) == min(dd)
    for a in range(k):
        if cent[a] is None:
            assert newp[a] == piv[a]
            continue
        mem = np.nonzero(asg == a)[0]
        best = min(mem, key=lambda i: (dist(i, a), i))
        assert newp[a] == best


# ---------------------------------------------------------------- full stress (Section 3, before Eq. 4)

@pytest.mark.parametrize("name", ["grid", "rbtree", "rgg"])
def test_full_sweep_is_the_sparse_model_with_every_node_a_pivot(name):
    """Section 3: with k = n the sparse model reduces to full stress.  The
    full-stress sweep (all j != i with w = 1/d^2, j ascending) against the
    sparse sweep with every node a pivot (neighbours first, then pivots), in
    both orders; the two differ only in the order of the sums."""
    n, s, d = {"grid": lambda: I.grid(7, 9), "rbtree": lambda: I.random_btree(60, 2),
               "rgg": lambda: I.rgg(90, 6.0, 3)}[name]()
    g = O.build_csr(n, s, d)
    D = O.apsp(g)
    piv = np.arange(n, dtype=np.int32)
    w = O.adapted_weights(D, O.regions(D))
    x = np.random.default_rng(7).normal(size=(n, 2)) * 4
    a, ra = O.full_sweep(D, x, 0)
    b, rb = O.sweep_jacobi(g, piv, D, w, x)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    assert ra == pytest.approx(rb, rel=1e-12)
    c, _ = O.full_sweep(D, x, 1)
    np.testing.assert_allclose(c, O.sweep_gs(g, piv, D, w, x), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_full_gauss_seidel_decreases_full_stress(seed):
    """The node-at-a-time update decreases full stress monotonically (the
    property Section 3 cites); exhaustive stress after every sweep."""
    rng = np.random.default_rng(seed)
    n, s, d = _rand_graph(rng, 40, 0.06)
    g = O.build_csr(n, s, d)
    D = O.apsp(g)
    x = rng.normal(size=(n, 2)) * 5
    prev = O.full_stress(g, x)[0]
    for _ in range(8):
        x, _ = O.full_sweep(D, x, 1)
        cur = O.full_stress(g, x)[0]
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_full_sweep_keeps_an_exact_layout():
    """A path drawn at unit spacing realises every distance (r = d), so every
    term is x_j + (x_i - x_j) = x_i and the layout is a fixed point."""
    n, s, d = I.path(12)
    D = O.apsp(O.build_csr(n, s, d))
    x = np.stack([np.arange(n, dtype=np.float64), np.zeros(n)], 1)
    for order in (0, 1):
        y, rel = O.full_sweep(D, x, order)
        np.testing.assert_allclose(y, x, atol=1e-12)
        assert rel < 1e-14


# ---------------------------------------------------------------- the paper's region tie rule

def test_regions_smallest_hand_derived_path():
    """Path 0..8 with pivots (0, 8, 4): distances to the nearest pivot are
    0 (nodes 0, 4, 8), 1 (1, 3, 5, 7), 2 (2, 6).  Level 0: each pivot joins its
    own region (sizes 1, 1, 1).  Level 1 in id order: 1 -> region 0, 3 ->
    region 2, 5 -> region 2, 7 -> region 1 (each has one nearest pivot):
    sizes 2, 2, 3.  Level 2: node 2 ties between regions 0 and 2 (sizes 2 and
    3) -> 0; node 6 ties between regions 1 and 2 (sizes 2 and 3) -> 1."""
    n, s, d = I.path(9)
    g = O.build_csr(n, s, d)
    dip = O.pivot_dist(g, [0, 8, 4])
    assert O.regions_smallest(dip).tolist() == [0, 0, 0, 2, 2, 2, 1, 1, 1]


def test_regions_smallest_differs_from_lowest_index():
    """A star with centre 0 and leaves 1..6, a path 6-7-8, pivots (0, 7).
    Level 0: node 0 -> region 0, node 7 -> region 1.  Level 1 in id order:
    leaves 1..5 -> region 0 (size 6 after them); node 6 is at distance 1 from
    both pivots and joins the smaller region 1 (size 1), where the
    lowest-index rule puts it in region 0; node 8 -> region 1."""
    s = [0, 0, 0, 0, 0, 0, 6, 7]
    d = [1, 2, 3, 4, 5, 6, 7, 8]
    g = O.build_csr(9, s, d)
    dip = O.pivot_dist(g, [0, 7])
    assert O.regions(dip)[6] == 0
    assert O.regions_smallest(dip).tolist() == [0, 0, 0, 0, 0, 0, 1, 1, 1]


@pytest.mark.parametrize("seed", range(4))
def test_regions_smallest_is_a_nearest_pivot_partition(seed):
    """Invariants of any tie rule: every node joins a nearest pivot, every
    pivot node its own region (distinct pivots), and nodes with a single
    nearest pivot agree with the lowest-index rule."""
    rng = np.random.default_rng(seed)
    n, s, d = _rand_graph(rng, 60, 0.05)
    g = O.build_csr(n, s, d)
    piv = O.maxmin(g, 9)
    dip = O.pivot_dist(g, piv)
    reg = O.regions_smallest(dip)
    low = O.regions(dip)
    m = dip.min(0)
    assert (dip[reg, np.arange(n)] == m).all()
    for a, p in enumerate(piv):
        assert reg[p] == a
    single = (dip == m).sum(0) == 1
    assert np.array_equal(reg[single], low[single])


# ---------------------------------------------------------------- Procrustes statistic (Section 4)

def test_procrustes_similarity_transform_is_a_perfect_match():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(200, 2))
    th, sc, t = 0.7, 2.5, np.array([3.0, -1.0])
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Y = sc * X @ R.T + t
    P, s, a = O.procrustes(X, Y)
    assert abs(P) < 1e-14
    assert s == pytest.approx(sc, rel=1e-13)
    assert a == pytest.approx(th, rel=1e-13)


def test_procrustes_matches_the_library_for_proper_rotations():
    """scipy.spatial.procrustes fits an orthogonal map (reflections allowed):
    where the best orthogonal fit is a rotation its disparity equals P; for a
    mirror image scipy finds a perfect fit and P does not (the paper notes
    that its Procrustes analysis cannot resolve reflections)."""
    sp_proc = pytest.importorskip("scipy.spatial").procrustes
    rng = np.random.default_rng(9)
    X = rng.normal(size=(150, 2))
    Y = X @ np.array([[0.6, -0.8], [0.8, 0.6]]).T + 0.3 * rng.normal(size=(150, 2))
    _, _, disp = sp_proc(X, Y)
    assert O.procrustes(X, Y)[0] == pytest.approx(disp, rel=1e-12)
    M = X * np.array([1.0, -1.0])
    _, _, disp = sp_proc(X, M)
    assert disp < 1e-14
    assert O.procrustes(X, M)[0] > 0.1


def test_procrustes_range():
    rng = np.random.default_rng(2)
    for _ in range(5):
        X, Y = rng.normal(size=(80, 2)), rng.normal(size=(80, 2))
        P = O.procrustes(X, Y)[0]
        assert 0.0 <= P <= 1.0


# ---------------------------------------------------------------- convex-hull error (Section 4, Fig. 4)

def test_hull_error_against_library_hull():
    """The per-node counts of the oracle against scipy's ConvexHull (Qhull) and
    matplotlib-free point-in-polygon by Delaunay.find_simplex on random layouts
    in general position (no three points collinear with probability 1)."""
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(12)
    n, s, d = I.rgg(120, 7.0, 5)
    g = O.build_csr(n, s, d)
    D = O.apsp(g)
    x = rng.normal(size=(n, 2))
    for kh in (1, 2, 4):
        mean, per = O.hull_error(D, x, kh)
        want = np.zeros(n)
        for v in range(n):
            ball = np.nonzero(D[v] <= kh)[0]
            out = np.nonzero(D[v] > kh)[0]
            if len(out) == 0:
                continue
            if len(ball) >= 3:
                tri = spatial.Delaunay(x[ball])
                inside = tri.find_simplex(x[out]) >= 0
            else:
                inside = np.zeros(len(out), bool)  # a point or a segment holds no other random point
            want[v] = inside.sum() / len(out)
        np.testing.assert_allclose(per, want, atol=0)
        assert mean == pytest.approx(want.mean(), rel=1e-12)


def test_hull_error_closed_forms():
    """A 5 x 5 grid drawn at its integer coordinates, radius 1: the ball of an
    interior node is a plus sign whose hull (a diamond) holds no other grid
    point, so every error is 0; radius 2 for the centre node: the diamond
    |dx| + |dy| <= 2 holds exactly the ball.  A layout that stacks every
    node on one point puts every other node on the hull: error 1."""
    n, s, d = I.grid(5, 5)
    D = O.apsp(O.build_csr(n, s, d))
    r, c = np.divmod(np.arange(n), 5)
    x = np.stack([c, r], 1).astype(np.float64)
    mean, per = O.hull_error(D, x, 1)
    assert mean == 0.0
    _, per2 = O.hull_error(D, x, 2)
    assert per2[12] == 0.0
    mean, per = O.hull_error(D, np.zeros((n, 2)), 1)
    assert (per == 1.0).all()


# ---------------------------------------------------------------- Gabriel graph similarity (Section 4, Fig. 3)

def test_gabriel_graph_is_the_delaunay_subgraph_of_empty_diameter_discs():
    """Library pin: the Gabriel graph is the set of Delaunay edges (scipy,
    Qhull) whose diameter disc holds no other point; on random points in
    general position the oracle's brute-force definition gives exactly that."""
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(3)
    x = rng.random((150, 2))
    adj = O.gabriel(x)
    tri = spatial.Delaunay(x)
    want = np.zeros_like(adj)
    tree = spatial.cKDTree(x)
    for simplex in tri.simplices:
        for a, b in ((0, 1), (1, 2), (0, 2)):
            u, v = simplex[a], simplex[b]
            m = (x[u] + x[v]) / 2
            r = np.linalg.norm(x[u] - x[v]) / 2
            inside = [w for w in tree.query_ball_point(m, r * (1 - 1e-12)) if w not in (u, v)]
            if not inside:
                want[u, v] = want[v, u] = 1
    assert np.array_equal(adj, want)


def test_gabriel_special_cases():
    """A square's corners: the other two corners lie on the diagonals'
    diameter circles, not inside, so under the open-disc reading all six pairs
    are Gabriel edges; identical positions are adjacent; a point at a
    segment's midpoint blocks it."""
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    adj = O.gabriel(sq)
    assert adj.sum() == 12  # all 6 pairs: the diagonals' circles pass through the other corners
    line = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]])
    assert O.gabriel(line).tolist() == [[0, 1, 0], [1, 0, 1], [0, 1, 0]]
    dup = np.array([[0.0, 0.0], [0.0, 0.0], [5.0, 5.0], [0.1, 4.9]])
    assert O.gabriel(dup)[0, 1] == 1


def test_gabriel_jaccard_identity_and_disjoint():
    rng = np.random.default_rng(8)
    x = rng.random((60, 2))
    mean, per = O.gabriel_jaccard(x, x, 2)
    assert mean == 1.0 and (per == 1.0).all()
    # a layout and its copy rotated by 90 degrees have the same Gabriel graph
    mean, _ = O.gabriel_jaccard(x, x[:, ::-1] * np.array([-1.0, 1.0]), 3)
    assert mean == 1.0
    # two layouts whose Gabriel graphs share no edge at radius 1
    line = np.stack([np.arange(6.0), np.zeros(6)], 1)
    perm = np.array([0, 2, 4, 1, 3, 5])
    mean, per = O.gabriel_jaccard(line, line[np.argsort(perm)], 1)
    adjA, adjB = O.gabriel(line), O.gabriel(line[np.argsort(perm)])
    for v in range(6):
        a, b = set(np.nonzero(adjA[v])[0]), set(np.nonzero(adjB[v])[0])
        assert per[v] == pytest.approx(len(a & b) / len(a | b))
