"""CUDA path against the FP64 oracle, through the C ABI.

Integer stages (CSR, pivots, d_ip, regions, counts) must match bit for bit;
floating-point stages within the tolerances stated in each test:
  * positions: max_i ||x_i^gpu - x_i^orc|| / RMS_i ||x_i^orc - mean|| <= 1e-5
    for the FP32 sweep at equal input (FP64 sweep: 1e-10);
  * stress: relative error <= 1e-9 at equal positions (FP64 sums);
  * PivotMDS eigenvalues: relative error <= 1e-10.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _rand_graph(seed, n, extra):
    rng = np.random.default_rng(seed)
    src = [int(rng.integers(0, v)) for v in range(1, n)]
    dst = list(range(1, n))
    e = rng.integers(0, n, (extra, 2))
    src += e[:, 0].tolist()  # includes self-loops and repeats
    dst += e[:, 1].tolist()
    return n, np.array(src, np.int32), np.array(dst, np.int32)


GRAPHS = {
    "grid32": lambda: I.grid(32, 32),
    "grid_ragged": lambda: I.grid(17, 45),
    "path": lambda: I.path(300),
    "btree": lambda: I.complete_btree(9),
    "rbtree": lambda: I.random_btree(3001, 4),
    "rgg": lambda: I.rgg(6000, 8.0, 7),
    "ba": lambda: I.ba(20000, 4, 3),
    "messy": lambda: _rand_graph(5, 2500, 9000),
}


def _gpu_graph(n, s, d):
    return ssm.ssm_build_graph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV))


def _norm_err(a, b):
    b = np.asarray(b, np.float64)
    a = np.asarray(a, np.float64)
    c = b - b.mean(0)
    rms = np.sqrt((c ** 2).sum(1).mean())
    return np.sqrt(((a - b) ** 2).sum(1)).max() / rms


# ------------------------------------------------------------------ a0 graph

@pytest.mark.parametrize("name", list(GRAPHS))
def test_build_graph_bit_exact(name):
    n, s, d = GRAPHS[name]()
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    assert g.m == og.m
    assert np.array_equal(g.rowptr.cpu().numpy(), og.rowptr)
    assert np.array_equal(g.colidx.cpu().numpy(), og.colidx)


def test_build_graph_hub_row():
    # a star with 20000 leaves (row longer than the shared-memory sort) plus repeats
    n = 20001
    leaves = np.arange(1, n, dtype=np.int32)
    rng = np.random.default_rng(0)
    perm = rng.permutation(leaves)
    s = np.concatenate([np.zeros(n - 1, np.int32), perm[:500]])
    d = np.concatenate([perm, np.zeros(500, np.int32)])
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    assert np.array_equal(g.colidx.cpu().numpy(), og.colidx)


def test_build_graph_errors():
    with pytest.raises(ssm.SSMError) as e:
        _gpu_graph(4, np.array([0, 1], np.int32), np.array([1, 4], np.int32))
    assert e.value.code == -2
    with pytest.raises(ssm.SSMError) as e:
        _gpu_graph(4, np.array([0, 2], np.int32), np.array([1, 3], np.int32))
    assert e.value.code == -3


@pytest.mark.parametrize("case", ["pieces", "crossed", "pairs"])
def test_build_graph_counts_components(case):
    """The connectivity check finds the exact number of components (named in
    the error), also where each node's first two neighbours join little and
    most nodes lie outside the largest component."""
    if case == "pieces":  # a grid, a BA graph and 7 isolated nodes
        n1, s1, d1 = I.grid(100, 100)
        n2, s2, d2 = I.ba(5000, 2, 3)
        n, want = n1 + n2 + 7, 9
        s = np.concatenate([s1, s2 + n1]).astype(np.int32)
        d = np.concatenate([d1, d2 + n1]).astype(np.int32)
    elif case == "crossed":  # 40 cycles of 250 nodes, node ids dealt round-robin over the cycles
        c, L = 40, 250
        ids = np.arange(c * L, dtype=np.int64).reshape(L, c).T  # cycle j holds j, j + c, j + 2c, ...
        s = ids.reshape(-1).astype(np.int32)
        d = np.roll(ids, -1, axis=1).reshape(-1).astype(np.int32)
        n, want = c * L, c
    else:  # 1000 disjoint edges
        n, want = 2000, 1000
        s = np.arange(0, n, 2, dtype=np.int32)
        d = s + 1
    with pytest.raises(ssm.SSMError) as e:
        _gpu_graph(n, s, d)
    assert e.value.code == -3
    assert f"{want} connected components" in str(e.value)


# ------------------------------------------------------------------ a1 pivots

@pytest.mark.parametrize("name,k,start", [("grid32", 50, 0), ("grid_ragged", 33, 5), ("path", 7, 150),
                                          ("btree", 40, 0), ("rbtree", 64, 17), ("rgg", 100, 0), ("ba", 100, 0),
                                          ("messy", 1, 3), ("messy", 65, 0)])
def test_select_pivots_bit_exact(name, k, start):
    n, s, d = GRAPHS[name]()
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    got = ssm.ssm_select_pivots(g, k, start).cpu().numpy()
    assert np.array_equal(got, O.maxmin(og, k, start))


def test_select_pivots_k_equals_n():
    n, s, d = I.grid(5, 7)
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    got = ssm.ssm_select_pivots(g, n, 0).cpu().numpy()
    assert np.array_equal(got, O.maxmin(og, n, 0))
    assert sorted(got.tolist()) == list(range(n))


def test_select_pivots_tiny_graphs():
    for n in (2, 3, 5):
        n_, s, d = I.path(n)
        og = O.build_csr(n_, s, d)
        g = _gpu_graph(n_, s, d)
        got = ssm.ssm_select_pivots(g, n_, n_ - 1).cpu().numpy()
        assert np.array_equal(got, O.maxmin(og, n_, n_ - 1))


def test_select_pivots_long_path():
    # 20000 BFS levels per pivot
    n, s, d = I.path(20000)
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    got = ssm.ssm_select_pivots(g, 6, 777).cpu().numpy()
    assert np.array_equal(got, O.maxmin(og, 6, 777))


@pytest.mark.parametrize("start", [0, 5])
def test_select_pivots_star_frontier_overflow(start):
    # one BFS level of 300000 nodes: more than the shared-memory queues of the
    # cluster kernel hold, so most of the level goes through the global spill
    n = 300001
    s = np.zeros(n - 1, np.int32)
    d = np.arange(1, n, dtype=np.int32)
    # a short tail so the pivots are not all leaves of the star
    s = np.concatenate([s, np.array([7, 300001, 300002], np.int32)])
    d = np.concatenate([d, np.array([300001, 300002, 300003], np.int32)])
    n += 3
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    got = ssm.ssm_select_pivots(g, 5, start).cpu().numpy()
    assert np.array_equal(got, O.maxmin(og, 5, start))


def test_select_pivots_4_byte_cluster_kernel():
    # 720000 nodes still fit a 4-byte mind in the cluster
    n, s, d = I.grid(900, 800)
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    got = ssm.ssm_select_pivots(g, 6, 12345).cpu().numpy()
    assert ssm.ssm_last_pivot_config() == {"cluster": 16, "mind_bytes": 4}
    assert np.array_equal(got, O.maxmin(og, 6, 12345))


def test_select_pivots_large_grid_kernel():
    # 960000 nodes: a 4-byte mind does not fit the cluster's shared memory, a
    # 2-byte one does (node pairs claimed by compare-and-swap); 1,900 levels
    n, s, d = I.grid(1000, 960)
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    got = ssm.ssm_select_pivots(g, 6, 12345).cpu().numpy()
    assert ssm.ssm_last_pivot_config() == {"cluster": 16, "mind_bytes": 2}
    assert np.array_equal(got, O.maxmin(og, 6, 12345))


def test_select_pivots_large_ba_kernel():
    # 1,000,000 nodes of a Barabasi-Albert graph (hubs, small diameter): one
    # search over every node, then many short pruned searches, with the
    # 2-byte mind of the cluster kernel
    n, s, d = I.ba(1000000, 4, 3)
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    got = ssm.ssm_select_pivots(g, 24, 0).cpu().numpy()
    assert ssm.ssm_last_pivot_config() == {"cluster": 16, "mind_bytes": 2}
    assert np.array_equal(got, O.maxmin(og, 24, 0))


@pytest.mark.parametrize("case", ["ba_pair", "path_pair"])
def test_select_pivots_disconnected(case):
    """Max/min on a disconnected CSR reports SSM_E_DISCONNECTED, whether the
    first search runs to its end (two small-world pieces) or hands the search
    over to the cluster kernel (two paths, deeper than its level limit)."""
    if case == "ba_pair":
        n1, s1, d1 = I.ba(3000, 2, 5)
        n = 2 * n1
        s, d = np.concatenate([s1, s1 + n1]), np.concatenate([d1, d1 + n1])
    else:
        n, half = 80, 40
        s = np.array(list(range(0, half - 1)) + list(range(half, n - 1)), np.int32)
        d = s + 1
    og = O.build_csr(n, s.astype(np.int32), d.astype(np.int32))
    g = ssm.Graph(n, og.m, torch.from_numpy(og.rowptr).to(DEV), torch.from_numpy(og.colidx).to(DEV))
    with pytest.raises(ssm.SSMError) as e:
        ssm.ssm_select_pivots(g, 10, 0)
    assert e.value.code == -3


def test_select_pivots_deep_search_hands_over_to_the_grid_kernel():
    # a 900,000-node path: the 2-byte mind of the cluster kernel cannot hold
    # level 65535, so the grid kernel queued behind it redoes the selection
    n, s, d = I.path(900000)
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    got = ssm.ssm_select_pivots(g, 3, 450000).cpu().numpy()
    assert ssm.ssm_last_pivot_config() == {"cluster": 16, "mind_bytes": 2}
    assert np.array_equal(got, O.maxmin(og, 3, 450000))


# ------------------------------------------------------------------ a2 d_ip

@pytest.mark.parametrize("name,k", [("grid32", 50), ("path", 7), ("btree", 33), ("rgg", 100), ("ba", 64),
                                    ("messy", 1), ("messy", 95), ("ba", 300), ("messy", 600)])
def test_pivot_bfs_bit_exact(name, k):
    """Small-diameter graphs (ba, messy, btree) take the pulled bitset BFS,
    k > 256 in several passes; the others give up on it after 24 levels and
    take the per-source BFS."""
    n, s, d = GRAPHS[name]()
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    piv = O.maxmin(og, k, 0)
    dip = ssm.ssm_pivot_bfs(g, torch.from_numpy(piv).to(DEV)).cpu().numpy()
    assert np.array_equal(dip, O.pivot_dist(og, piv))


def test_pivot_bfs_repeated_pivots():
    n, s, d = GRAPHS["rbtree"]()
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    piv = np.array([5, 5, 0, 17, 5, 2999] * 7, np.int32)
    dip = ssm.ssm_pivot_bfs(g, torch.from_numpy(piv).to(DEV)).cpu().numpy()
    assert np.array_equal(dip, O.pivot_dist(og, piv))


def test_pivot_bfs_long_graph_with_hub_rows():
    """A path of 300 nodes (too deep for the pulled BFS) carrying a star of 1000
    leaves and nodes of degree 20 to 40: the per-source BFS walks short rows
    one lane per row and the long ones with the whole warp, in one level."""
    rng = np.random.default_rng(11)
    L = 300
    s = list(range(L - 1))
    d = list(range(1, L))
    nxt = L
    for hub, leaves in [(150, 1000), (40, 33), (41, 32), (260, 20), (261, 40)]:
        s += [hub] * leaves
        d += list(range(nxt, nxt + leaves))
        nxt += leaves
    # a few chords between leaves of different hubs
    leaves_all = np.arange(L, nxt)
    a, b = rng.choice(leaves_all, 50), rng.choice(leaves_all, 50)
    keep = a != b
    s += list(a[keep])
    d += list(b[keep])
    n = nxt
    s, d = np.array(s, np.int32), np.array(d, np.int32)
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    piv = O.maxmin(og, 12, 0)
    dip = ssm.ssm_pivot_bfs(g, torch.from_numpy(piv).to(DEV)).cpu().numpy()
    assert np.array_equal(dip, O.pivot_dist(og, piv))


def _broom_graph(B):
    """A path of 40 nodes ending in a hub with B leaves, each leaf with a
    pendant node: two BFS levels of B nodes behind a hub row, deep enough for
    the per-source BFS."""
    L = 40
    s = list(range(L - 1)) + [L - 1] * B + list(range(L, L + B))
    d = list(range(1, L)) + list(range(L, L + B)) + list(range(L + B, L + 2 * B))
    return L + 2 * B, np.array(s, np.int32), np.array(d, np.int32)


@pytest.mark.parametrize("k,B", [(6, 70000), (400, 5000), (6, 5000)])
def test_pivot_bfs_wide_levels(k, B):
    """Frontiers larger than the shared-memory part of the frontier queue
    (few sources on a graph above 131072 nodes: 4096 entries per level there,
    the rest in global memory; otherwise all in global memory), reached
    through a row of B entries."""
    n, s, d = _broom_graph(B)
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    rng = np.random.default_rng(k)
    piv = np.concatenate([[0, 20], rng.integers(0, n, k - 2)]).astype(np.int32)
    dip = ssm.ssm_pivot_bfs(g, torch.from_numpy(piv).to(DEV)).cpu().numpy()
    assert np.array_equal(dip, O.pivot_dist(og, piv))


def test_pivot_bfs_many_sources_deep_graph():
    """More sources than two per SM on a large-diameter graph: four blocks
    per SM, frontier in global memory."""
    n, s, d = GRAPHS["rgg"]()
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    piv = np.random.default_rng(5).integers(0, n, 700).astype(np.int32)
    dip = ssm.ssm_pivot_bfs(g, torch.from_numpy(piv).to(DEV)).cpu().numpy()
    assert np.array_equal(dip, O.pivot_dist(og, piv))


@pytest.mark.parametrize("long_arm", [False, True])
def test_pivot_bfs_disconnected(long_arm):
    # two paths: short (the pulled BFS notices) or longer than 24 levels (the
    # per-source BFS does)
    n = 80 if long_arm else 40
    half = n // 2
    s = np.array(list(range(0, half - 1)) + list(range(half, n - 1)), np.int32)
    d = s + 1
    og = O.build_csr(n, s, d)
    g = ssm.Graph(n, og.m, torch.from_numpy(og.rowptr).to(DEV), torch.from_numpy(og.colidx).to(DEV))
    with pytest.raises(ssm.SSMError) as e:
        ssm.ssm_pivot_bfs(g, torch.tensor([0, half + 5], dtype=torch.int32, device=DEV))
    assert e.value.code == -3


# ------------------------------------------------------------------ a3 regions and counts

@pytest.mark.parametrize("name,k", [("grid32", 50), ("path", 7), ("btree", 33), ("rgg", 100), ("ba", 64),
                                    ("messy", 95)])
def test_aggregate_bit_exact(name, k):
    n, s, d = GRAPHS[name]()
    og = O.build_csr(n, s, d)
    piv = O.maxmin(og, k, 0)
    dip = O.pivot_dist(og, piv)
    reg, (ecc, off, cnt) = O.regions(dip), O.histograms(dip, O.regions(dip))
    gd = torch.from_numpy(dip).to(DEV)
    assert ssm.ssm_aggregate_size(gd) == len(cnt)
    greg, goff, gcnt = ssm.ssm_aggregate(gd)
    assert np.array_equal(greg.cpu().numpy(), reg)
    assert np.array_equal(goff.cpu().numpy().astype(np.int64), off)
    assert np.array_equal(gcnt.cpu().numpy(), cnt)


# ------------------------------------------------------------------ a4/a5 PivotMDS

def _gram_u128(lo, hi):
    lo = lo.cpu().numpy().view(np.uint64)
    hi = hi.cpu().numpy().view(np.uint64)
    return lo, hi


@pytest.mark.parametrize("k,n,dmax,offset", [
    (200, 20001, 3, 0),        # one 7-bit digit, odd n (two-byte loads), ragged second tile
    (300, 70001, 11, 0),       # one 7-bit digit at its largest (121): read out every 17 chunks
    (200, 300001, 2, 0),       # one digit read out every 256 chunks, odd n
    (256, 150000, 8, 0),       # one digit read out every 64 chunks (d <= 8), full tiles, 4-byte loads
    (150, 65538, 7, 0),        # one digit, even n with a ragged last chunk
    (300, 70000, 12, 0),       # the smallest squared distance that needs 5-bit digits (144)
    (200, 20001, 15, 0),       # two digits
    (130, 33000, 200, 0),      # four digits, even n (four-byte loads), three node ranges
    (130, 33000, 200, 1),      # the same table two bytes off a 4-byte boundary
    (129, 16389, 3000, 0),     # six digits, a node range of 5 nodes
    (256, 5000, 65534, 0),     # eight digits (16 digit blocks), full tiles
    (1, 70, 65534, 0),         # one pivot: G is one number, above 2^64
    (3, 1, 9, 0),              # one node
])
def test_gram_exact(k, n, dmax, offset):
    """The tensor-core Gram matrix, every entry a <= b bit-exact in 128 bits,
    zero below the diagonal."""
    dip = I.distance_table(k, n, dmax, 11 + k + n)
    buf = torch.zeros(k * n + offset, dtype=torch.int16, device=DEV)
    buf[offset:] = torch.from_numpy(dip.view(np.int16).reshape(-1)).to(DEV)
    gd = buf[offset:].view(k, n)
    lo, hi = _gram_u128(*ssm.ssm_gram(gd))
    G = O.gram(dip)
    iu = np.triu_indices(k)
    got = [(int(h) << 64) | int(l) for h, l in zip(hi[iu], lo[iu])]
    assert got == list(G[iu])
    il = np.tril_indices(k, -1)
    assert not lo[il].any() and not hi[il].any()


@pytest.mark.parametrize("name,k", [("grid32", 50), ("rgg", 100), ("ba", 64), ("btree", 33), ("path", 7)])
def test_pivotmds_matches_oracle(name, k):
    """Eigenvalues to 1e-10; positions to FP32 rounding where the eigenvector is
    unique.  Where lambda_2 is degenerate (the complete binary tree is
    symmetric, lambda_2 = lambda_3) any unit vector of the eigenspace is a
    valid second axis, so the test checks what is unique: the first axis, and
    that the second axis y = C v has ||y||^2 = lambda_2 and y . x = 0."""
    n, s, d = GRAPHS[name]()
    og = O.build_csr(n, s, d)
    piv = O.maxmin(og, k, 0)
    dip = O.pivot_dist(og, piv)
    opos, oeig, B = O.pivotmds(dip, return_b=True)
    lam = np.linalg.eigvalsh(B)[::-1]
    unique2 = (lam[1] - lam[2]) > 1e-6 * lam[0] and oeig[1] > 1e-6 * oeig[0]
    g = _gpu_graph(n, s, d)
    for prec in (32, 64):
        pos, eig = ssm.ssm_pivotmds(g, torch.from_numpy(dip).to(DEV), precision=prec, rescale=False)
        eig = eig.cpu().numpy()
        np.testing.assert_allclose(eig[0], oeig[0], rtol=1e-10)
        if oeig[1] > 1e-9 * oeig[0]:
            np.testing.assert_allclose(eig[1], oeig[1], rtol=1e-10)
        p = pos.cpu().numpy().astype(np.float64)
        tol = 2e-6 if prec == 32 else 1e-9
        if unique2:
            assert _norm_err(p, opos) < tol
        else:
            assert _norm_err(p[:, :1], opos[:, :1]) < tol
            if oeig[1] > 1e-6 * oeig[0]:
                y = p[:, 1] - p[:, 1].mean()
                x = p[:, 0] - p[:, 0].mean()
                assert np.dot(y, y) == pytest.approx(oeig[1], rel=1e-5)
                assert abs(np.dot(x, y)) <= 1e-5 * np.sqrt(oeig[0] * oeig[1])
    # with the rescale of Algorithm 1 line 4
    pos, _ = ssm.ssm_pivotmds(g, torch.from_numpy(dip).to(DEV), precision=64, rescale=True)
    if unique2:
        assert _norm_err(pos.cpu().numpy(), O.rescale(og, opos)) < 1e-9


@pytest.mark.parametrize("n0,seed", [(83, 2573530203214907681), (725, 3306426093002437330)])
def test_pivotmds_small_second_eigenvalue(n0, seed):
    """Small RGGs whose lambda_2 / lambda_1 is below 1e-2: the second pair sinks
    below FP64 precision in the powers of B, and the solver finishes on B
    itself; eigenvalues to 1e-10, positions to FP32 / FP64 rounding."""
    n, s, d = I.mixed_graph("rgg", n0, seed)
    k = max(2, min(100, n // 4))
    og = O.build_csr(n, s, d)
    dip = O.pivot_dist(og, O.maxmin(og, k, 0))
    opos, oeig, B = O.pivotmds(dip, return_b=True)
    lam = np.linalg.eigvalsh(B)[::-1]
    assert lam[1] < 0.03 * lam[0]
    g = _gpu_graph(n, s, d)
    for prec, tol in ((32, 2e-6), (64, 1e-9)):
        pos, eig = ssm.ssm_pivotmds(g, torch.from_numpy(dip).to(DEV), precision=prec, rescale=False)
        eig = eig.cpu().numpy()
        np.testing.assert_allclose(eig[:2], oeig, rtol=1e-10)
        assert _norm_err(pos.cpu().numpy().astype(np.float64), opos) < tol


# ------------------------------------------------------------------ a6/a7 sweep

def _gpu_pivots(k, prep):
    return ssm.Pivots(k, torch.from_numpy(prep.pivots).to(DEV), torch.from_numpy(prep.dip).to(DEV),
                      torch.from_numpy(prep.region).to(DEV),
                      torch.from_numpy(prep.cnt_off.astype(np.int32)).to(DEV), torch.from_numpy(prep.cnt).to(DEV))


@pytest.mark.parametrize("name,k", [("grid32", 50), ("rgg", 100), ("ba", 64), ("btree", 33), ("messy", 95)])
def test_sweep_fp64_matches_oracle(name, k):
    """The FP64 sweep rounds every operation as the oracle does, in the same
    order, so the trajectories agree bit for bit even where the Jacobi
    dynamics amplify rounding differences (near-coincident nodes of the
    PivotMDS start: a 1e-15 perturbation grows to 1e-2 within 5 iterations
    on the RGG and to 0.4 on the binary tree)."""
    n, s, d = GRAPHS[name]()
    prep = O.prepare(n, s, d, k)
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(k, prep)
    pos = torch.from_numpy(prep.pos0.copy()).to(DEV)
    iters = 20
    done, rel = ssm.ssm_iterate(g, P, pos, iters)
    opos, orel = O.iterate(prep, prep.pos0, iters)
    assert int(done.item()) == iters
    assert np.array_equal(pos.cpu().numpy(), opos)
    assert rel.item() == pytest.approx(orel, rel=1e-12)


@pytest.mark.parametrize("name,k", [("grid32", 50), ("grid_ragged", 33), ("rgg", 100), ("ba", 64), ("btree", 33),
                                    ("messy", 95), ("rbtree", 64), ("ba", 377)])
def test_sweep_fp32_single_step(name, k):
    n, s, d = GRAPHS[name]()
    prep = O.prepare(n, s, d, k)
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(k, prep)
    x0 = prep.pos0.astype(np.float32)
    pos = torch.from_numpy(x0.copy()).to(DEV)
    done, rel = ssm.ssm_iterate(g, P, pos, 1)
    opos, orel = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, x0.astype(np.float64))
    assert _norm_err(pos.cpu().numpy(), opos) < 1e-5
    assert rel.item() == pytest.approx(orel, rel=1e-4)


def _hubs_graph():
    """A long row (node 0, degree 3999), a medium row (node 1, degree ~500) and
    short rows (a random tree plus random extra edges)."""
    n, s, d = _rand_graph(11, 4000, 3000)
    s = np.concatenate([s, np.zeros(3999, np.int32), np.ones(500, np.int32)])
    d = np.concatenate([d, np.arange(1, 4000, dtype=np.int32), np.arange(3000, 3500, dtype=np.int32)])
    return n, s, d


@pytest.mark.parametrize("k", [8, 60])
def test_sweep_fp32_long_medium_short_rows(k):
    """Neighbour sums are taken per thread (short rows), per warp (medium rows)
    and per block (rows above 1024 entries); one step from the same state."""
    n, s, d = _hubs_graph()
    prep = O.prepare(n, s, d, k)
    deg = np.diff(prep.g.rowptr)
    assert deg.max() > 1024 and ((deg > 32) & (deg <= 1024)).any()
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(k, prep)
    x0 = prep.pos0.astype(np.float32)
    pos = torch.from_numpy(x0.copy()).to(DEV)
    ssm.ssm_iterate(g, P, pos, 1)
    opos, _ = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, x0.astype(np.float64))
    assert _norm_err(pos.cpu().numpy(), opos) < 1e-5


@pytest.mark.parametrize("k", [12, 100])
def test_sweep_fp32_both_weight_table_modes(k):
    """The FP32 sweep keeps a (w, w d) table over all pivots and distances when
    k * (max d + 1) entries fit (k = 12 on this graph) and a clamped s table
    otherwise (k = 100); both must meet the tolerance from the same state."""
    n, s, d = GRAPHS["rgg"]()
    prep = O.prepare(n, s, d, k)
    dmax = int(prep.dip.max())
    assert (k * (dmax + 1) <= 6112) == (k == 12)
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(k, prep)
    x = prep.pos0
    for _ in range(3):
        x, _ = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, x)
    x0 = x.astype(np.float32)
    pos = torch.from_numpy(x0.copy()).to(DEV)
    ssm.ssm_iterate(g, P, pos, 1)
    cfg = ssm.ssm_last_sweep_config()
    assert cfg["kernel"] == ("f32_full_table" if k == 12 else "f32_clamped_smem")
    assert cfg["dmax"] == dmax
    opos, _ = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, x0.astype(np.float64))
    assert _norm_err(pos.cpu().numpy(), opos) < 1e-5


def test_sweep_fp32_single_node_regions():
    """Pivots whose region is the pivot alone (ecc = 0) still weigh every node at
    distance d >= 2 with s = |R(a)| = 1 (w' = 1/d^2), in the clamped-table mode
    (a 2000-node path, so k (max d + 1) is far above the full table) of the
    single-graph sweep and in the batched sweep."""
    n, s, d = I.path(2000)
    og = O.build_csr(n, s, d)
    piv = np.array(list(range(9)) + [1000, 1999], np.int32)
    k = len(piv)
    dip = O.pivot_dist(og, piv)
    reg = O.regions(dip)
    ecc, off, cnt = O.histograms(dip, reg)
    assert (np.asarray(ecc)[:8] == 0).all()
    w = O.adapted_weights(dip, reg)
    rng = np.random.default_rng(5)
    x0 = rng.normal(size=(n, 2)).astype(np.float32)
    want, _ = O.sweep_jacobi(og, piv, dip, w, x0.astype(np.float64))
    g = _gpu_graph(n, s, d)
    P = ssm.Pivots(k, torch.from_numpy(piv).to(DEV), torch.from_numpy(dip).to(DEV), torch.from_numpy(reg).to(DEV),
                   torch.from_numpy(np.asarray(off).astype(np.int32)).to(DEV), torch.from_numpy(cnt).to(DEV))
    pos = torch.from_numpy(x0.copy()).to(DEV)
    ssm.ssm_iterate(g, P, pos, 1)
    assert _norm_err(pos.cpu().numpy(), want) < 1e-5
    pos = torch.from_numpy(x0.copy()).to(DEV)
    ssm.ssm_batch_iterate([(g, P, pos)], 1)
    assert _norm_err(pos.cpu().numpy(), want) < 1e-5


@pytest.mark.parametrize("name,k", [("rgg", 100), ("ba", 64), ("btree", 33)])
def test_sweep_fp32_along_oracle_trajectory(name, k):
    """FP32 step error along the oracle's FP64 trajectory: at every iteration t
    the GPU computes X^{t+1} from the oracle's X^t (rounded to FP32)."""
    n, s, d = GRAPHS[name]()
    prep = O.prepare(n, s, d, k)
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(k, prep)
    x = prep.pos0
    worst = 0.0
    for _ in range(25):
        pos = torch.from_numpy(x.astype(np.float32)).to(DEV)
        ssm.ssm_iterate(g, P, pos, 1)
        x_next, _ = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, x.astype(np.float32).astype(np.float64))
        worst = max(worst, _norm_err(pos.cpu().numpy(), x_next))
        x, _ = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, x)
    assert worst < 1e-5


def test_sweep_fp32_grid_200_iterations():
    """The small plain configuration: 32x32 grid, k=50, 200 Jacobi iterations."""
    n, s, d = I.grid(32, 32)
    prep = O.prepare(n, s, d, 50)
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(50, prep)
    x0 = prep.pos0.astype(np.float32)
    pos = torch.from_numpy(x0.copy()).to(DEV)
    ssm.ssm_iterate(g, P, pos, 200)
    opos, _ = O.iterate(prep, x0.astype(np.float64), 200)
    assert _norm_err(pos.cpu().numpy(), opos) < 1e-5


def test_sweep_early_stop():
    """tol > 0 stops on the device at the first iteration whose relative change
    is below tol (43 on this grid; the Jacobi change then plateaus near 5.7e-5)."""
    n, s, d = I.grid(32, 32)
    prep = O.prepare(n, s, d, 50)
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(50, prep)
    pos = torch.from_numpy(prep.pos0.copy()).to(DEV)
    done, rel = ssm.ssm_iterate(g, P, pos, 500, tol=1e-4)
    t = int(done.item())
    assert 1 <= t < 500
    opos, orel = O.iterate(prep, prep.pos0, t)
    assert orel < 1e-4
    _, prev = O.iterate(prep, prep.pos0, t - 1) if t > 1 else (None, 1.0)
    assert prev >= 1e-4
    assert _norm_err(pos.cpu().numpy(), opos) < 1e-10


def test_sweep_odd_n_and_tail():
    n, s, d = I.grid(13, 13)  # n = 169 (odd) -> one-node-per-thread path with a ragged tile
    prep = O.prepare(n, s, d, 9)
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(9, prep)
    x0 = prep.pos0.astype(np.float32)
    pos = torch.from_numpy(x0.copy()).to(DEV)
    ssm.ssm_iterate(g, P, pos, 3)
    opos, _ = O.iterate(prep, x0.astype(np.float64), 3)
    assert _norm_err(pos.cpu().numpy(), opos) < 1e-5


# ------------------------------------------------------------------ a8 stress

@pytest.mark.parametrize("name", ["grid32", "btree", "messy"])
def test_stress_exhaustive(name):
    n, s, d = GRAPHS[name]()
    prep = O.prepare(n, s, d, 20)
    g = _gpu_graph(n, s, d)
    for prec in (32, 64):
        x = prep.pos0.astype(np.float32).astype(np.float64) if prec == 32 else prep.pos0
        pos = torch.from_numpy(x.astype(np.float32) if prec == 32 else x).to(DEV)
        out, sums = ssm.ssm_stress(g, pos)
        want, wsums = O.full_stress(prep.g, x, return_sums=True)
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-9)
        assert sums[3].item() == wsums[3] == n * (n - 1) / 2


@pytest.mark.parametrize("name,S,T,seed", [("rgg", 64, 256, 1), ("rgg", 100, 37, 9), ("ba", 600, 100, 3),
                                           ("ba", 256, 64, 5)])
def test_stress_sampled(name, S, T, seed):
    """Sampled pairs: on the geometric graph (large diameter) the pulled BFS
    gives up and the distance table is written; on the Barabasi-Albert graph
    each pass of it sums its sources' pairs from its level bits (three passes
    for 600 sources, the last one partial)."""
    n, s, d = GRAPHS[name]()
    prep = O.prepare(n, s, d, 30)
    g = _gpu_graph(n, s, d)
    x = prep.pos0.astype(np.float32)
    out, sums = ssm.ssm_stress(g, torch.from_numpy(x).to(DEV), S, T, seed)
    want, wsums = O.full_stress(prep.g, x.astype(np.float64), S, T, seed, return_sums=True)
    np.testing.assert_allclose(sums.cpu().numpy(), wsums, rtol=1e-9)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-9)


# ------------------------------------------------------------------ whole pipeline

def test_pipeline_grid32_end_to_end():
    """All rows on the small plain configuration, GPU pipeline vs oracle pipeline."""
    n, s, d = I.grid(32, 32)
    prep = O.prepare(n, s, d, 50)
    g, P, pos, eig = ssm.prepare(n, s, d, 50, precision=64)
    assert np.array_equal(P.pivots.cpu().numpy(), prep.pivots)
    assert np.array_equal(P.dip.cpu().numpy(), prep.dip)
    assert _norm_err(pos.cpu().numpy(), prep.pos0) < 1e-9
    ssm.ssm_iterate(g, P, pos, 200)
    opos, _ = O.iterate(prep, prep.pos0, 200)
    assert _norm_err(pos.cpu().numpy(), opos) < 1e-8
    out, _ = ssm.ssm_stress(g, pos)
    np.testing.assert_allclose(out.cpu().numpy(), O.full_stress(prep.g, opos), rtol=1e-8)


# ------------------------------------------------------------------ hints: no host wait in the sweep

@pytest.mark.parametrize("name,k", [("rgg", 100), ("ba", 64), ("messy", 95), ("path", 7)])
def test_iterate_hints_from_the_synchronous_calls(name, k):
    """The largest distance from ssm_aggregate_size and the row classes from
    ssm_build_graph equal what ssm_iterate_hints computes, and the sweep
    gives the same bits with and without them."""
    n, s, d = GRAPHS[name]()
    g, P, pos, _ = ssm.prepare(n, s, d, k)
    assert P.dmax is not None and g.row_classes is not None
    assert ssm.ssm_iterate_hints(g, P.dip) == (P.dmax, g.row_classes[0], g.row_classes[1])
    deg = np.diff(g.rowptr.cpu().numpy())
    assert g.row_classes == (int(((deg > 32) & (deg <= 1024)).sum()), int((deg > 1024).sum()))
    assert P.dmax == int(P.dip.cpu().numpy().max())
    a, b = pos.clone(), pos.clone()
    ssm.ssm_iterate(g, P, a, 3)
    cfg_a = ssm.ssm_last_sweep_config()
    P0 = ssm.Pivots(P.k, P.pivots, P.dip, P.region, P.cnt_off, P.cnt)  # no hints: computed inside
    ssm.ssm_iterate(g, P0, b, 3)
    assert ssm.ssm_last_sweep_config() == cfg_a
    assert torch.equal(a, b)


def test_iterate_with_hints_returns_before_the_stream_drains():
    """With hints the FP32 call only enqueues: it returns while a half-second
    kernel queued before it still runs; without hints it waits once."""
    import time

    n, s, d = GRAPHS["rgg"]()
    g, P, pos, _ = ssm.prepare(n, s, d, 50)
    ssm.ssm_iterate(g, P, pos.clone(), 1)  # first-use costs outside the timing
    torch.cuda.synchronize()
    cycles = 1_000_000_000  # about half a second at the GB300's 2 GHz SM clock
    torch.cuda._sleep(cycles)
    t0 = time.perf_counter()
    ssm.ssm_iterate(g, P, pos.clone(), 1, check=False)
    with_hints = time.perf_counter() - t0
    torch.cuda.synchronize()
    P0 = ssm.Pivots(P.k, P.pivots, P.dip, P.region, P.cnt_off, P.cnt)
    torch.cuda._sleep(cycles)
    t0 = time.perf_counter()
    ssm.ssm_iterate(g, P0, pos.clone(), 1, check=False)
    without = time.perf_counter() - t0
    torch.cuda.synchronize()
    assert with_hints < 0.2 < without


def test_iterate_rejects_a_dmax_hint_below_the_largest_distance():
    """A largest-distance hint below the true one would send table reads past
    the table: the tiled copy clamps them and the call fails with
    SSM_E_ARG instead."""
    n, s, d = GRAPHS["ba"]()
    g, P, pos, _ = ssm.prepare(n, s, d, 64)
    assert P.dmax >= 4
    bad = ssm.Pivots(P.k, P.pivots, P.dip, P.region, P.cnt_off, P.cnt, P.dmax - 2)
    with pytest.raises(ssm.SSMError) as e:
        ssm.ssm_iterate(g, bad, pos.clone(), 1)
    assert e.value.code == -1
    # the context stays usable
    ssm.ssm_iterate(g, P, pos, 1)
