"""Full stress majorization over all-pairs distances (Section 3, the update
before Eq. 4) and the sparse model in the paper's in-place order (Algorithm
1 lines 6-10), against the oracle through the C ABI:
  * all-pairs distances (ssm_pivot_bfs with every node a source): bit-exact;
  * full stress, Jacobi, FP64: bit-identical trajectories;
  * full stress, Jacobi, FP32: 1e-5 on positions after one step;
  * Gauss-Seidel, FP64 (full stress and the sparse model): 1e-11 after one
    sweep (the GPU adds a node's terms in a fixed tree instead of in order),
    and full stress decreasing sweep by sweep."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"

GRAPHS = {
    "grid32": lambda: I.grid(32, 32),
    "btree": lambda: I.complete_btree(9),
    "rgg": lambda: I.rgg(1500, 8.0, 5),
    "grid_ragged": lambda: I.grid(17, 45),
}


def _setup(name):
    n, s, d = GRAPHS[name]()
    og = O.build_csr(n, s, d)
    g = ssm.ssm_build_graph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV))
    return n, og, g


def _norm_err(a, b):
    b = np.asarray(b, np.float64)
    c = b - b.mean(0)
    return np.sqrt(((np.asarray(a, np.float64) - b) ** 2).sum(1)).max() / np.sqrt((c ** 2).sum(1).mean())


@pytest.mark.parametrize("name", list(GRAPHS))
def test_apsp_bit_exact(name):
    n, og, g = _setup(name)
    assert np.array_equal(ssm.ssm_apsp(g).cpu().numpy(), O.apsp(og))


@pytest.mark.parametrize("name", ["grid32", "btree", "rgg"])
def test_full_jacobi_fp64_bit_identical(name):
    n, og, g = _setup(name)
    D = O.apsp(og)
    x0, _ = O.pivotmds(D[: min(50, n)])
    x = O.rescale(og, x0)
    want, rel = x, 0.0
    for _ in range(5):
        want, rel = O.full_sweep(D, want, 0)
    pos = torch.from_numpy(x.copy()).to(DEV)
    got_rel = ssm.ssm_full_iterate(torch.from_numpy(D).to(DEV), pos, 5, order=0)
    assert np.array_equal(pos.cpu().numpy(), want)
    assert got_rel.item() == pytest.approx(rel, rel=1e-12)


@pytest.mark.parametrize("name", ["grid32", "btree", "rgg", "grid_ragged"])
def test_full_jacobi_fp32_one_step(name):
    """From a start with seeded noise added: the complete binary tree's
    PivotMDS layout is degenerate (its second axis is rounding noise, so many
    nodes lie within 1e-12 of each other), and FP32 keeps r^2 above 1e-24
    (r = 0 exactly adds w x_j, as the rule says; 0 < r < 1e-11 is not resolved
    in FP32)."""
    n, og, g = _setup(name)
    D = O.apsp(og)
    x0, _ = O.pivotmds(D[: min(50, n)])
    x = (O.rescale(og, x0) + np.random.default_rng(3).normal(scale=0.1, size=x0.shape)).astype(np.float32)
    want, rel = O.full_sweep(D, x.astype(np.float64), 0)
    pos = torch.from_numpy(x.copy()).to(DEV)
    got_rel = ssm.ssm_full_iterate(torch.from_numpy(D).to(DEV), pos, 1, order=0)
    assert _norm_err(pos.cpu().numpy(), want) < 1e-5
    assert got_rel.item() == pytest.approx(rel, rel=1e-4)


@pytest.mark.parametrize("name", ["grid32", "rgg"])
def test_full_gauss_seidel_fp64(name):
    n, og, g = _setup(name)
    D = O.apsp(og)
    x0, _ = O.pivotmds(D[: min(50, n)])
    x = O.rescale(og, x0)
    want, rel = O.full_sweep(D, x, 1)
    Dg = torch.from_numpy(D).to(DEV)
    pos = torch.from_numpy(x.copy()).to(DEV)
    got_rel = ssm.ssm_full_iterate(Dg, pos, 1, order=1)
    assert _norm_err(pos.cpu().numpy(), want) < 1e-11
    assert got_rel.item() == pytest.approx(rel, rel=1e-9)
    # full stress decreases sweep by sweep (node-at-a-time majorization)
    prev, _ = ssm.ssm_stress(g, pos)
    prev = prev[0].item()
    for _ in range(3):
        ssm.ssm_full_iterate(Dg, pos, 1, order=1)
        cur = ssm.ssm_stress(g, pos)[0][0].item()
        assert cur <= prev * (1 + 1e-12)
        prev = cur


@pytest.mark.parametrize("name,k", [("grid32", 50), ("rgg", 40), ("btree", 33)])
def test_sparse_gauss_seidel_fp64(name, k):
    n, og, g = _setup(name)
    n_, s, d = GRAPHS[name]()
    prep = O.prepare(n_, s, d, k)
    P = ssm.Pivots(k, torch.from_numpy(prep.pivots).to(DEV), torch.from_numpy(prep.dip).to(DEV),
                   torch.from_numpy(prep.region).to(DEV), torch.from_numpy(prep.cnt_off.astype(np.int32)).to(DEV),
                   torch.from_numpy(prep.cnt).to(DEV))
    want = O.sweep_gs(prep.g, prep.pivots, prep.dip, prep.w, prep.pos0)
    pos = torch.from_numpy(prep.pos0.copy()).to(DEV)
    ssm.ssm_iterate_gs(g, P, pos, 1)
    assert _norm_err(pos.cpu().numpy(), want) < 1e-11
    # two more sweeps: the trajectories stay together
    for _ in range(2):
        want = O.sweep_gs(prep.g, prep.pivots, prep.dip, prep.w, want)
    ssm.ssm_iterate_gs(g, P, pos, 2)
    assert _norm_err(pos.cpu().numpy(), want) < 1e-9


def test_full_iterate_rejects_disconnected_tables():
    n = 300
    D = np.ones((n, n), np.uint16)
    np.fill_diagonal(D, 0)
    D[5, 9] = D[9, 5] = 0xFFFF
    pos = torch.from_numpy(np.random.default_rng(0).normal(size=(n, 2))).to(DEV)
    with pytest.raises(ssm.SSMError) as e:
        ssm.ssm_full_iterate(torch.from_numpy(D).to(DEV), pos, 1, order=0)
    assert e.value.code == -3


# ------------------------------------------------------------------ the paper's region tie rule (Section 3)

TIE_GRAPHS = {
    "grid32": (lambda: I.grid(32, 32), 50),
    "grid_ragged": (lambda: I.grid(17, 45), 33),
    "path": (lambda: I.path(300), 7),
    "btree": (lambda: I.complete_btree(9), 40),
    "rgg": (lambda: I.rgg(6000, 8.0, 7), 100),
    "ba": (lambda: I.ba(20000, 4, 3), 64),
}


@pytest.mark.parametrize("name", list(TIE_GRAPHS))
def test_regions_smallest_and_counts_bit_exact(name):
    make, k = TIE_GRAPHS[name]
    n, s, d = make()
    og = O.build_csr(n, s, d)
    piv = O.maxmin(og, k, 0)
    dip = O.pivot_dist(og, piv)
    want = O.regions_smallest(dip)
    gd = torch.from_numpy(dip).to(DEV)
    reg = ssm.ssm_regions_smallest(gd)
    assert np.array_equal(reg.cpu().numpy(), want)
    ecc, off, cnt = O.histograms(dip, want)
    goff, gcnt = ssm.ssm_aggregate_regions(gd, reg)
    assert np.array_equal(goff.cpu().numpy().astype(np.int64), off)
    assert np.array_equal(gcnt.cpu().numpy(), cnt)


def test_sweep_with_the_paper_tie_rule():
    """One FP32 Jacobi step whose weights come from the smallest-partition
    regions, against the oracle's weights counted directly on those regions."""
    n, s, d = I.grid(32, 32)
    og = O.build_csr(n, s, d)
    k = 50
    piv = O.maxmin(og, k, 0)
    dip = O.pivot_dist(og, piv)
    reg = O.regions_smallest(dip)
    assert not np.array_equal(reg, O.regions(dip))  # the rules differ on this grid
    w = O.adapted_weights(dip, reg)
    x0, _ = O.pivotmds(dip)
    x0 = O.rescale(og, x0).astype(np.float32)
    want, _ = O.sweep_jacobi(og, piv, dip, w, x0.astype(np.float64))
    g = ssm.ssm_build_graph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV))
    gd = torch.from_numpy(dip).to(DEV)
    greg = ssm.ssm_regions_smallest(gd)
    off, cnt = ssm.ssm_aggregate_regions(gd, greg)
    P = ssm.Pivots(k, torch.from_numpy(piv).to(DEV), gd, greg, off, cnt)
    pos = torch.from_numpy(x0.copy()).to(DEV)
    ssm.ssm_iterate(g, P, pos, 1)
    assert _norm_err(pos.cpu().numpy(), want) < 1e-5
