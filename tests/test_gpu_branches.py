"""Kernel variants that the everyday workloads do not reach, each against the
oracle through the C ABI:

* the grid-wide push bitset BFS (k_msbfs), taken when a graph has more nodes
  than the per-source BFS's shared-memory visited bitmap holds (1,638,400);
* the FP32 sweep with its clamped s table in global memory and the FP64 sweep
  with its counts in global memory, taken when the tables pass 200 KB of
  shared memory (a long path: regions of thousands of hops);
* coincident positions (r = 0, observed by the paper's weakness analysis in
  Section 4): a term whose points coincide adds w x_j only, in every sweep
  form (FP32 full table, FP32 clamped table, FP64, batched).

ssm_last_sweep_config() reports which sweep kernel ran, so each test checks
that it reached the variant it is named for.
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"
THREADS = max(1, min(16, os.cpu_count() or 1))


def _gpu_graph(n, s, d):
    return ssm.ssm_build_graph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV))


def _norm_err(a, b):
    b = np.asarray(b, np.float64)
    c = b - b.mean(0)
    return np.sqrt(((np.asarray(a, np.float64) - b) ** 2).sum(1)).max() / np.sqrt((c ** 2).sum(1).mean())


def _gpu_pivots(k, prep):
    return ssm.Pivots(k, torch.from_numpy(prep.pivots).to(DEV), torch.from_numpy(prep.dip).to(DEV),
                      torch.from_numpy(prep.region).to(DEV),
                      torch.from_numpy(prep.cnt_off.astype(np.int32)).to(DEV), torch.from_numpy(prep.cnt).to(DEV))


# ------------------------------------------------------------------ push bitset BFS above the bitmap limit

@pytest.mark.parametrize("family,k", [("grid", 3), ("ba", 40)])
def test_pivot_bfs_above_bitmap_limit(family, k):
    """n above 1,638,400: d_ip and the max/min pivots through the cooperative
    kernels (k_msbfs for the distances), bit-exact; the grid has 2,600 BFS
    levels, the BA graph few levels of up to a million nodes."""
    if family == "grid":
        n, s, d = I.grid(1300, 1300)
    else:
        n, s, d = I.ba(1700000, 4, 5)
    assert n > 1638400
    og = O.build_csr(n, s, d)
    g = _gpu_graph(n, s, d)
    piv = ssm.ssm_select_pivots(g, k, 0)
    assert ssm.ssm_last_pivot_config() == {"cluster": 0, "mind_bytes": 4}
    opiv = O.maxmin(og, k, 0)
    assert np.array_equal(piv.cpu().numpy(), opiv)
    dip = ssm.ssm_pivot_bfs(g, piv).cpu().numpy()
    assert np.array_equal(dip, O.pivot_dist_threads(og, opiv, THREADS))


# ------------------------------------------------------------------ tables in global memory

@pytest.fixture(scope="module")
def long_path():
    """A 60000-node path with 6 max/min pivots; its PivotMDS layout is exactly
    collinear and already a fixed point of the sweep, so the sweeps start from
    it with seeded noise added (a relative change well above FP32 rounding)."""
    n, s, d = I.path(60000)
    prep = O.prepare(n, s, d, 6)
    assert prep.dip.max() <= 65534
    x0 = prep.pos0 + np.random.default_rng(12).normal(scale=200.0, size=prep.pos0.shape)
    return n, s, d, prep, x0


def test_sweep_fp32_clamped_table_in_global_memory(long_path):
    n, s, d, prep, start = long_path
    k = len(prep.pivots)
    assert (2 * len(prep.cnt) + k) * 4 + k * 24 > 200 * 1024
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(k, prep)
    x0 = start.astype(np.float32)
    pos = torch.from_numpy(x0.copy()).to(DEV)
    _, rel = ssm.ssm_iterate(g, P, pos, 1)
    assert ssm.ssm_last_sweep_config()["kernel"] == "f32_clamped_global"
    want, orel = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, x0.astype(np.float64))
    assert _norm_err(pos.cpu().numpy(), want) < 1e-5
    assert rel.item() == pytest.approx(orel, rel=1e-4)


def test_sweep_fp64_counts_in_global_memory(long_path):
    n, s, d, prep, start = long_path
    k = len(prep.pivots)
    assert k * 24 + len(prep.cnt) * 8 > 200 * 1024
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(k, prep)
    pos = torch.from_numpy(start.copy()).to(DEV)
    _, rel = ssm.ssm_iterate(g, P, pos, 5)
    assert ssm.ssm_last_sweep_config()["kernel"] == "f64_counts_global"
    want, orel = O.iterate(prep, start, 5)
    assert np.array_equal(pos.cpu().numpy(), want)
    assert rel.item() == pytest.approx(orel, rel=1e-12)


# ------------------------------------------------------------------ coincident positions

def _coincident_state(prep, rng, count):
    """The PivotMDS start rounded to FP32 with `count` nodes moved onto a pivot
    and `count` nodes moved onto one of their neighbours (exact copies, so
    r = 0 in both precisions)."""
    x = prep.pos0.astype(np.float32).copy()
    g = prep.g
    n = g.n
    nodes = rng.choice(n, 2 * count, replace=False)
    for i in nodes[:count]:
        x[i] = x[prep.pivots[rng.integers(0, len(prep.pivots))]]
    for i in nodes[count:]:
        nb = g.colidx[g.rowptr[i]:g.rowptr[i + 1]]
        x[i] = x[nb[rng.integers(0, len(nb))]]
    return x


@pytest.mark.parametrize("name,k,kernel", [("grid32", 50, "f32_full_table"), ("rgg", 100, "f32_clamped_smem"),
                                           ("ba", 40, "f32_full_table")])
def test_sweep_coincident_positions(name, k, kernel):
    n, s, d = {"grid32": lambda: I.grid(32, 32), "rgg": lambda: I.rgg(6000, 8.0, 7),
               "ba": lambda: I.ba(12000, 4, 3)}[name]()
    prep = O.prepare(n, s, d, k)
    x0 = _coincident_state(prep, np.random.default_rng(3), 40)
    # the state really has coincident pivot and edge terms
    piv_pos = x0[prep.pivots]
    assert any((x0[i] == piv_pos).all(1).any() for i in range(n) if i not in set(prep.pivots.tolist()))
    g = _gpu_graph(n, s, d)
    P = _gpu_pivots(k, prep)
    want, orel = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, x0.astype(np.float64))
    assert np.isfinite(want).all()
    # FP32
    pos = torch.from_numpy(x0.copy()).to(DEV)
    _, rel = ssm.ssm_iterate(g, P, pos, 1)
    assert ssm.ssm_last_sweep_config()["kernel"] == kernel
    assert _norm_err(pos.cpu().numpy(), want) < 1e-5
    # FP64: bit for bit
    pos = torch.from_numpy(x0.astype(np.float64)).to(DEV)
    ssm.ssm_iterate(g, P, pos, 1)
    assert np.array_equal(pos.cpu().numpy(), want)
    # batched sweep
    pos = torch.from_numpy(x0.copy()).to(DEV)
    ssm.ssm_batch_iterate([(g, P, pos)], 1)
    assert _norm_err(pos.cpu().numpy(), want) < 1e-5
