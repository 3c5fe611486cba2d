"""Batched sweeps (ssm_batch_iterate) against the FP64 oracle, graph by graph:
one Jacobi step of Eq. 4 from the same FP32 start at several points of the
oracle's trajectory, on a batch of mixed small graphs (grids, random binary
trees, RGGs; odd and even n, a single-tile graph, k from 1 to 100)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _norm_err(a, b):
    b = np.asarray(b, np.float64)
    c = b - b.mean(0)
    rms = np.sqrt((c ** 2).sum(1).mean())
    return np.sqrt(((np.asarray(a, np.float64) - b) ** 2).sum(1)).max() / rms


def _batch():
    specs = [("grid", 64, 1), ("btree", 97, 2), ("rgg", 300, 3), ("grid", 1023, 4), ("btree", 2049, 5),
             ("rgg", 3001, 6), ("grid", 4096, 7), ("btree", 555, 8), ("rgg", 1200, 9), ("grid", 130, 10)]
    out = []
    for fam, n0, seed in specs:
        n, s, d = I.mixed_graph(fam, n0, seed)
        k = max(1, min(100, n // 4))
        prep = O.prepare(n, s, d, k)
        g = ssm.ssm_build_graph(n, torch.from_numpy(s).to(DEV), torch.from_numpy(d).to(DEV))
        P = ssm.Pivots(k, torch.from_numpy(prep.pivots).to(DEV), torch.from_numpy(prep.dip).to(DEV),
                       torch.from_numpy(prep.region).to(DEV), torch.from_numpy(prep.cnt_off.astype(np.int32)).to(DEV),
                       torch.from_numpy(prep.cnt).to(DEV))
        out.append((prep, g, P))
    return out


@pytest.fixture(scope="module")
def batch():
    return _batch()


def test_batch_step_matches_oracle(batch):
    xs = [prep.pos0 for prep, _, _ in batch]
    for t in range(4):
        items = [(g, P, torch.from_numpy(x.astype(np.float32)).to(DEV)) for x, (_, g, P) in zip(xs, batch)]
        rel, used = ssm.ssm_batch_iterate(items, 1)
        assert used[0] in (128, 256, 512) and used[1] in (2, 4)
        rel = rel.cpu().numpy()
        nxt = []
        for i, ((prep, _, _), (_, _, pos)) in enumerate(zip(batch, items)):
            x32 = xs[i].astype(np.float32).astype(np.float64)
            want, wrel = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, x32)
            assert _norm_err(pos.cpu().numpy(), want) < 1e-5, (i, t)
            assert rel[i] == pytest.approx(wrel, rel=1e-4, abs=1e-9)
            x, _ = O.sweep_jacobi(prep.g, prep.pivots, prep.dip, prep.w, xs[i])
            nxt.append(x)
        xs = nxt


def test_batch_shapes_agree_bit_for_bit(batch):
    """Every block size and both tile shapes (64-node tiles with two nodes per
    lane, 128-node tiles with four) give the same positions bit for bit: a
    node's terms are added in the same order whatever the shape; the relative
    change adds a lane's nodes in FP32 before the FP64 tile sums, so it agrees
    bit for bit within a tile shape and to FP32 rounding across them."""
    res = {}
    for npl in (2, 4):
        for threads in (128, 256, 512):
            items = [(g, P, torch.from_numpy(prep.pos0.astype(np.float32)).to(DEV)) for prep, g, P in batch]
            rel, used = ssm.ssm_batch_iterate(items, 7, threads=threads, nodes_per_lane=npl)
            assert used == (threads, npl)
            res[(threads, npl)] = ([p.cpu().numpy() for _, _, p in items], rel.cpu().numpy())
    ref_pos, ref_rel = res[(128, 2)]
    for (threads, npl), (pos, rel) in res.items():
        assert all(np.array_equal(a, b) for a, b in zip(pos, ref_pos)), (threads, npl)
        if npl == 2:
            assert np.array_equal(rel, ref_rel)
        else:
            np.testing.assert_allclose(rel, ref_rel, rtol=1e-6)
            assert np.array_equal(rel, res[(128, 4)][1])


def test_batch_tuned_shape_is_kept(batch):
    """The first call with threads = nodes_per_lane = 0 tunes; a second call on
    a batch of the same shape takes the kept choice."""
    items = [(g, P, torch.from_numpy(prep.pos0.astype(np.float32)).to(DEV)) for prep, g, P in batch]
    _, first = ssm.ssm_batch_iterate(items, 3)
    items = [(g, P, torch.from_numpy(prep.pos0.astype(np.float32)).to(DEV)) for prep, g, P in batch]
    _, again = ssm.ssm_batch_iterate(items, 3)
    assert first == again


def test_batch_many_iterations_finite_and_converging(batch):
    items = [(g, P, torch.from_numpy(prep.pos0.astype(np.float32)).to(DEV)) for prep, g, P in batch]
    rel, _ = ssm.ssm_batch_iterate(items, 150)
    rel = rel.cpu().numpy()
    assert all(np.isfinite(p.cpu().numpy()).all() for _, _, p in items)
    assert (rel < 0.05).all()
