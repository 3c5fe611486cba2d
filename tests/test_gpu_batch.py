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
        assert used in (128, 256, 512)
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


def test_batch_block_sizes_agree_bit_for_bit(batch):
    res = []
    for threads in (128, 256, 512):
        items = [(g, P, torch.from_numpy(prep.pos0.astype(np.float32)).to(DEV)) for prep, g, P in batch]
        rel, used = ssm.ssm_batch_iterate(items, 7, threads=threads)
        assert used == threads
        res.append(([p.cpu().numpy() for _, _, p in items], rel.cpu().numpy()))
    for pos, rel in res[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(pos, res[0][0]))
        assert np.array_equal(rel, res[0][1])


def test_batch_many_iterations_finite_and_converging(batch):
    items = [(g, P, torch.from_numpy(prep.pos0.astype(np.float32)).to(DEV)) for prep, g, P in batch]
    rel, _ = ssm.ssm_batch_iterate(items, 150)
    rel = rel.cpu().numpy()
    assert all(np.isfinite(p.cpu().numpy()).all() for _, _, p in items)
    assert (rel < 0.05).all()
