"""Layout quality measures of Section 4 on the GPU against the oracle:
the Procrustes statistic (FP64 sums in another order: 1e-12) and the
convex-hull error of Fig. 4 (counts from the same FP64 orientation tests:
every per-node error and the mean bit-exact) and the Gabriel-graph Jaccard
comparison (the same FP64 disc predicate: bit-exact)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1608_08909_gb300 as ssm
from paper_1608_08909_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda"


def test_procrustes_matches_oracle():
    rng = np.random.default_rng(5)
    for n in (1, 2, 37, 1000, 20011):
        X = rng.normal(size=(n, 2)) * 3 + 1
        th = 0.4
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        Y = 1.7 * X @ R.T + rng.normal(scale=0.2, size=(n, 2))
        want = np.array(O.procrustes(X, Y))
        got = ssm.ssm_procrustes(torch.from_numpy(X).to(DEV), torch.from_numpy(Y).to(DEV)).cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12)
        got32 = ssm.ssm_procrustes(torch.from_numpy(X.astype(np.float32)).to(DEV),
                                   torch.from_numpy(Y.astype(np.float32)).to(DEV)).cpu().numpy()
        want32 = np.array(O.procrustes(X.astype(np.float32), Y.astype(np.float32)))
        np.testing.assert_allclose(got32, want32, rtol=1e-10, atol=1e-12)


def _layouts():
    out = {}
    n, s, d = I.rgg(600, 7.0, 3)
    g = O.build_csr(n, s, d)
    D = O.apsp(g)
    x, _ = O.pivotmds(D[:40])
    out["rgg_pmds"] = (D, O.rescale(g, x))
    n, s, d = I.grid(20, 24)
    D = O.apsp(O.build_csr(n, s, d))
    r, c = np.divmod(np.arange(n), 24)
    out["grid_integer"] = (D, np.stack([c, r], 1).astype(np.float64))  # collinear and cocircular points
    n, s, d = I.complete_btree(8)
    g = O.build_csr(n, s, d)
    D = O.apsp(g)
    x, _ = O.pivotmds(D[:30])
    out["btree"] = (D, x)
    return out


LAYOUTS = _layouts()


@pytest.mark.parametrize("name", list(LAYOUTS))
@pytest.mark.parametrize("kh", [1, 2, 4])
def test_hull_error_bit_exact(name, kh):
    D, x = LAYOUTS[name]
    want_mean, want = O.hull_error(D, x, kh)
    for prec in (64, 32):
        xx = x if prec == 64 else x.astype(np.float32)
        if prec == 32:
            want_mean, want = O.hull_error(D, xx.astype(np.float64), kh)
        mean, per = ssm.ssm_hull_error(torch.from_numpy(D).to(DEV), torch.from_numpy(xx).to(DEV), kh)
        assert np.array_equal(per.cpu().numpy(), want)
        assert mean.item() == want_mean


def test_hull_error_large_balls_are_thinned():
    """Balls of more than 4096 nodes: points strictly inside the quadrilateral
    of the ball's extreme points are dropped before the sort."""
    n, s, d = I.rgg(6000, 8.0, 7)
    g = O.build_csr(n, s, d)
    D = O.apsp(g)
    x, _ = O.pivotmds(D[:30])
    kh = int(np.median(D[0])) + 10
    assert (D <= kh).sum(1).max() > 4096
    want_mean, want = O.hull_error(D, x, kh)
    mean, per = ssm.ssm_hull_error(torch.from_numpy(D).to(DEV), torch.from_numpy(x).to(DEV), kh)
    assert np.array_equal(per.cpu().numpy(), want)
    assert mean.item() == want_mean


def _gabriel_pairs():
    rng = np.random.default_rng(11)
    out = {}
    D, x = LAYOUTS["rgg_pmds"]
    out["rgg_pmds_vs_noisy"] = (x, x + rng.normal(scale=0.3, size=x.shape))
    D, x = LAYOUTS["grid_integer"]
    out["grid_vs_sheared"] = (x, x + np.stack([0.5 * x[:, 1], np.zeros(len(x))], 1))
    D, x = LAYOUTS["btree"]  # siblings of the unsampled leaves coincide
    out["btree_vs_rotated"] = (x, x @ np.array([[0.0, -1.0], [1.0, 0.0]]) + rng.normal(scale=1e-3, size=x.shape))
    u = rng.uniform(size=(1500, 2)) * 40.0
    out["uniform1500_vs_noisy"] = (u, u + rng.normal(scale=0.5, size=u.shape))
    u = rng.uniform(size=(6000, 2)) * 80.0
    out["uniform6000_vs_noisy"] = (u, u + rng.normal(scale=0.5, size=u.shape))
    c = rng.normal(size=(700, 2))
    c[::7] = c[1::7][: len(c[::7])]  # coincident pairs
    out["gauss_coincident"] = (c, c[::-1].copy())
    return out


GABRIEL_PAIRS = _gabriel_pairs()


@pytest.mark.parametrize("name", list(GABRIEL_PAIRS))
@pytest.mark.parametrize("kh", [1, 2, 3])
def test_gabriel_jaccard_bit_exact(name, kh):
    A, B = GABRIEL_PAIRS[name]
    for prec in (64, 32):
        if prec == 32:
            A, B = A.astype(np.float32), B.astype(np.float32)
        want_mean, want = O.gabriel_jaccard(A.astype(np.float64), B.astype(np.float64), kh)
        mean, per = ssm.ssm_gabriel_jaccard(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), kh)
        assert np.array_equal(per.cpu().numpy(), want)
        assert mean.item() == want_mean


def test_gabriel_jaccard_identical_layouts_and_tiny():
    x = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 0.1], [0.0, 0.0]])
    mean, per = ssm.ssm_gabriel_jaccard(torch.from_numpy(x).to(DEV), torch.from_numpy(x).to(DEV), 2)
    assert np.array_equal(per.cpu().numpy(), np.ones(4)) and mean.item() == 1.0
    one = np.zeros((1, 2))
    mean, per = ssm.ssm_gabriel_jaccard(torch.from_numpy(one).to(DEV), torch.from_numpy(one).to(DEV), 1)
    assert per.item() == 1.0  # both neighbourhoods empty
    want_mean, want = O.gabriel_jaccard(x, x[[3, 2, 1, 0]], 1)
    mean, per = ssm.ssm_gabriel_jaccard(torch.from_numpy(x).to(DEV), torch.from_numpy(x[[3, 2, 1, 0]]).to(DEV), 1)
    assert np.array_equal(per.cpu().numpy(), want) and mean.item() == want_mean
