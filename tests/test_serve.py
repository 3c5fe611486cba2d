"""The continuous-batching layout server: admission under an HBM budget and a
slot count, arrival order, error paths and latency statistics on the host
(fake job runner, no GPU); on the GPU, that every request's result is the same
alone and in the mix."""
import random
import threading
import time

import numpy as np
import pytest

from paper_1608_08909_gb300 import serve as S


class _Probe:
    """Fake runner: holds each job for a short random time and records how many
    bytes and jobs were on the 'device' at once."""

    def __init__(self, seed=0):
        self.lock = threading.Lock()
        self.bytes = 0
        self.jobs = 0
        self.peak_bytes = 0
        self.peak_jobs = 0
        self.rng = random.Random(seed)

    def __call__(self, job, stream):
        with self.lock:
            self.bytes += job.n
            self.jobs += 1
            self.peak_bytes = max(self.peak_bytes, self.bytes)
            self.peak_jobs = max(self.peak_jobs, self.jobs)
            d = self.rng.uniform(0.0005, 0.004)
        time.sleep(d)
        with self.lock:
            self.bytes -= job.n
            self.jobs -= 1
        return S.LayoutResult(pos=np.zeros((job.n, 2), np.float32), eig=np.zeros(2), stress=None, device_bytes=0)


def _jobs(sizes):
    return [S.LayoutJob(n=int(s), src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), tag=i)
            for i, s in enumerate(sizes)]


@pytest.mark.parametrize("budget,slots", [(100, 8), (60, 3), (1000, 2)])
def test_budget_slots_and_arrival_order(budget, slots):
    rng = np.random.default_rng(budget + slots)
    jobs = _jobs(rng.integers(5, 60, size=80))
    probe = _Probe(slots)
    with S.LayoutServer(budget, slots=slots, runner=probe, sizer=lambda j: j.n) as srv:
        futs = [srv.submit(j) for j in jobs]
        res = [f.result(timeout=30) for f in futs]
        assert srv.reserved == 0
        order = list(srv.admit_order)
        assert srv.peak_reserved <= budget
        assert srv.peak_active <= slots
    assert len(res) == len(jobs)
    assert probe.peak_bytes <= budget and probe.peak_jobs <= slots
    assert order == [j.tag for j in jobs]  # admitted strictly in arrival order
    assert all(r.t_arrival <= r.t_admit <= r.t_done for r in res)


def test_waits_are_attributed_to_the_budget_or_the_slots():
    # budget-bound: 8 slots, but two 40-byte requests never fit a 60-byte budget together
    with S.LayoutServer(60, slots=8, runner=_Probe(2), sizer=lambda j: j.n) as srv:
        [f.result(timeout=30) for f in [srv.submit(j) for j in _jobs([40] * 20)]]
        assert srv.waited_for_budget > 0 and srv.waited_for_slot == 0
    # slot-bound: the budget holds everything, one slot
    with S.LayoutServer(10_000, slots=1, runner=_Probe(3), sizer=lambda j: j.n) as srv:
        [f.result(timeout=30) for f in [srv.submit(j) for j in _jobs([40] * 20)]]
        assert srv.waited_for_slot > 0 and srv.waited_for_budget == 0


def test_requests_run_concurrently_when_they_fit():
    probe = _Probe(1)
    with S.LayoutServer(10_000, slots=4, runner=probe, sizer=lambda j: j.n) as srv:
        res = [f.result(timeout=30) for f in [srv.submit(j) for j in _jobs([10] * 40)]]
    assert len(res) == 40 and probe.peak_jobs > 1


def test_oversized_request_is_rejected_and_others_still_run():
    probe = _Probe(2)
    with S.LayoutServer(50, slots=2, runner=probe, sizer=lambda j: j.n) as srv:
        big, small = srv.submit(_jobs([51])[0]), srv.submit(_jobs([20])[0])
        with pytest.raises(MemoryError):
            big.result(timeout=30)
        assert small.result(timeout=30).pos.shape == (20, 2)


def test_runner_failure_reaches_the_future_and_frees_the_budget():
    def boom(job, stream):
        if job.tag == 1:
            raise RuntimeError("device status 7")
        return S.LayoutResult(pos=np.zeros((job.n, 2), np.float32), eig=np.zeros(2), stress=None, device_bytes=0)

    with S.LayoutServer(30, slots=1, runner=boom, sizer=lambda j: j.n) as srv:
        futs = [srv.submit(j) for j in _jobs([30, 30, 30])]
        assert futs[0].result(timeout=30).pos.shape == (30, 2)
        with pytest.raises(RuntimeError, match="status 7"):
            futs[1].result(timeout=30)
        assert futs[2].result(timeout=30).pos.shape == (30, 2)
        assert srv.reserved == 0


def test_latency_percentiles_and_open_loop_replay():
    rs = [S.LayoutResult(np.zeros((1, 2)), np.zeros(2), None, 0, t_arrival=0.0, t_done=float(x))
          for x in range(1, 101)]
    p = S.latency_percentiles(rs)
    assert p["p50"] == pytest.approx(50.5) and p["p99"] == pytest.approx(99.01)

    class Clock:
        t = 0.0

        def __call__(self):
            return self.t

        def sleep(self, d):
            self.t += d

    clk = Clock()
    seen = []

    class Rec:
        def submit(self, job, t_arrival=None):
            seen.append((clk(), t_arrival))
            return None

    gaps = [0.5, 1.0, 0.25, 2.0]
    S.replay(Rec(), _jobs([1, 1, 1, 1]), gaps, rate=2.0, clock=clk, sleep=clk.sleep)
    want = np.cumsum(gaps) / 2.0
    assert [a for _, a in seen] == pytest.approx(list(want))
    assert [t for t, _ in seen] == pytest.approx(list(want))


def test_job_device_bytes_covers_the_buffers():
    n, m, k = 20000, 60000, 100
    b = S.job_device_bytes(n, m, k)
    assert b >= 2 * k * n + 16 * m + 8 * n
    assert S.job_device_bytes(2 * n, 2 * m, k) > b


# ------------------------------------------------------------------ GPU

@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    from paper_1608_08909_gb300 import inputs as I

    reqs = I.request_stream(8, 5, n_min=1000, n_max=30000)
    jobs = []
    for i, r in enumerate(reqs):
        n, s, d = I.mixed_graph(r["family"], r["n"], r["seed"])
        jobs.append(S.LayoutJob(n=n, src=s, dst=d, k=50, iters=30, stress_sources=16, stress_targets=64,
                                seed=r["seed"], tag=i))
    with S.LayoutServer(120 << 30, slots=4) as srv:
        mixed = [f.result(timeout=600) for f in [srv.submit(j) for j in jobs]]
        assert srv.peak_active > 1
    alone = []
    with S.LayoutServer(120 << 30, slots=1) as srv:
        for j in jobs:
            alone.append(srv.submit(j).result(timeout=600))
    for a, b in zip(mixed, alone):
        assert np.array_equal(a.pos, b.pos)
        assert np.array_equal(a.eig, b.eig)
        assert np.array_equal(a.stress, b.stress)
        assert np.isfinite(a.pos).all()


@pytest.mark.gpu
def test_small_budget_serialises_admission():
    from paper_1608_08909_gb300 import inputs as I

    jobs = []
    for i, fam in enumerate(["grid", "btree", "rgg", "grid", "rgg"]):
        n, s, d = I.mixed_graph(fam, 6000 + 500 * i, 100 + i)
        jobs.append(S.LayoutJob(n=n, src=s, dst=d, k=40, iters=10, tag=i))
    needs = [S.job_device_bytes(j.n, len(j.src), j.k) for j in jobs]
    budget = max(needs) + 1
    assert 2 * min(needs) > budget  # no two requests fit together
    with S.LayoutServer(budget, slots=4) as srv:
        res = [f.result(timeout=600) for f in [srv.submit(j) for j in jobs]]
        assert srv.peak_reserved <= budget
        assert srv.peak_active == 1
    assert all(np.isfinite(r.pos).all() for r in res)


@pytest.mark.gpu
@pytest.mark.parametrize("family,n0,stress", [("grid", 9000, 0), ("rgg", 30000, 32), ("btree", 20000, 0)])
def test_job_device_bytes_bounds_the_allocation(family, n0, stress):
    """What admission charges is at least what one request really allocates:
    the rise of torch's peak allocated bytes over a whole request stays
    within job_device_bytes."""
    import torch

    from paper_1608_08909_gb300 import inputs as I

    n, s, d = I.mixed_graph(family, n0, 7)
    job = S.LayoutJob(n=n, src=s, dst=d, k=100, iters=5, stress_sources=stress, stress_targets=64 if stress else 0)
    stream = torch.cuda.Stream()
    S.run_layout_job(job, stream)  # library load and first-use costs
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    S.run_layout_job(job, stream)
    torch.cuda.synchronize()
    rise = torch.cuda.max_memory_allocated() - base
    bound = S.job_device_bytes(n, len(s), job.k, job.stress_sources, job.stress_targets)
    assert 0 < rise <= bound
