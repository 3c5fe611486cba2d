"""Continuous-batching layout server on one GPU.

Layout requests (an edge list, k, iteration count) arrive at any time.  The
server admits them in arrival order as soon as a slot is free and the
request's device memory fits the HBM budget next to the requests already on
the GPU; each admitted request runs the whole pipeline of Algorithm 1
(graph, max/min pivots, d_ip, regions and counts, PivotMDS, the Jacobi
sweeps of Eq. 4, optionally the sampled stress) on its own CUDA stream, so
the kernels of different requests overlap on the device while every request
keeps its CSR, d_ip and positions resident until it finishes.  Results do not
depend on what else is running: each request has its own buffers, and every
reduction of the library runs in a fixed order.

``job_device_bytes`` bounds the device memory a request allocates at its
peak (the library's own workspace queries plus its buffers, with a margin for
the allocator's rounding of small tensors), which is what admission charges
against the budget.  The budget counts allocated bytes: blocks that torch's
caching allocator keeps after a request frees them are outside it.  The scheduler itself is host logic
that takes the job runner as a parameter, so it is tested without a GPU.
"""
from __future__ import annotations

import collections
import concurrent.futures
import threading
import time
from dataclasses import dataclass, field

import numpy as np

_MB = 1 << 20


@dataclass
class LayoutJob:
    """One layout request: a graph on nodes 0..n-1 given by its host edge list."""
    n: int
    src: np.ndarray
    dst: np.ndarray
    k: int = 100
    iters: int = 100
    start: int = 0
    stress_sources: int = 0    # sampled stress (Eq. 1) with this many BFS sources; 0: none
    stress_targets: int = 0
    seed: int = 0
    tag: object = None


@dataclass
class LayoutResult:
    pos: np.ndarray            # [n, 2] float32 final positions
    eig: np.ndarray            # the two PivotMDS eigenvalues
    stress: np.ndarray | None  # {raw, alpha*, scaled, normalized} if asked
    device_bytes: int          # what admission charged for the request
    t_arrival: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def job_device_bytes(n: int, m_in: int, k: int, stress_sources: int = 0, stress_targets: int = 0) -> int:
    """An upper bound of the device bytes a request allocates at its peak: the
    edge list, CSR, pivots, d_ip, regions and counts, positions and the
    largest stage workspace (the count table is bounded by n + k entries,
    since ecc_a + 1 <= |R(a)|), plus 1 MB for the allocator's rounding of the
    small status and result tensors."""
    from . import lib

    L = lib()
    k = min(k, n)
    cnt_len = n + k
    persist = (8 * m_in                     # src, dst
               + 4 * (n + 1) + 8 * m_in     # rowptr, colidx (capacity 2 m_in)
               + 4 * k + 2 * k * n          # pivots, d_ip
               + 4 * n + 4 * (k + 1) + 4 * cnt_len  # region, cnt_off, cnt
               + 8 * n + 64)                # positions, eigenvalues
    ws = max(L.ssm_build_graph_workspace(n, m_in), L.ssm_select_pivots_workspace(n, m_in),
             L.ssm_pivot_bfs_workspace(n, m_in, k), L.ssm_aggregate_workspace(k),
             L.ssm_pivotmds_workspace(n, k), L.ssm_iterate_workspace(n, m_in, k, cnt_len, 32),
             L.ssm_stress_workspace(n, m_in, stress_sources, stress_targets) if stress_sources > 0 else 0)
    return int(persist + ws + _MB)


def run_layout_job(job: LayoutJob, stream, device="cuda") -> LayoutResult:
    """The whole pipeline for one request on `stream` (blocks the calling thread)."""
    import torch

    from . import (Pivots, ssm_aggregate, ssm_aggregate_size, ssm_build_graph, ssm_iterate, ssm_pivot_bfs, ssm_pivotmds,
                   ssm_select_pivots, ssm_stress)

    k = min(job.k, job.n)
    with torch.cuda.stream(stream):
        src = torch.from_numpy(np.ascontiguousarray(job.src, dtype=np.int32)).to(device, non_blocking=True)
        dst = torch.from_numpy(np.ascontiguousarray(job.dst, dtype=np.int32)).to(device, non_blocking=True)
        g = ssm_build_graph(job.n, src, dst, stream)
        del src, dst
        piv = ssm_select_pivots(g, k, job.start, stream)
        dip = ssm_pivot_bfs(g, piv, stream)
        cnt_len, dmax = ssm_aggregate_size(dip, stream, with_dmax=True)
        region, off, cnt = ssm_aggregate(dip, cnt_len, stream=stream)
        pos, eig = ssm_pivotmds(g, dip, 32, True, stream)
        ssm_iterate(g, Pivots(k, piv, dip, region, off, cnt, dmax), pos, job.iters, stream=stream)
        stress = None
        if job.stress_sources > 0:
            out, _ = ssm_stress(g, pos, job.stress_sources, job.stress_targets, job.seed, stream)
            stress = out.cpu().numpy()
        pos_h = pos.cpu().numpy()
        eig_h = eig.cpu().numpy()[:2]
    return LayoutResult(pos=pos_h, eig=eig_h, stress=stress, device_bytes=0)


class LayoutServer:
    """Admits requests in arrival order under an HBM budget and a slot count and
    runs each on its own stream; ``submit`` returns a future of LayoutResult."""

    def __init__(self, hbm_budget: int, slots: int = 8, device="cuda", runner=None, sizer=None,
                 clock=time.perf_counter):
        if slots < 1 or hbm_budget <= 0:
            raise ValueError("need slots >= 1 and a positive budget")
        self.budget = int(hbm_budget)
        self.slots = slots
        self.device = device
        self._clock = clock
        self._runner = runner if runner is not None else (lambda job, stream: run_layout_job(job, stream, device))
        self._sizer = sizer if sizer is not None else (
            lambda job: job_device_bytes(job.n, len(job.src), job.k, job.stress_sources, job.stress_targets))
        if runner is None:
            import torch
            self._streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        else:
            self._streams = [None] * slots
        self._free = list(range(slots))
        self._queue: collections.deque = collections.deque()
        self._cv = threading.Condition()
        self._reserved = 0
        self._active = 0
        self._closed = False
        self.peak_reserved = 0
        self.peak_active = 0
        # requests that reached the head of the queue and had to wait: for
        # bytes (a slot was free but the budget was not) or for a slot
        self.waited_for_budget = 0
        self.waited_for_slot = 0
        self._head_seen = None
        self.admit_order: list = []
        self._pool = concurrent.futures.ThreadPoolExecutor(max_workers=slots, thread_name_prefix="ssm-slot")
        self._thread = threading.Thread(target=self._dispatch, name="ssm-dispatch", daemon=True)
        self._thread.start()

    # ------------------------------------------------------------------ API
    def submit(self, job: LayoutJob, t_arrival: float | None = None) -> concurrent.futures.Future:
        fut: concurrent.futures.Future = concurrent.futures.Future()
        need = int(self._sizer(job))
        t = self._clock() if t_arrival is None else t_arrival
        with self._cv:
            if self._closed:
                raise RuntimeError("server is closed")
            if need > self.budget:
                fut.set_exception(MemoryError(f"request needs {need} bytes, budget is {self.budget}"))
                return fut
            self._queue.append((job, fut, need, t))
            self._cv.notify_all()
        return fut

    def close(self, wait: bool = True):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        self._thread.join()
        self._pool.shutdown(wait=wait)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def reserved(self) -> int:
        with self._cv:
            return self._reserved

    # ------------------------------------------------------------ internals
    def _dispatch(self):
        while True:
            with self._cv:
                while True:
                    if self._queue:
                        job, fut, need, t = self._queue[0]
                        if self._free and self._reserved + need <= self.budget:
                            break
                        if self._head_seen is not fut:
                            self._head_seen = fut
                            if self._free:
                                self.waited_for_budget += 1
                            else:
                                self.waited_for_slot += 1
                    elif self._closed:
                        return
                    self._cv.wait()
                self._queue.popleft()
                slot = self._free.pop()
                self._reserved += need
                self._active += 1
                self.peak_reserved = max(self.peak_reserved, self._reserved)
                self.peak_active = max(self.peak_active, self._active)
                self.admit_order.append(job.tag)
                t_admit = self._clock()
            self._pool.submit(self._work, job, fut, need, t, t_admit, slot)

    def _work(self, job, fut, need, t_arrival, t_admit, slot):
        try:
            res = self._runner(job, self._streams[slot])
            res.device_bytes = need
            res.t_arrival, res.t_admit, res.t_done = t_arrival, t_admit, self._clock()
            fut.set_result(res)
        except BaseException as e:  # surfaced through the future
            fut.set_exception(e)
        finally:
            with self._cv:
                self._reserved -= need
                self._active -= 1
                self._free.append(slot)
                self._cv.notify_all()


def latency_percentiles(results, qs=(50, 99)) -> dict:
    """p50 / p99 (seconds) of arrival-to-result latencies."""
    lat = np.array([r.latency for r in results], dtype=np.float64)
    return {f"p{q}": float(np.percentile(lat, q)) for q in qs} if lat.size else {f"p{q}": None for q in qs}


def replay(server: LayoutServer, jobs, gaps, rate: float, clock=time.perf_counter, sleep=time.sleep):
    """Open-loop replay: request j arrives gaps[0] + ... + gaps[j] (unit-rate
    exponential gaps) divided by `rate` seconds after the start and is
    submitted then; returns the futures in arrival order."""
    t0 = clock()
    futs = []
    t = 0.0
    for job, gap in zip(jobs, gaps):
        t += gap / rate
        wait = t0 + t - clock()
        if wait > 0:
            sleep(wait)
        futs.append(server.submit(job, t_arrival=t0 + t))
    return futs
