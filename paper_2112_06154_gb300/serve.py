"""Continuous-batching server for sampled (k,h)-core decompositions.

Requests (a graph as CSR, its h, and the sampling parameters) arrive at any
time.  A request is admitted as soon as a worker slot is free and its
device-memory footprint fits in the budget next to the requests already on
the GPU; each slot owns a library context with its own CUDA stream, so the
admitted requests' kernels overlap on the device.  Requests are admitted in
arrival order; one that can never fit the budget is rejected at submission.
A queued request can be cancelled (Future.cancel) or carry a deadline: one
still waiting when its deadline passes fails with TimeoutError and is never
started.  A started request runs to completion.

Every result is the deterministic function of (graph, h, seed, M) that
kh_core_sampled computes, so a request returns the same core numbers alone
or in any mix.  The execution step is a plain function (`runner`), which lets
host-side tests drive the admission logic without a GPU.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np


def budget_M(n: int, eps: float, delta: float) -> int:
    """M of Eq. (buffer) as the library computes it (kh_footprint)."""
    from . import khcore as K
    return K.kh_footprint(n, 0, 1, 0, eps, delta)[0]


def footprint_bytes(n: int, nnz: int, h: int, M: int) -> int:
    """The library's upper bound of the device bytes a sampled decomposition of
    this graph allocates (kh_footprint)."""
    from . import khcore as K
    return K.kh_footprint(n, nnz, h, M)[1]


@dataclass
class Request:
    rid: int
    rowptr: np.ndarray
    col: np.ndarray
    h: int
    seed: int = 1
    M: int = 0
    eps: float = 0.5
    delta: float = 0.05
    arrival: float = field(default_factory=time.perf_counter)
    footprint: int = 0
    future: Future = field(default_factory=Future)
    admitted: float = 0.0
    finished: float = 0.0
    deadline: float | None = None  # perf_counter time by which it must start


def gpu_runner(device: int = 0):
    """A runner factory: each worker thread gets its own context (own stream)."""
    from . import khcore as K

    K.load()

    def make():
        ctx = K.kh_ctx_create(device)

        def run(req: Request):
            G = K.kh_graph_load_csr(ctx, req.rowptr, req.col)
            try:
                K.kh_set_h(G, req.h)
                K.kh_set_sampling(G, seed=req.seed, M=req.M, eps=req.eps, delta=req.delta)
                core = K.kh_core_sampled(G)
                _, rounds, updates = K.kh_peel_info(G, False)
                return {"core": core, "rounds": rounds, "updates": updates}
            finally:
                G.close()

        def close():
            ctx.close()

        return run, close

    return make


class KhServer:
    """slots: concurrent requests on the GPU; mem_budget: device bytes they may hold."""

    def __init__(self, runner_factory, slots: int = 4, mem_budget: int = 64 << 30):
        if slots < 1 or mem_budget < 1:
            raise ValueError("a server needs at least one slot and a positive memory budget")
        self.slots = slots
        self.mem_budget = mem_budget
        self.mem_in_use = 0
        self.peak_mem = 0
        self.peak_running = 0
        self.running = 0
        self.queue: deque[Request] = deque()
        self.cv = threading.Condition()
        self.closing = False
        self.next_id = 0
        self.done: list[Request] = []
        self.dropped = 0  # cancelled or past their deadline before admission
        self.workers = [threading.Thread(target=self._worker, args=(runner_factory,), daemon=True)
                        for _ in range(slots)]
        for w in self.workers:
            w.start()

    def submit(self, rowptr, col, h: int, seed: int = 1, M: int = 0, eps: float = 0.5,
               delta: float = 0.05, arrival: float | None = None,
               deadline: float | None = None) -> Future:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        n = int(rowptr.size - 1)
        Mv = M if M > 0 else budget_M(n, eps, delta)
        with self.cv:
            req = Request(self.next_id, rowptr, col, h, seed, M, eps, delta,
                          arrival if arrival is not None else time.perf_counter())
            req.deadline = deadline
            self.next_id += 1
            req.footprint = footprint_bytes(n, int(col.size), h, Mv)
            if req.footprint > self.mem_budget:
                req.future.set_exception(MemoryError(
                    f"request {req.rid} needs {req.footprint} bytes, budget is {self.mem_budget}"))
                return req.future
            self.queue.append(req)
            self.cv.notify_all()
        return req.future

    def _drop_expired(self):
        # cancelled heads leave; heads past their deadline fail without starting
        now = time.perf_counter()
        while self.queue:
            head = self.queue[0]
            if head.future.cancelled():
                self.queue.popleft()
                self.dropped += 1
            elif head.deadline is not None and now > head.deadline:
                self.queue.popleft()
                self.dropped += 1
                if head.future.set_running_or_notify_cancel():
                    head.future.set_exception(TimeoutError(
                        f"request {head.rid} not started before its deadline"))
            else:
                return

    def _admit(self) -> Request | None:
        # arrival order: the head is admitted when it fits
        self._drop_expired()
        if self.queue and self.mem_in_use + self.queue[0].footprint <= self.mem_budget:
            req = self.queue.popleft()
            if not req.future.set_running_or_notify_cancel():
                self.dropped += 1  # cancelled between the check and now
                return None
            self.mem_in_use += req.footprint
            self.running += 1
            self.peak_mem = max(self.peak_mem, self.mem_in_use)
            self.peak_running = max(self.peak_running, self.running)
            return req
        return None

    def _worker(self, runner_factory):
        run, close = runner_factory()
        try:
            while True:
                with self.cv:
                    req = self._admit()
                    while req is None:
                        if self.closing and not self.queue:
                            return
                        self.cv.wait(0.05)
                        req = self._admit()
                req.admitted = time.perf_counter()
                try:
                    result = run(req)
                    err = None
                except Exception as e:  # the request fails, the server goes on
                    result, err = None, e
                req.finished = time.perf_counter()
                with self.cv:
                    self.mem_in_use -= req.footprint
                    self.running -= 1
                    self.done.append(req)
                    self.cv.notify_all()
                if err is None:
                    req.future.set_result(result)
                else:
                    req.future.set_exception(err)
        finally:
            close()

    def close(self):
        with self.cv:
            self.closing = True
            self.cv.notify_all()
        for w in self.workers:
            w.join()

    def latency_stats(self):
        lat = np.array([r.finished - r.arrival for r in self.done if r.finished > 0])
        if lat.size == 0:
            return {}
        first = min(r.arrival for r in self.done)
        last = max(r.finished for r in self.done)
        return {"requests": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "throughput_rps": float(lat.size / (last - first)) if last > first else 0.0,
                "peak_concurrent": self.peak_running, "peak_mem_bytes": self.peak_mem}
