"""Host-side tests of the continuous-batching server (no GPU): admission by
slots and device-memory budget, arrival order, rejection of requests that
can never fit, and failure isolation, driven by a fake runner."""
import threading
import time

import numpy as np
import pytest

from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import serve as S
from tests.conftest import read_golden


def fake_factory(log, delay=0.01, fail_ids=()):
    lock = threading.Lock()

    def make():
        def run(req):
            with lock:
                log.append(("start", req.rid))
            time.sleep(delay)
            if req.rid in fail_ids:
                raise RuntimeError(f"request {req.rid} failed")
            with lock:
                log.append(("end", req.rid))
            return {"rid": req.rid, "n": int(req.rowptr.size - 1)}

        return run, lambda: None

    return make


def test_budget_M_matches_table1():
    for name, n, M in read_golden("table1_budget_M.txt"):
        assert S.budget_M(int(n), 0.5, 0.05) == int(M), name


def test_footprint_grows_with_size_and_h():
    assert S.footprint_bytes(1000, 8000, 2, 500) < S.footprint_bytes(2000, 8000, 2, 500)
    assert S.footprint_bytes(1000, 8000, 2, 500) < S.footprint_bytes(1000, 8000, 3, 500)
    # h = 1 keeps no level lists
    assert S.footprint_bytes(1000, 8000, 1, 500) < S.footprint_bytes(1000, 8000, 2, 500)


def test_admission_respects_slots_and_budget():
    g = gg.erdos_renyi(200, 800, 1)
    one = S.footprint_bytes(200, 1600, 3, S.budget_M(200, 0.5, 0.05))
    log = []
    srv = S.KhServer(fake_factory(log, delay=0.02), slots=4, mem_budget=2 * one + 10)
    futs = [srv.submit(*g, h=3) for _ in range(10)]
    for f in futs:
        f.result(timeout=10)
    srv.close()
    assert srv.peak_running <= 2          # the budget allows two at a time
    assert srv.peak_mem <= srv.mem_budget
    assert srv.mem_in_use == 0 and srv.running == 0


def test_arrival_order_with_one_slot():
    log = []
    srv = S.KhServer(fake_factory(log, delay=0.005), slots=1, mem_budget=1 << 40)
    rp, cl = gg.path(20)
    futs = [srv.submit(rp, cl, h=2) for _ in range(8)]
    assert [f.result(timeout=10)["rid"] for f in futs] == list(range(8))
    srv.close()
    starts = [rid for kind, rid in log if kind == "start"]
    assert starts == list(range(8))


def test_oversized_request_is_rejected_at_submission():
    srv = S.KhServer(fake_factory([]), slots=2, mem_budget=1 << 10)
    rp, cl = gg.grid(30, 30)
    f = srv.submit(rp, cl, h=4)
    with pytest.raises(MemoryError):
        f.result(timeout=1)
    srv.close()


def test_failed_request_does_not_stop_the_server():
    log = []
    srv = S.KhServer(fake_factory(log, fail_ids={2}), slots=2, mem_budget=1 << 40)
    rp, cl = gg.cycle(10)
    futs = [srv.submit(rp, cl, h=2) for _ in range(5)]
    for i, f in enumerate(futs):
        if i == 2:
            with pytest.raises(RuntimeError):
                f.result(timeout=10)
        else:
            assert f.result(timeout=10)["rid"] == i
    srv.close()
    st = srv.latency_stats()
    assert st["requests"] == 5 and st["p99_s"] >= st["p50_s"] >= 0


def test_cancelled_request_never_starts():
    log = []
    srv = S.KhServer(fake_factory(log, delay=0.05), slots=1, mem_budget=1 << 40)
    rp, cl = gg.path(30)
    futs = [srv.submit(rp, cl, h=2) for _ in range(4)]
    assert futs[2].cancel()  # still queued behind the first request
    assert [futs[q].result(timeout=10)["rid"] for q in (0, 1, 3)] == [0, 1, 3]
    srv.close()
    assert futs[2].cancelled()
    assert 2 not in [rid for kind, rid in log if kind == "start"]
    assert srv.dropped == 1 and srv.mem_in_use == 0 and srv.running == 0


def test_deadline_fails_a_request_that_waits_too_long():
    log = []
    srv = S.KhServer(fake_factory(log, delay=0.2), slots=1, mem_budget=1 << 40)
    rp, cl = gg.path(30)
    first = srv.submit(rp, cl, h=2)
    late = srv.submit(rp, cl, h=2, deadline=time.perf_counter() + 0.05)
    relaxed = srv.submit(rp, cl, h=2, deadline=time.perf_counter() + 60.0)
    with pytest.raises(TimeoutError):
        late.result(timeout=10)
    assert first.result(timeout=10)["rid"] == 0
    assert relaxed.result(timeout=10)["rid"] == 2
    srv.close()
    assert 1 not in [rid for kind, rid in log if kind == "start"]
    assert srv.dropped == 1


def test_concurrent_clients():
    # several client threads submit at once; every result reaches its caller
    log = []
    srv = S.KhServer(fake_factory(log, delay=0.002), slots=3, mem_budget=1 << 40)
    graphs = [gg.path(10 + k) for k in range(8)]
    results = {}
    lock = threading.Lock()

    def client(k):
        rp, cl = graphs[k]
        fs = [srv.submit(rp, cl, h=2) for _ in range(10)]
        got = [f.result(timeout=30)["n"] for f in fs]
        with lock:
            results[k] = got

    threads = [threading.Thread(target=client, args=(k,)) for k in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    srv.close()
    for k in range(8):
        assert results[k] == [10 + k] * 10
    assert len(srv.done) == 80 and srv.mem_in_use == 0 and srv.peak_running <= 3


def test_server_refuses_a_configuration_that_cannot_serve():
    with pytest.raises(ValueError):
        S.KhServer(fake_factory([]), slots=0)
    with pytest.raises(ValueError):
        S.KhServer(fake_factory([]), slots=2, mem_budget=0)
