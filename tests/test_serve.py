"""Admission logic of the serving loop (CPU, fake solves): every request is
served once, in arrival order, never more solves in flight than slots, never
more reserved device memory than the budget, oversized requests rejected."""
import threading
import time

import pytest

from paper_2504_02117_gb300 import serve


def _requests(k, spread):
    out = []
    for i in range(k):
        n = (8, 12, 16)[i % 3]
        out.append(serve.SlabRequest(rid=i, arrival=spread * i, dims=(n, n, n), s=(2, 4, 8)[i % 3],
                                     precision=("fp32", "fp64")[i % 2]))
    return out


def _fake(record, dur=0.03):
    lock = threading.Lock()
    live = {"n": 0}

    def solve(slot, r):
        with lock:
            live["n"] += 1
            record.append(live["n"])
        time.sleep(dur)
        with lock:
            live["n"] -= 1
        return {"status": 0, "outer": 1, "inner": 1}
    return solve


def test_all_served_in_arrival_order_within_slots():
    seen = []
    srv = serve.SlabServer(slots=3, hbm_budget=1 << 40, solve=_fake(seen))
    reqs = _requests(20, 0.002)
    summ = srv.run(reqs)
    assert summ["completed"] == 20 and summ["rejected"] == 0 and summ["failed"] == 0
    assert max(seen) <= 3 and summ["max_concurrent"] == 3       # they overlapped
    adm = [r.admitted for r in sorted(reqs, key=lambda r: r.arrival)]
    assert adm == sorted(adm)                                     # FIFO admission
    for r in reqs:
        assert r.arrival <= r.admitted <= r.finished and r.slot in (0, 1, 2)
    assert summ["p99_latency_s"] >= summ["p50_latency_s"] > 0.0


def test_memory_budget_limits_concurrency():
    reqs = _requests(12, 0.0)
    need = max(serve.estimate_bytes(r.cells, r.s, r.precision) for r in reqs)
    budget = int(2.2 * need)                     # at most two of the largest at a time
    seen = []
    srv = serve.SlabServer(slots=8, hbm_budget=budget, solve=_fake(seen))
    summ = srv.run(reqs)
    assert summ["completed"] == 12 and summ["peak_reserved_bytes"] <= budget
    # reserved memory of the requests in flight at each admission stays in budget
    for r in reqs:
        live = [q for q in reqs if q.admitted <= r.admitted < q.finished]
        assert sum(serve.estimate_bytes(q.cells, q.s, q.precision) for q in live) <= budget


def test_oversized_request_is_rejected_not_queued():
    reqs = _requests(4, 0.0)
    big = serve.SlabRequest(rid=99, arrival=0.0, dims=(512, 512, 512), s=16)
    srv = serve.SlabServer(slots=2, hbm_budget=1 << 30, solve=_fake([]))
    summ = srv.run(reqs + [big])
    assert summ["rejected"] == 1 and big.status == -2 and big.finished is None
    assert summ["completed"] == 4


def test_failing_solve_does_not_stop_the_server():
    def solve(slot, r):
        if r.rid == 1:
            raise RuntimeError("planted failure")
        return {"status": 0}
    reqs = _requests(5, 0.0)
    summ = serve.SlabServer(slots=2, hbm_budget=1 << 40, solve=solve).run(reqs)
    assert summ["completed"] == 4 and summ["failed"] == 1
    assert reqs[1].error.startswith("planted")


def _lane_requests(k, spread):
    out = []
    for i in range(k):
        small = i % 3 != 2
        n = 8 if small else 40
        out.append(serve.SlabRequest(rid=i, arrival=spread * i, dims=(n, n, n), s=4,
                                     precision="fp64" if i % 4 != 3 else "fp32"))
    return out


def test_batch_lane_takes_small_fp64_requests_in_batches():
    """Small float64 requests need no slot: each is solved exactly once by the
    lane, several per launch when they queue up while a batch runs; the rest
    go through the slots; FIFO admission and the memory budget still hold."""
    calls, lock = [], threading.Lock()

    def solve_batch(rs):
        with lock:
            calls.append([r.rid for r in rs])
        time.sleep(0.05)
        return [{"status": 0, "outer": 1, "inner": 3} for _ in rs]

    reqs = _lane_requests(30, 0.004)
    srv = serve.SlabServer(slots=2, hbm_budget=1 << 40, solve=_fake([], 0.02), batch_lane=True,
                           batch_max_unknowns=8 ** 3 * 4, solve_batch=solve_batch)
    summ = srv.run(reqs)
    assert summ["completed"] == 30 and summ["failed"] == 0
    lane = [r for r in reqs if srv.batchable(r)]
    assert lane and all(r.slot == "batch" for r in lane)
    assert all(r.slot in (0, 1) for r in reqs if not srv.batchable(r))
    solved = sorted(x for c in calls for x in c)
    assert solved == sorted(r.rid for r in lane)                 # each exactly once
    assert summ["batch_launches"] == len(calls) < len(lane)      # batched
    assert summ["max_batch"] >= 2
    adm = [r.admitted for r in sorted(reqs, key=lambda r: r.arrival)]
    assert adm == sorted(adm)
    # a lane request is never larger than the threshold or float32
    assert all(r.cells * r.s <= 8 ** 3 * 4 and r.precision == "fp64" for r in lane)


def test_batch_lane_failure_marks_its_requests_and_the_server_goes_on():
    def solve_batch(rs):
        raise RuntimeError("planted batch failure")
    reqs = _lane_requests(9, 0.0)
    srv = serve.SlabServer(slots=2, hbm_budget=1 << 40, solve=_fake([], 0.01), batch_lane=True,
                           batch_max_unknowns=8 ** 3 * 4, solve_batch=solve_batch)
    summ = srv.run(reqs)
    lane = [r for r in reqs if srv.batchable(r)]
    assert summ["failed"] == len(lane) and summ["completed"] == 9 - len(lane)
    assert all(r.status == -1 and "planted" in r.error for r in lane)


def test_batch_lane_respects_the_memory_budget():
    reqs = _lane_requests(12, 0.0)
    srv0 = serve.SlabServer(slots=4, hbm_budget=1 << 40, solve=_fake([]), batch_lane=True,
                            batch_max_unknowns=8 ** 3 * 4, solve_batch=lambda rs: [{}] * len(rs))
    need = max(srv0.need_bytes(r) for r in reqs)
    budget = int(2.5 * need)

    def solve_batch(rs):
        time.sleep(0.02)
        return [{"status": 0} for _ in rs]
    srv = serve.SlabServer(slots=4, hbm_budget=budget, solve=_fake([], 0.02), batch_lane=True,
                           batch_max_unknowns=8 ** 3 * 4, solve_batch=solve_batch)
    summ = srv.run(reqs)
    assert summ["completed"] == 12 and summ["peak_reserved_bytes"] <= budget
