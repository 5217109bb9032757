"""Scheduling logic of the solve server on the CPU (a fake backend stands in
for the GPU): admission by footprint, lanes, FIFO order, completion."""
import threading
import time

import numpy as np

from paper_0812_2769_gb300 import serve
from problems import cd


def _sys(n_side):
    return cd.build(n_side, 2, cd.Constant(1.0), [cd.Constant(0.0)] * 2)


class FakeBackend:
    def __init__(self):
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.batches = []

    def _enter(self):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)

    def _leave(self):
        with self.lock:
            self.active -= 1

    def run_single(self, slot, req):
        self._enter()
        time.sleep(0.002 + req.system.n * 2e-7)
        self._leave()
        return np.full(req.system.n, float(req.rid)), {"conv": 0, "iters": 1}, 0

    def run_batch(self, reqs):
        self._enter()
        self.batches.append([r.rid for r in reqs])
        time.sleep(0.003)
        self._leave()
        return [(np.full(r.system.n, float(r.rid)), {"conv": 0, "iters": 1}, 0) for r in reqs]


def _requests(k, seed=0):
    rs = np.random.default_rng(seed)
    out = []
    for i in range(k):
        side = int(rs.integers(8, 64))
        solver = "gmres" if rs.uniform() < 0.4 else "bicgstab"
        out.append(serve.Request(i, _sys(side), solver=solver, m=20, arrival=float(i) * 0.001))
    return out


def test_every_request_completes_with_its_own_result():
    be = FakeBackend()
    srv = serve.Server(be, slots=3, budget_bytes=1 << 40, small_n=1000)
    reqs = _requests(40)
    res = srv.run(reqs, realtime=True)
    assert [r.rid for r in res] == [q.rid for q in reqs]
    for q, r in zip(reqs, res):
        assert r.status == 0 and np.all(r.x == q.rid)
        assert r.lane == ("batch" if q.solver == "bicgstab" and q.system.n <= 1000 else "slot")
        assert r.t_done >= r.t_admit >= r.t_arrival
    s = serve.summarize(res)
    assert s["completed"] == 40 and s["p99_s"] >= s["p50_s"] > 0


def test_budget_is_never_exceeded_and_slots_are_bounded():
    be = FakeBackend()
    reqs = _requests(60, seed=1)
    fps = [serve.footprint_bytes(q) for q in reqs]
    budget = int(2.5 * max(fps))
    srv = serve.Server(be, slots=4, budget_bytes=budget, small_n=1000)
    res = srv.run(reqs, realtime=False)
    assert all(r.status == 0 for r in res)
    assert srv.peak_in_use <= budget
    assert srv.in_use == 0 and srv.free_slots == 4
    assert be.max_active <= 4 + 1  # slot workers plus the batch lane


def test_oversized_request_is_rejected_not_stalled():
    be = FakeBackend()
    reqs = _requests(5)
    big = serve.Request(99, _sys(200), solver="gmres")
    srv = serve.Server(be, slots=2, budget_bytes=serve.footprint_bytes(big) - 1, small_n=1000)
    res = srv.run(reqs + [big], realtime=False)
    assert res[-1].lane == "rejected" and res[-1].status == -1
    assert all(r.status == 0 for r in res[:-1])


def test_requests_arriving_during_a_batch_join_a_later_launch():
    be = FakeBackend()
    reqs = [serve.Request(i, _sys(10), solver="bicgstab", arrival=0.002 * i) for i in range(30)]
    srv = serve.Server(be, slots=1, budget_bytes=1 << 40, small_n=1000, batch_max=64)
    srv.run(reqs, realtime=True)
    assert len(be.batches) > 1  # continuous: several launches, not one queue drained at the end
    assert sorted(sum(be.batches, [])) == list(range(30))
    assert any(len(b) > 1 for b in be.batches)  # and arrivals were grouped
