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


class TrimBackend(FakeBackend):
    def __init__(self):
        super().__init__()
        self.trims = []

    def trim_slot(self, slot):
        self.trims.append(slot)


def test_slot_workspace_is_counted_until_trimmed():
    """A slot's context keeps the workspace of its largest solve: the server
    counts it after the request finishes, and frees idle slots' workspace
    when the head of the queue would not fit otherwise."""
    be = TrimBackend()
    big = serve.Request(0, _sys(120), solver="gmres", m=40)
    small = [serve.Request(i, _sys(40), solver="gmres", m=20, arrival=0.0) for i in range(1, 6)]
    own_b, ws_b = serve.footprint_parts(big)
    own_s, ws_s = serve.footprint_parts(small[0])
    # room for the big request's retained workspace plus one small request at
    # a time in a second slot, but not for two retained big workspaces
    budget = own_b + serve.retained_workspace(ws_b) + own_s + serve.retained_workspace(ws_s) + 1
    srv = serve.Server(be, slots=2, budget_bytes=budget, small_n=0)
    res = srv.run([big] + small, realtime=False)
    assert all(r.status == 0 for r in res)
    assert srv.peak_in_use <= budget
    assert srv.in_use == 0
    # the slots still hold their workspaces after the run; their sum is what
    # the resident count reports
    assert srv.resident() == sum(srv.slot_ws) > 0


def test_trim_frees_idle_slots_for_a_request_that_needs_the_room():
    be = TrimBackend()
    a = serve.Request(0, _sys(100), solver="gmres", m=30)
    b = serve.Request(1, _sys(100), solver="gmres", m=30, arrival=0.0)
    own, ws = serve.footprint_parts(a)
    budget = own + serve.retained_workspace(ws) + own // 2  # one retained workspace at a time
    srv = serve.Server(be, slots=2, budget_bytes=budget, small_n=0)
    res = srv.run([a, b], realtime=False)
    assert all(r.status == 0 for r in res)
    assert srv.peak_in_use <= budget
    # the second request went to the slot that already held the workspace,
    # or an idle slot was trimmed to make room
    assert sum(1 for w in srv.slot_ws if w > 0) == 1 or be.trims


def test_summary_counts_converged_solves_only():
    mk = lambda rid, conv, t: serve.Result(rid, None, {"conv": conv}, 0, "slot", 0.0, 0.0, t)
    res = [mk(0, 0, 1.0), mk(1, 0, 2.0), mk(2, 1, 4.0), mk(3, 0, 3.0)]
    s = serve.summarize(res)
    assert s["completed"] == 4 and s["converged"] == 3 and s["latency_samples"] == 3
    assert abs(s["solves_per_s"] - 3 / 4.0) < 1e-12
    assert abs(s["completed_per_s"] - 4 / 4.0) < 1e-12
    assert s["p99_s"] <= 3.0 < s["p99_completed_s"]
