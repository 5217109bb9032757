"""Continuous-batching solve server on one GPU.

Requests (a sparse system plus solver choice) arrive over time.  The server
admits a request when its HBM footprint fits the budget next to the requests
already on the GPU, and runs it in one of two lanes:

* slot lane: large systems and every GMRES request.  Each slot owns a library
  context (its own workspace and cached graphs) and a CUDA stream; a worker
  thread per slot copies the request to the device, applies GS(p), runs the
  whole solve as one graph launch and copies x back.  The C calls release the
  Python interpreter lock, so the slots' solves overlap on the device.
* batch lane: small Bi-CGSTAB systems.  A worker collects the admitted small
  requests that are waiting and solves them together with one launch of the
  batched persistent kernel; requests that arrive while a batch is running
  join the next launch (continuous batching at launch granularity).

A request's result does not depend on what else is running: a slot solve uses
its own workspace and the same kernels and launch geometry as a solve alone,
and a batched system is solved by one thread block with a fixed reduction
order.  The device-resident part of every solve (Krylov vectors, scalars,
iteration control) never leaves the GPU until x is copied back.

The GPU work goes through `GpuBackend`; the scheduling logic can run against
any object with the same two methods (the tests use a fake one on the CPU).
"""
from __future__ import annotations

import math
import threading
import time
from collections import deque
from dataclasses import dataclass

import numpy as np


@dataclass
class Request:
    rid: int
    system: object  # host CSR system (problems.cd.System)
    solver: str = "bicgstab"  # "bicgstab" or "gmres"
    m: int = 30
    p: float = 2.0
    tol: float = 1e-8
    precision: str = "mixed"  # "mixed" or "f64"
    arrival: float = 0.0  # seconds after the run starts
    maxit: int = 10000


@dataclass
class Result:
    rid: int
    x: np.ndarray | None
    info: dict
    status: int
    lane: str
    t_arrival: float
    t_admit: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def footprint_parts(req: Request, workspace_fn=None) -> tuple[int, int]:
    """(bytes of the request's own arrays: CSR, b and x; bytes of solver
    workspace it needs)."""
    s = req.system
    n, nnz = s.n, int(s.rowptr[-1])
    own = 4 * (n + 1) + 12 * nnz + 16 * n
    if workspace_fn is not None:
        ws = workspace_fn(n, nnz, req.solver, req.m, req.precision)
    else:
        vec = 4 if req.precision == "mixed" else 8
        ws = (vec * n * (req.m + 2) if req.solver == "gmres" else 8 * vec * n) + 24 * n + 4 * nnz + (1 << 20)
    return own, ws


def footprint_bytes(req: Request, workspace_fn=None) -> int:
    """Device bytes a request holds while it runs: its CSR, b and x, and the
    solver workspace."""
    own, ws = footprint_parts(req, workspace_fn)
    return own + ws


def retained_workspace(ws: int) -> int:
    """What a library context holds after a solve that needed ws bytes of
    workspace: it grows its workspace to ws + ws/8 + 1 MiB and keeps it."""
    return ws + ws // 8 + (1 << 20)


class GpuBackend:
    """Runs requests through the library's C ABI on one device."""

    def __init__(self, device: int = 0, slots: int = 4):
        import torch

        import paper_0812_2769_gb300 as g

        self.g = g
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        self.ctxs = [g.Context(device) for _ in range(slots)]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.bctx = g.Context(device)
        self.bstream = torch.cuda.Stream(device=device)

    def trim_slot(self, slot: int):
        """Free an idle slot's workspace (a new, empty context)."""
        self.ctxs[slot].close()
        self.ctxs[slot] = self.g.Context(self.device)

    def workspace(self, n, nnz, solver, m, precision):
        g = self.g
        return g.workspace_bytes(n, nnz, solver, m, g.PREC_MIXED if precision == "mixed" else g.PREC_F64)

    def _opts(self, req):
        g = self.g
        return g.opts(precision=g.PREC_MIXED if req.precision == "mixed" else g.PREC_F64, maxit=req.maxit)

    def run_single(self, slot: int, req: Request):
        g, torch = self.g, self.torch
        s = req.system
        st = self.streams[slot]
        ctx = self.ctxs[slot]
        with torch.cuda.stream(st):
            A = g.Csr.from_host(s.rowptr, s.colidx, s.val, device=f"cuda:{self.device}")
            b = torch.as_tensor(s.b, device=f"cuda:{self.device}")
            x = torch.zeros(s.n, dtype=torch.float64, device=f"cuda:{self.device}")
            try:
                g.gs_scale(A, b, p=req.p, ctx=ctx, stream=st)
                if req.solver == "gmres":
                    info = g.gmres_solve(A, b, x, m=req.m, tol=req.tol, options=self._opts(req), ctx=ctx, stream=st)
                else:
                    info = g.bicgstab_solve(A, b, x, tol=req.tol, options=self._opts(req), ctx=ctx, stream=st)
                status = g.OK
            except g.GskError as e:
                info, status = {}, e.status
            xh = x.cpu().numpy()
            st.synchronize()
        return xh, info, status

    def run_batch(self, reqs: list[Request]):
        g, torch = self.g, self.torch
        dev = f"cuda:{self.device}"
        st = self.bstream
        with torch.cuda.stream(st):
            As = [g.Csr.from_host(r.system.rowptr, r.system.colidx, r.system.val, device=dev) for r in reqs]
            bs = [torch.as_tensor(r.system.b, device=dev) for r in reqs]
            xs = [torch.zeros(r.system.n, dtype=torch.float64, device=dev) for r in reqs]
            prec = reqs[0].precision
            o = g.opts(precision=g.PREC_MIXED if prec == "mixed" else g.PREC_F64, maxit=reqs[0].maxit)
            infos, stats = g.bicgstab_solve_batched(As, bs, xs, p=[r.p for r in reqs], tol=reqs[0].tol, options=o,
                                                    ctx=self.bctx, stream=st, check=False)
            out = [(x.cpu().numpy(), i, s_) for x, i, s_ in zip(xs, infos, stats)]
            st.synchronize()
        return out


class Server:
    """Admission by HBM footprint, a slot lane and a continuous batch lane.

    Device memory is accounted as the library holds it: a request's own arrays
    (CSR, b, x) while it runs; for the slot lane, each slot's context keeps
    the workspace its largest solve so far needed (a context grows its
    workspace and does not shrink it), so a request is assigned a slot at
    admission and counted by how much it would grow that slot's workspace;
    the batch lane's requests count their workspace while they run.  When the
    head of the queue does not fit, the workspaces of idle slots are freed
    first (the backend's trim_slot, if it has one)."""

    def __init__(self, backend, slots: int = 4, budget_bytes: int | None = None, small_n: int = 65536,
                 batch_max: int = 256):
        self.backend = backend
        self.nslots = slots
        if budget_bytes is None:
            import torch

            free, _ = torch.cuda.mem_get_info()
            budget_bytes = int(0.8 * free)
        self.budget = budget_bytes
        self.small_n = small_n
        self.batch_max = batch_max
        self.lock = threading.Condition()
        self.pending: deque = deque()  # arrived, not yet admitted (FIFO)
        self.slot_q = [deque() for _ in range(slots)]  # admitted, assigned to a slot
        self.batch_q: deque = deque()  # admitted, waiting for the next batch launch
        self.in_use = 0  # running requests' arrays, and the batch lane's workspace
        self.slot_ws = [0] * slots  # workspace each slot's context holds
        self.slot_busy = [False] * slots
        self.peak_in_use = 0
        self.free_slots = slots
        self.batch_busy = False
        self.results: dict[int, Result] = {}
        self.t0 = 0.0
        self.done = False
        self.workspace_fn = getattr(backend, "workspace", None)

    def lane_of(self, req: Request) -> str:
        return "batch" if (req.solver == "bicgstab" and req.system.n <= self.small_n) else "slot"

    def _now(self):
        return time.perf_counter() - self.t0

    def resident(self) -> int:
        """Device bytes the server's requests and slot contexts hold now."""
        return self.in_use + sum(self.slot_ws)

    # -------- admission (called with the lock held)
    def _pick_slot(self, need: int):
        """The idle slot a request needing `need` bytes of workspace grows the
        least, and by how much."""
        best, grow = None, None
        for k in range(self.nslots):
            if self.slot_busy[k]:
                continue
            g = max(0, retained_workspace(need) - self.slot_ws[k]) if need > self.slot_ws[k] else 0
            if grow is None or g < grow:
                best, grow = k, g
        return best, grow

    def _trim_idle(self, keep: int | None) -> bool:
        trim = getattr(self.backend, "trim_slot", None)
        freed = False
        for k in range(self.nslots):
            if k != keep and not self.slot_busy[k] and self.slot_ws[k] > 0:
                if trim is not None:
                    trim(k)
                self.slot_ws[k] = 0
                freed = True
        return freed

    def _admit(self):
        while self.pending:
            req, t_arr = self.pending[0]
            own, ws = footprint_parts(req, self.workspace_fn)
            lane = self.lane_of(req)
            total = own + (retained_workspace(ws) if lane == "slot" else ws)
            if total > self.budget:  # can never fit: reject
                self.pending.popleft()
                self.results[req.rid] = Result(req.rid, None, {}, -1, "rejected", t_arr, self._now(), self._now())
                continue
            if lane == "slot":
                if self.free_slots == 0:
                    break
                k, grow = self._pick_slot(ws)
                if self.resident() + own + grow > self.budget:
                    if self._trim_idle(keep=k):
                        continue  # try again with the idle slots' workspaces freed
                    break  # FIFO: wait for memory to free up
                self.pending.popleft()
                self.in_use += own
                if ws > self.slot_ws[k]:
                    self.slot_ws[k] = retained_workspace(ws)
                self.slot_busy[k] = True
                self.free_slots -= 1
                self.slot_q[k].append((req, t_arr, self._now(), own))
            else:
                if self.resident() + own + ws > self.budget:
                    if self._trim_idle(keep=None):
                        continue
                    break
                self.pending.popleft()
                self.in_use += own + ws
                self.batch_q.append((req, t_arr, self._now(), own + ws))
            self.peak_in_use = max(self.peak_in_use, self.resident())
            self.lock.notify_all()

    def _finish(self, req, t_arr, t_adm, fp, x, info, status, lane, slot=None):
        with self.lock:
            self.results[req.rid] = Result(req.rid, x, info, status, lane, t_arr, t_adm, self._now())
            self.in_use -= fp
            if lane == "slot":
                self.free_slots += 1
                self.slot_busy[slot] = False
            self._admit()
            self.lock.notify_all()

    def _slot_worker(self, slot: int):
        q = self.slot_q[slot]
        while True:
            with self.lock:
                while not q and not self.done:
                    self.lock.wait(0.05)
                if not q:
                    return
                req, t_arr, t_adm, fp = q.popleft()
            x, info, status = self.backend.run_single(slot, req)
            self._finish(req, t_arr, t_adm, fp, x, info, status, "slot", slot)

    def _batch_worker(self):
        while True:
            with self.lock:
                while not self.batch_q and not self.done:
                    self.lock.wait(0.05)
                if not self.batch_q:
                    return
                group = []
                while self.batch_q and len(group) < self.batch_max:
                    group.append(self.batch_q.popleft())
            # one launch per precision/tolerance class
            classes: dict = {}
            for item in group:
                classes.setdefault((item[0].precision, item[0].tol, item[0].maxit), []).append(item)
            for items in classes.values():
                outs = self.backend.run_batch([it[0] for it in items])
                for (req, t_arr, t_adm, fp), (x, info, status) in zip(items, outs):
                    self._finish(req, t_arr, t_adm, fp, x, info, status, "batch")

    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Feed the requests at their arrival times (or all at once) and
        return the results in request order."""
        self.t0 = time.perf_counter()
        self.done = False
        workers = [threading.Thread(target=self._slot_worker, args=(k,), daemon=True) for k in range(self.nslots)]
        workers.append(threading.Thread(target=self._batch_worker, daemon=True))
        for w in workers:
            w.start()
        for req in sorted(requests, key=lambda r: r.arrival):
            if realtime:
                delay = req.arrival - self._now()
                if delay > 0:
                    time.sleep(delay)
            with self.lock:
                self.pending.append((req, self._now()))
                self._admit()
        with self.lock:
            while len(self.results) < len(requests):
                self.lock.wait(0.05)
            self.done = True
            self.lock.notify_all()
        for w in workers:
            w.join()
        return [self.results[r.rid] for r in requests]


def summarize(results: list[Result]) -> dict:
    """Throughput and latency of a run.  The headline counts only the solves
    that converged (reached tol): solves that stopped at maxit finished
    without the accuracy asked for and are reported apart.  Percentiles come
    with their sample size (p99 of n < 100 samples is an order statistic near
    the maximum)."""
    done = [r for r in results if r.status == 0]
    conv = [r for r in done if r.info.get("conv") == 0]
    span = (max(r.t_done for r in results) - min(r.t_arrival for r in results)) if results else math.nan

    def pct(rs, q):
        return float(np.percentile([r.latency for r in rs], q)) if rs else math.nan

    return {"requests": len(results), "completed": len(done), "converged": len(conv),
            "solves_per_s": len(conv) / span if span > 0 else math.nan,
            "p50_s": pct(conv, 50), "p99_s": pct(conv, 99), "latency_samples": len(conv),
            "completed_per_s": len(done) / span if span > 0 else math.nan,
            "p50_completed_s": pct(done, 50), "p99_completed_s": pct(done, 99),
            "lanes": {ln: sum(1 for r in results if r.lane == ln) for ln in ("slot", "batch", "rejected")}}
