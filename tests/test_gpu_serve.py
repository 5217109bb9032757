"""The solve server on the GPU: requests of several sizes, solvers and
scalings arrive while others run; each result equals the same request solved
alone (bit for bit: a solve's arithmetic does not depend on what runs beside
it), and every converged result meets the FP64 metric (recomputed by the
oracle)."""

import numpy as np
import pytest

import oracle
from gpu_util import gsk
from problems import serving as sv

pytestmark = pytest.mark.gpu


def _requests():
    specs = sv.stream(14, rate=200.0, seed=11, side2d=(16, 96), side3d=(8, 24))
    from paper_0812_2769_gb300 import serve

    return [serve.Request(sp.rid, sp.build(), solver=sp.solver, m=sp.m, p=sp.p, tol=1e-8, precision="mixed",
                          arrival=sp.arrival) for sp in specs]


def test_results_same_alone_and_in_the_mix():
    gsk()
    from paper_0812_2769_gb300 import serve

    reqs = _requests()
    assert {r.solver for r in reqs} == {"gmres", "bicgstab"}
    be = serve.GpuBackend(0, slots=4)
    mixed = serve.Server(be, slots=4, small_n=2000).run(reqs, realtime=True)
    lanes = {r.lane for r in mixed}
    assert lanes == {"slot", "batch"}
    for q in reqs:
        alone = serve.Server(be, slots=1, small_n=2000).run([serve.Request(q.rid, q.system, q.solver, q.m, q.p,
                                                                            q.tol, q.precision, 0.0)],
                                                             realtime=False)[0]
        r = mixed[q.rid]
        assert r.status == alone.status == 0, (q.rid, q.solver, r.lane, r.status, alone.status,
                                                [c.last_error() for c in be.ctxs + [be.bctx]])
        assert np.all(np.isfinite(r.x)), q.rid
        assert np.array_equal(r.x, alone.x), q.rid
    summary = serve.summarize(mixed)
    assert summary["completed"] == len(reqs) and summary["p99_s"] >= summary["p50_s"]


def test_served_results_meet_the_metric():
    gsk()
    from paper_0812_2769_gb300 import serve

    reqs = _requests()
    res = serve.Server(serve.GpuBackend(0, slots=3), slots=3, small_n=2000).run(reqs, realtime=False)
    for q, r in zip(reqs, res):
        if r.info.get("conv") != 0:
            continue
        s = q.system
        val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)  # the metric of Sec. 2.2
        assert oracle.relres(s.rowptr, s.colidx, val, b, r.x) < 1e-8
    assert sum(r.info.get("conv") == 0 for r in res) >= len(reqs) // 2
