"""Small systems on one thread-block cluster, GMRES(m): gmres_solve takes
that path when the system's basis fits the cluster's shared memory (the
other solver tests exercise it on C1, the small grids and the restart
branches against the oracle).  Here: availability, exact step counts against
the oracle over ragged sizes and every restart length class, agreement with
the grid-wide solver (a context created with GSK_SMALL_N=0), the metric
options, degenerate cases and errors."""
import os

import numpy as np
import pytest

import oracle
from gpu_util import gsk
from problems import cd, configs

pytestmark = pytest.mark.gpu


def _ctx(grid_wide):
    g = gsk()
    old = os.environ.get("GSK_SMALL_N")
    os.environ["GSK_SMALL_N"] = "0" if grid_wide else "32768"
    try:
        return g.Context(0)
    finally:
        if old is None:
            del os.environ["GSK_SMALL_N"]
        else:
            os.environ["GSK_SMALL_N"] = old


def _solve(sys_, m, tol=1e-8, ctx=None, **kw):
    import torch

    g = gsk()
    A = g.Csr.from_host(sys_.rowptr, sys_.colidx, sys_.val)
    b = torch.as_tensor(sys_.b, device="cuda")
    x = torch.zeros(sys_.n, dtype=torch.float64, device="cuda")
    info = g.gmres_solve(A, b, x, m=m, tol=tol, options=g.opts(**kw), ctx=ctx)
    return x.cpu().numpy(), info


def _well_conditioned(n, seed, per_row=6):
    rs = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        c = np.unique(np.concatenate([[i], rs.integers(0, n, per_row)]))
        v = rs.uniform(-1, 1, len(c))
        v[c == i] = rs.uniform(2, 3) * (per_row + 1)
        rows.append(len(c))
        cols.append(c)
        vals.append(v)
    rp = np.concatenate([[0], np.cumsum(rows)]).astype(np.int32)
    return cd.System(n, rp, np.concatenate(cols).astype(np.int32), np.concatenate(vals), rs.normal(size=n))


def test_the_cluster_path_is_available():
    g = gsk()
    c = _ctx(False)
    rows = [g.gmres_small_system_rows(m, ctx=c) for m in (10, 20, 30, 64)]
    # C1 (1,024 rows) and the 12^3 grid take it at every restart length used
    assert rows[1] >= 4096 and rows[-1] >= 1728, rows
    assert rows == sorted(rows, reverse=True)  # a longer basis leaves fewer rows
    assert g.gmres_small_system_rows(20, ctx=_ctx(True)) == 0


@pytest.mark.parametrize("n,m", [(5, 4), (17, 8), (1000, 20), (4099, 16), (3000, 64)])
def test_exact_steps_against_the_oracle(n, m):
    # ragged sizes (n = 5, 17: most CTAs own no row) and every column class;
    # well conditioned, so the oracle's step count is not decided by rounding
    s = _well_conditioned(n, seed=n + m)
    o = dict(metric=gsk().METRIC_PLAIN)
    x, info = _solve(s, m, tol=1e-12, **o)
    xo, io = oracle.gmres(s.rowptr, s.colidx, s.val, s.b, m=m, tol=1e-12, w=np.ones(n))
    assert info["conv"] == io["conv"] == oracle.CONVERGED, (info, io)
    assert info["iters"] == io["iters"] and info["restarts"] == io["restarts"], (info, io)
    assert np.abs(x - xo).max() <= 1e-11 * np.abs(xo).max()
    mu = oracle.relres(s.rowptr, s.colidx, s.val, s.b, x, w=np.ones(n))
    assert abs(mu - info["relres_true"]) <= 1e-6 * mu + 1e-15


def test_restarts_and_maxit_against_the_oracle():
    # a short restart length on a harder system: several cycles, then maxit
    s = _well_conditioned(2000, seed=3, per_row=12)
    for maxit in (7, 45):
        x, info = _solve(s, 5, tol=1e-14, maxit=maxit, metric=gsk().METRIC_PLAIN)
        xo, io = oracle.gmres(s.rowptr, s.colidx, s.val, s.b, m=5, tol=1e-14, maxit=maxit, w=np.ones(s.n))
        assert (info["conv"], info["iters"], info["restarts"]) == (io["conv"], io["iters"], io["restarts"]), (info, io)
        assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()


def test_cluster_and_grid_wide_solvers_agree():
    g = gsk()
    c1 = configs.c1()
    v, b, _ = oracle.gs_scale(c1.rowptr, c1.colidx, c1.val, c1.b, 2.0)
    s = cd.System(c1.n, c1.rowptr, c1.colidx, v, b)
    c_cl, c_gw = _ctx(False), _ctx(True)
    # GMRES(20) on C1 stagnates: both run the 400 steps and end at the same metric
    x1, i1 = _solve(s, 20, ctx=c_cl, maxit=400)
    x2, i2 = _solve(s, 20, ctx=c_gw, maxit=400)
    x3, i3 = _solve(s, 20, ctx=c_cl, maxit=400)
    assert np.array_equal(x1, x3) and i1["iters"] == i3["iters"]  # deterministic
    assert i1["conv"] == i2["conv"] == g.MAXIT and i1["iters"] == i2["iters"] == 400
    assert abs(i1["relres_true"] - i2["relres_true"]) <= 1e-2 * i2["relres_true"]
    # 12^3 grid, GS(2): converges, in the oracle's rounding ensemble
    c2 = configs.c2(12)
    v, b, _ = oracle.gs_scale(c2.rowptr, c2.colidx, c2.val, c2.b, 2.0)
    s2 = cd.System(c2.n, c2.rowptr, c2.colidx, v, b)
    xa, ia = _solve(s2, 30, ctx=c_cl)
    xb, ib = _solve(s2, 30, ctx=c_gw)
    assert ia["conv"] == ib["conv"] == g.CONVERGED
    assert abs(ia["iters"] - ib["iters"]) <= 2 + 0.05 * ib["iters"], (ia, ib)
    for x in (xa, xb):
        assert oracle.relres(s2.rowptr, s2.colidx, s2.val, s2.b, x) < 1e-8
    c_cl.close()
    c_gw.close()


def test_metric_options_on_the_cluster():
    import torch

    g = gsk()
    s = configs.c2(10)  # unscaled: the GS(2) weights are not the identity (~2,000 steps)
    x, info = _solve(s, 30, tol=1e-8, metric=g.METRIC_PLAIN)
    r = s.b - oracle.spmv(s.rowptr, s.colidx, s.val, x)
    assert info["conv"] == g.CONVERGED
    assert abs(np.linalg.norm(r) / np.linalg.norm(s.b) - info["relres_true"]) <= 1e-6 * info["relres_true"]
    x, info = _solve(s, 30, tol=1e-8)
    assert info["conv"] == g.CONVERGED
    assert oracle.relres(s.rowptr, s.colidx, s.val, s.b, x) < 1e-8
    w = torch.as_tensor(oracle.metric_weights(s.rowptr, s.val), device="cuda")
    xw, iw = _solve(s, 30, tol=1e-8, weights=w)
    # the same metric as the default (weights within an ulp or two of the
    # library's own): the same outcome, the count within a few percent
    assert iw["conv"] == g.CONVERGED and abs(iw["iters"] - info["iters"]) <= 0.05 * info["iters"]
    assert oracle.relres(s.rowptr, s.colidx, s.val, s.b, xw) < 1e-8


def test_trivial_and_degenerate_cases():
    g = gsk()
    s = configs.c1(8)
    z = cd.System(s.n, s.rowptr, s.colidx, s.val, np.zeros(s.n))
    x, info = _solve(z, 10)
    assert info["conv"] == g.CONVERGED and info["iters"] == 0 and not x.any()
    x, info = _solve(s, 10, maxit=0)
    assert info["conv"] == g.MAXIT and info["iters"] == 0
    # a multiple of the identity: one step
    n = 100
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    eye = cd.System(n, rp, ci, np.full(n, 3.0), np.arange(1.0, n + 1.0))
    x, info = _solve(eye, 10, tol=1e-12)
    assert info["conv"] == g.CONVERGED and info["iters"] == 1
    assert np.allclose(x, np.arange(1.0, n + 1.0) / 3.0, rtol=1e-15)
    # k distinct eigenvalues: finite termination in k steps (Krylov space invariant)
    d = np.repeat([1.0, 2.0, 5.0], [30, 30, 40])
    diag = cd.System(n, rp, ci, d, np.ones(n))
    x, info = _solve(diag, 20, tol=1e-14, metric=g.METRIC_PLAIN)
    xo, io = oracle.gmres(rp, ci, d, np.ones(n), m=20, tol=1e-14, w=np.ones(n))
    assert info["conv"] == io["conv"] == g.CONVERGED and info["iters"] == io["iters"] == 3, (info, io)


def test_errors_on_the_cluster():
    g = gsk()
    s = configs.c1(8)
    ci = s.colidx.copy()
    ci[7] = s.n + 3
    with pytest.raises(g.GskError) as ei:
        _solve(cd.System(s.n, s.rowptr, ci, s.val, s.b), 10)
    assert ei.value.status == g.ERR_ARG
    val = s.val.copy()
    val[s.rowptr[10]:s.rowptr[11]] = 0.0
    with pytest.raises(g.GskError) as ei:
        _solve(cd.System(s.n, s.rowptr, s.colidx, val, s.b), 10)
    assert ei.value.status == g.ERR_ZERO_ROW
    val = s.val.copy()
    val[5] = np.nan
    with pytest.raises(g.GskError) as ei:
        _solve(cd.System(s.n, s.rowptr, s.colidx, val, s.b), 10)
    assert ei.value.status == g.ERR_NONFINITE
