"""Small systems on one thread-block cluster: bicgstab_solve takes that path
for systems of at most 32,768 rows (the other solver tests exercise it on
C1 and the 12^3 and 21^3 grids against the oracle).  Here: its edge cases
against the oracle, its agreement with the grid-wide solver (a context
created with GSK_SMALL_N=0), and its errors."""
import os

import numpy as np
import pytest

import oracle
from gpu_util import gsk, random_csr
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


def _solve(sys_, tol=1e-8, ctx=None, **kw):
    import torch

    g = gsk()
    A = g.Csr.from_host(sys_.rowptr, sys_.colidx, sys_.val)
    b = torch.as_tensor(sys_.b, device="cuda")
    x = torch.zeros(sys_.n, dtype=torch.float64, device="cuda")
    info = g.bicgstab_solve(A, b, x, tol=tol, options=g.opts(**kw), ctx=ctx)
    return x.cpu().numpy(), info


def _scaled(s):
    v, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    return cd.System(s.n, s.rowptr, s.colidx, v, b, s.x_true)


def test_the_cluster_path_is_available():
    # on a GB300 every system of these tests (and C1) takes the cluster path;
    # GSK_SMALL_N=0 turns it off
    g = gsk()
    assert g.small_system_rows(_ctx(False)) >= 32768
    assert g.small_system_rows(_ctx(True)) == 0


@pytest.mark.parametrize("n", [5, 17, 1000, 4099])
def test_ragged_sizes_match_the_oracle(n):
    # row counts that are not multiples of the cluster's 16 CTAs (n = 5: most
    # CTAs own no row); a well-conditioned system, so the counts agree exactly
    rp, ci, va = random_csr(n, 40 + n, min_len=1, max_len=6)
    b = np.random.default_rng(n).normal(size=n)
    s = cd.System(n, rp, ci, va, b)
    x, info = _solve(s, tol=1e-10, refresh=0)
    xo, io = oracle.bicgstab(rp, ci, va, b, tol=1e-10, refresh=0)
    assert info["conv"] == io["conv"] == oracle.CONVERGED, (info, io)
    assert abs(info["iters"] - io["iters"]) <= 1, (info, io)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    mu = oracle.relres(rp, ci, va, b, x)
    # (at the rounding floor the recomputed residual differs in its last digits)
    assert mu < 1e-10 and abs(mu - info["relres_true"]) <= 1e-6 * mu + 1e-14


def test_cluster_and_grid_wide_solvers_agree():
    g = gsk()
    s = _scaled(configs.c1())
    c_cl, c_gw = _ctx(False), _ctx(True)
    x1, i1 = _solve(s, ctx=c_cl)
    x2, i2 = _solve(s, ctx=c_gw)
    x3, i3 = _solve(s, ctx=c_cl)
    assert np.array_equal(x1, x3) and i1["iters"] == i3["iters"]  # deterministic
    assert i1["conv"] == i2["conv"] == g.CONVERGED
    # the two sum their dot products in different orders; the counts are in
    # the oracle's rounding ensemble (test_gpu_solvers), here within 25%
    assert abs(i1["iters"] - i2["iters"]) <= 0.25 * i2["iters"], (i1, i2)
    for x in (x1, x2):
        assert oracle.relres(s.rowptr, s.colidx, s.val, s.b, x) < 1e-8
    c_cl.close()
    c_gw.close()


def test_metric_options_on_the_cluster():
    import torch

    g = gsk()
    s = configs.c1()  # unscaled: the GS(2) weights are not the identity
    # plain metric: ||b - Ax|| / ||b||
    x, info = _solve(s, tol=1e-8, metric=g.METRIC_PLAIN)
    r = s.b - oracle.spmv(s.rowptr, s.colidx, s.val, x)
    assert info["conv"] == g.CONVERGED
    assert abs(np.linalg.norm(r) / np.linalg.norm(s.b) - info["relres_true"]) <= 1e-6 * info["relres_true"]
    # caller's weights (here the GS(2) scales, computed by the oracle): the
    # same metric as the default, so the reported values agree
    w = torch.as_tensor(oracle.metric_weights(s.rowptr, s.val), device="cuda")
    xw, iw = _solve(s, tol=1e-8, weights=w)
    x0, i0 = _solve(s, tol=1e-8)
    assert iw["conv"] == i0["conv"] == g.CONVERGED
    assert oracle.relres(s.rowptr, s.colidx, s.val, s.b, xw) < 1e-8


def test_trivial_and_degenerate_cases():
    g = gsk()
    s = configs.c1(8)
    # b = 0: converged at once, x = 0
    z = cd.System(s.n, s.rowptr, s.colidx, s.val, np.zeros(s.n))
    x, info = _solve(z)
    assert info["conv"] == g.CONVERGED and info["iters"] == 0 and not x.any()
    # maxit = 0: no iteration, outcome maxit
    x, info = _solve(s, maxit=0)
    assert info["conv"] == g.MAXIT and info["iters"] == 0
    # a multiple of the identity converges in one iteration
    n = 100
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    eye = cd.System(n, rp, ci, np.full(n, 3.0), np.arange(1.0, n + 1.0))
    x, info = _solve(eye, tol=1e-12)
    assert info["conv"] == g.CONVERGED and info["iters"] == 1
    assert np.allclose(x, np.arange(1.0, n + 1.0) / 3.0, rtol=1e-15)
    # breakdown: a rotation (sigma = <r^, A r> = 0 at the first step)
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([1, 0], dtype=np.int32)
    rot = cd.System(2, rp, ci, np.array([1.0, -1.0]), np.array([1.0, 0.0]))
    _, info = _solve(rot, tol=1e-10, metric=g.METRIC_PLAIN)
    _, io = oracle.bicgstab(rp, ci, np.array([1.0, -1.0]), np.array([1.0, 0.0]), tol=1e-10, w=np.ones(2))
    assert info["conv"] == io["conv"] == g.BREAKDOWN


def test_errors_on_the_cluster():
    g = gsk()
    s = configs.c1(8)
    ci = s.colidx.copy()
    ci[7] = s.n + 3
    with pytest.raises(g.GskError) as ei:
        _solve(cd.System(s.n, s.rowptr, ci, s.val, s.b))
    assert ei.value.status == g.ERR_ARG
    val = s.val.copy()
    val[s.rowptr[10]:s.rowptr[11]] = 0.0
    with pytest.raises(g.GskError) as ei:
        _solve(cd.System(s.n, s.rowptr, s.colidx, val, s.b))
    assert ei.value.status == g.ERR_ZERO_ROW
