"""Pins for the two branches of the oracle's solvers that only fire when the
cheap convergence estimate and the true residual disagree (CPU, no GPU):

* Bi-CGSTAB's true-residual refresh (Sec. 2.2, and the remark in Sec. 4 that
  the updated residual can report convergence that the true residual does
  not confirm): when the recursive residual meets tol but the true one does
  not, r, r^ and p restart from the true residual b - Ax and the iteration
  goes on, at most `refresh` times; then the outcome is STAGNATED.
* GMRES(m)'s cycle target: a cycle ends when its least-squares estimate
  |g_{j+1}| / ||r0|| falls below tau (tau = tol at first); if the weighted
  true metric after the cycle's update is still >= tol, the next cycle runs
  with tau * tol / metric.

Each branch is pinned by a restart identity rather than by re-deriving its
formulas: a refreshed Bi-CGSTAB run must continue exactly like a fresh run
started from the x at which the refresh happened, and the cycle after a
tightening must end exactly where a fresh GMRES(m) run from that cycle's x,
given the tightened target, ends its own first cycle.  The fresh runs are
the plain textbook starts, which test_oracle_scipy pins against SciPy.  So
a refresh that keeps the old r^ or p, an iteration or refresh count that is
not carried over, a tau that is not tightened or tightened by the wrong
factor, or an outcome decided by the estimate rather than the true metric,
each breaks one of these tests.
"""
import numpy as np
import pytest

import oracle

pytest.importorskip("scipy.sparse")
from branch_cases import ill_posed_c1 as _ill_posed_c1, row_scaled_system  # noqa: E402


# ----------------------------------------------------- Bi-CGSTAB refresh
def _wmetric(rp, ci, va, b, x):
    """||W(b - Ax)|| / ||W b|| in numpy (x0 = 0), W = 1/||a_i||_2."""
    w = np.array([1.0 / np.linalg.norm(va[rp[i]:rp[i + 1]]) for i in range(len(rp) - 1)])
    r = b - oracle.spmv(rp, ci, va, x)
    return float(np.linalg.norm(w * r) / np.linalg.norm(w * b))


def test_bicgstab_without_refresh_reports_stagnation_with_the_true_metric():
    rp, ci, va, b = _ill_posed_c1()
    tol = 1e-13
    x, info, hist, checks = oracle.bicgstab(rp, ci, va, b, tol=tol, refresh=0, history=True, trace=True)
    assert info["conv"] == oracle.STAGNATED and info["refreshes"] == 0
    assert len(checks) == 1 and checks[0]["iters"] == info["iters"]
    # the recursive metric met tol, the true one (recomputed here) did not
    assert hist[-1] < tol and info["relres_rec"] < tol
    mu = _wmetric(rp, ci, va, b, x)
    assert mu >= tol
    assert abs(info["relres_true"] - mu) <= 1e-10 * mu


@pytest.mark.parametrize("tol,refresh", [(1e-13, 1), (1e-13, 3), (1e-11, 3)])
def test_bicgstab_refresh_continues_as_a_fresh_start(tol, refresh):
    rp, ci, va, b = _ill_posed_c1()
    x, info, hist, checks = oracle.bicgstab(rp, ci, va, b, tol=tol, refresh=refresh, history=True, trace=True)
    assert info["refreshes"] >= 1, "the case must take the refresh branch"
    # the x of the first confirmation: the same run with no refresh allowed
    x1, i1 = oracle.bicgstab(rp, ci, va, b, tol=tol, refresh=0)
    k1 = i1["iters"]
    assert checks[0]["iters"] == k1 and i1["conv"] == oracle.STAGNATED
    # a fresh run from x1; its metric is relative to ||W(b - A x1)||, so the
    # tolerance is rescaled to keep every stopping test the same
    w = np.array([1.0 / np.linalg.norm(va[rp[i]:rp[i + 1]]) for i in range(len(rp) - 1)])
    mu0 = np.linalg.norm(w * b)
    mu1 = np.linalg.norm(w * (b - oracle.spmv(rp, ci, va, x1)))
    x2, i2, hist2 = oracle.bicgstab(rp, ci, va, b, tol=tol * mu0 / mu1, refresh=refresh - 1, x0=x1, history=True)
    assert info["iters"] == k1 + i2["iters"]
    assert info["refreshes"] == 1 + i2["refreshes"]
    assert info["conv"] == i2["conv"]
    assert np.array_equal(x, x2), "the refreshed iterates differ from a fresh start"
    np.testing.assert_allclose(hist[k1:], hist2 * (mu1 / mu0), rtol=1e-13, atol=0)
    # the outcome follows the true metric of the returned x
    mu = _wmetric(rp, ci, va, b, x)
    assert (info["conv"] == oracle.CONVERGED) == (mu < tol)
    assert abs(info["relres_true"] - mu) <= 1e-10 * mu


def test_bicgstab_refreshes_are_bounded_then_stagnate():
    rp, ci, va, b = _ill_posed_c1()
    for k in (1, 2, 4):
        x, info, checks = oracle.bicgstab(rp, ci, va, b, tol=1e-13, refresh=k, trace=True)
        assert info["conv"] == oracle.STAGNATED and info["refreshes"] == k
        assert len(checks) == k + 1
        assert all(c["mu"] >= 1e-13 for c in checks)
        assert [c["iters"] for c in checks] == sorted(c["iters"] for c in checks)


# ------------------------------------------------- GMRES cycle target tau
@pytest.mark.parametrize("seed,m", [(11, 20), (3, 20), (29, 20), (3, 40)])
def test_gmres_tightened_target_ends_the_next_cycle(seed, m):
    tol = 1e-10
    rp, ci, va, b = row_scaled_system(seed)
    x, info, hist, cyc = oracle.gmres(rp, ci, va, b, m=m, tol=tol, maxit=2000, history=True, trace=True)
    assert info["conv"] == oracle.CONVERGED
    assert len(cyc) == info["restarts"] + 1 and sum(c["steps"] for c in cyc) == info["iters"]
    # the first cycle whose estimate met tau while the true metric did not
    hits = [k for k, c in enumerate(cyc) if c["est"] < c["tau"] and c["mu"] >= tol]
    assert hits, "the case must take the tightening branch"
    c = hits[0]
    assert all(cc["tau"] == tol for cc in cyc[:c + 1])
    assert cyc[c + 1]["tau"] == cyc[c]["tau"] * (tol / cyc[c]["mu"])
    # the tightened cycle runs past the point where the old target would
    # have ended it
    start = sum(cc["steps"] for cc in cyc[:c + 1])
    nxt = hist[start:start + cyc[c + 1]["steps"]]
    if len(nxt) > 1:
        assert nxt[:-1].min() < cyc[c]["tau"]
    assert (nxt[:-1] >= cyc[c + 1]["tau"]).all()
    # x after cycle c: the same run stopped there by maxit
    xc, ic = oracle.gmres(rp, ci, va, b, m=m, tol=tol, maxit=start)
    assert ic["iters"] == start and ic["conv"] == oracle.MAXIT
    # a fresh GMRES(m) from xc whose first target is the tightened tau,
    # expressed relative to its own ||r0||, ends its first cycle where the
    # original run ended cycle c + 1
    rho0 = np.linalg.norm(b)
    rho_c = np.linalg.norm(b - oracle.spmv(rp, ci, va, xc))
    tol_f = cyc[c + 1]["tau"] * rho0 / rho_c
    _, _, hist_f, cyc_f = oracle.gmres(rp, ci, va, b, m=m, tol=tol_f, maxit=m, x0=xc, history=True, trace=True)
    assert cyc_f[0]["steps"] == cyc[c + 1]["steps"]
    np.testing.assert_allclose(hist_f[:cyc_f[0]["steps"]] * (rho_c / rho0), nxt, rtol=1e-9, atol=0)
    # the outcome follows the true metric, recomputed here
    w = np.array([1.0 / np.linalg.norm(va[rp[i]:rp[i + 1]]) for i in range(len(rp) - 1)])
    mu = np.linalg.norm(w * (b - oracle.spmv(rp, ci, va, x))) / np.linalg.norm(w * b)
    assert mu < tol and abs(info["relres_true"] - mu) <= 1e-9 * mu


def test_gmres_cycles_end_only_on_target_breakdown_or_length():
    tol = 1e-10
    rp, ci, va, b = row_scaled_system(11)
    m = 20
    _, info, hist, cyc = oracle.gmres(rp, ci, va, b, m=m, tol=tol, maxit=2000, history=True, trace=True)
    k = 0
    for c in cyc:
        seg = hist[k:k + c["steps"]]
        k += c["steps"]
        # every step but the last stayed above the cycle's target; a cycle
        # shorter than m ended because its last estimate met the target
        assert (seg[:-1] >= c["tau"]).all()
        if c["steps"] < m:
            assert seg[-1] < c["tau"]
        assert seg[-1] == c["est"]
