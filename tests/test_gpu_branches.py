"""GPU parity of the two solver branches that fire only when the cheap
convergence estimate and the true residual disagree, against the oracle
(whose branches are pinned in test_oracle_branches):

* Bi-CGSTAB's true-residual refresh and STAGNATED outcome (Sec. 2.2): on an
  ill-posed right-hand side the true metric cannot fall below ~5e-11, so at
  tol = 1e-13 every allowed refresh is taken and the solve ends STAGNATED.
  The first confirmation comes at the oracle's count (rounding ensemble, 5%,
  at least +-2).  After a restart from a residual at the rounding floor the
  counts are rounding noise, so there the GPU is held to the same restart
  identity that pins the oracle's branch (bit for bit, on the GPU itself),
  to the oracle's outcome and refresh count, and to the range of true
  metrics the oracle ends in.
* GMRES(m)'s tightened cycle target: on a row-scaled system the unweighted
  least-squares estimate meets tol a cycle before the GS(2)-weighted metric
  of Sec. 2.2 does, so the next cycle runs with tau * tol / metric.  These
  counts do not move with rounding (the oracle's ensemble has one value),
  so the GPU must take exactly the oracle's steps and restarts.

These systems are small, so the solvers run them on one thread-block
cluster; every test also runs the grid-wide kernels (a context created with
GSK_SMALL_N=0), whose branches are the same decisions in other code.
"""
import os

import numpy as np
import pytest

import oracle
from branch_cases import ill_posed_c1, row_scaled_system
from gpu_util import gsk

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


PATHS = ["cluster", "grid"]
_CTX = {}


def _ctx(path):
    """A context whose small systems take the cluster path, or none do."""
    if path not in _CTX:
        g = gsk()
        old = os.environ.get("GSK_SMALL_N")
        os.environ["GSK_SMALL_N"] = "32768" if path == "cluster" else "0"
        try:
            _CTX[path] = g.Context(0)
        finally:
            if old is None:
                del os.environ["GSK_SMALL_N"]
            else:
                os.environ["GSK_SMALL_N"] = old
    return _CTX[path]


def _gpu_solve(solver, rp, ci, va, b, tol, m=None, refresh=3, maxit=10000, x0=None, path="cluster"):
    import torch

    g = gsk()
    A = g.Csr.from_host(rp, ci, va, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bd) if x0 is None else torch.as_tensor(np.array(x0), device="cuda")
    o = g.opts(maxit=maxit, refresh=refresh)
    if solver == "gmres":
        info = g.gmres_solve(A, bd, x, m=m, tol=tol, options=o, ctx=_ctx(path))
    else:
        info = g.bicgstab_solve(A, bd, x, tol=tol, options=o, ctx=_ctx(path))
    return x.cpu().numpy(), info


def _perturbed(b, k):
    if k == 0:
        return b
    return b * (1.0 + np.random.default_rng(k).uniform(-1, 1, len(b)) * EPS)


@pytest.mark.parametrize("path", PATHS)
def test_bicgstab_stagnation_matches_the_oracle(path):
    """refresh = 0: the first true-residual confirmation ends the solve as
    STAGNATED, at the oracle's iteration count (rounding ensemble) and with a
    true metric in the range the oracle's runs end in."""
    rp, ci, va, b = ill_posed_c1()
    tol = 1e-13
    x_g, ig = _gpu_solve("bicgstab", rp, ci, va, b, tol, refresh=0, path=path)
    ens = [oracle.bicgstab(rp, ci, va, _perturbed(b, k), tol=tol, refresh=0) for k in range(8)]
    its = [e[1]["iters"] for e in ens]
    mus = [e[1]["relres_true"] for e in ens]
    msg = f"gpu={ig} oracle iters={its} mu={mus}"
    assert all(e[1]["conv"] == oracle.STAGNATED for e in ens)
    assert ig["conv"] == oracle.STAGNATED and ig["refreshes"] == 0, msg
    lo, hi = min(its), max(its)
    assert min(0.95 * lo, lo - 2) <= ig["iters"] <= max(1.05 * hi, hi + 2), msg
    assert ig["relres_rec"] < tol, msg
    # the true metric of the GPU's x, recomputed by the oracle: at this floor
    # (eps cond(A)) the residual itself carries rounding noise of a few per
    # cent, so the reported and recomputed values agree to 10%
    mu_g = oracle.relres(rp, ci, va, b, x_g)
    assert abs(mu_g - ig["relres_true"]) <= 0.1 * mu_g, (mu_g, msg)
    assert mu_g >= tol and 0.3 * min(mus) <= mu_g <= 3.0 * max(mus), (mu_g, msg)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("refresh", [1, 3])
def test_bicgstab_refresh_continues_as_a_fresh_start_on_the_gpu(refresh, path):
    """The GPU's refresh restarts r, r^ and p from the true residual: a solve
    with `refresh` restarts continues exactly (bit for bit) like a fresh GPU
    solve started from the x of the first confirmation with refresh - 1, its
    tolerance rescaled to the fresh start's ||W r0|| -- the identity that
    pins the oracle's branch (test_oracle_branches).  After the restarts the
    solve is STAGNATED, as in the oracle, every refresh taken, and its true
    metric lies in the oracle's range."""
    rp, ci, va, b = ill_posed_c1()
    tol = 1e-13
    x, info = _gpu_solve("bicgstab", rp, ci, va, b, tol, refresh=refresh, path=path)
    x1, i1 = _gpu_solve("bicgstab", rp, ci, va, b, tol, refresh=0, path=path)
    assert i1["conv"] == oracle.STAGNATED
    w = oracle.metric_weights(rp, va)
    mu0 = np.linalg.norm(w * b)
    mu1 = np.linalg.norm(w * (b - oracle.spmv(rp, ci, va, x1)))
    x2, i2 = _gpu_solve("bicgstab", rp, ci, va, b, tol * mu0 / mu1, refresh=refresh - 1, x0=x1, path=path)
    msg = f"full={info} first={i1} fresh={i2}"
    assert info["iters"] == i1["iters"] + i2["iters"], msg
    assert info["refreshes"] == 1 + i2["refreshes"], msg
    assert np.array_equal(x, x2), msg
    # outcome against the oracle
    ens = [oracle.bicgstab(rp, ci, va, _perturbed(b, k), tol=tol, refresh=refresh) for k in range(8)]
    mus = [e[1]["relres_true"] for e in ens]
    assert all(e[1]["conv"] == oracle.STAGNATED and e[1]["refreshes"] == refresh for e in ens)
    assert info["conv"] == oracle.STAGNATED and info["refreshes"] == refresh, msg
    mu = oracle.relres(rp, ci, va, b, x)
    assert mu >= tol and 0.3 * min(mus) <= mu <= 3.0 * max(mus), (mu, mus, msg)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("seed,m", [(11, 20), (3, 20), (29, 20), (3, 40)])
def test_gmres_tightened_target_matches_the_oracle(seed, m, path):
    rp, ci, va, b = row_scaled_system(seed)
    tol = 1e-10
    x_o, io, cyc = oracle.gmres(rp, ci, va, b, m=m, tol=tol, maxit=2000, trace=True)
    assert any(c["est"] < c["tau"] and c["mu"] >= tol for c in cyc), "the case must tighten tau"
    x_g, ig = _gpu_solve("gmres", rp, ci, va, b, tol, m=m, maxit=2000, path=path)
    msg = f"gpu={ig} oracle={io} cycles={[c['steps'] for c in cyc]}"
    assert ig["conv"] == oracle.CONVERGED, msg
    assert ig["iters"] == io["iters"] and ig["restarts"] == io["restarts"], msg
    mu_g = oracle.relres(rp, ci, va, b, x_g)
    assert mu_g < tol and abs(mu_g - ig["relres_true"]) <= 1e-6 * mu_g, msg
    assert np.linalg.norm(x_g - x_o) <= 1e-8 * np.linalg.norm(x_o), msg
