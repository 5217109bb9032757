"""Degenerate inputs through the C ABI: the empty system (n = 0) at every
entry point of the path, and an empty member inside a batch.  An empty
system is solved by x = [] with zero iterations (its initial residual is
zero, the converged outcome of Sec. 2.2's test), and scaling it is a no-op."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import gsk
from problems import cd, configs

pytestmark = pytest.mark.gpu


def _empty(g):
    import torch

    A = g.Csr.from_host(np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    return A, z


@pytest.mark.parametrize("p", [1.0, 2.0, math.inf])
def test_scalings_of_the_empty_system(p):
    import torch

    g = gsk()
    A, z = _empty(g)
    g.gs_scale(A, z, p=p)
    d = torch.zeros(0, dtype=torch.float64, device="cuda")
    g.gs_scale(A, z, p=p, d_out=d)
    g.gs_scale_static(A, z, p=p)
    s = torch.zeros(0, dtype=torch.float64, device="cuda")
    g.gs_scale_sym(A, z, p=p, s_out=s)
    assert g.profile_gs_scale(A, z, p=p) == 0.0
    y = torch.zeros(0, dtype=torch.float64, device="cuda")
    g.gsk_spmv(A, z, y)


def test_solvers_on_the_empty_system():
    import torch

    g = gsk()
    A, z = _empty(g)
    e = (np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0), np.zeros(0))
    _, ib = oracle.bicgstab(*e, tol=1e-8)
    _, ig = oracle.gmres(*e, m=20, tol=1e-8)
    for prec in (g.PREC_F64, g.PREC_MIXED):
        o = g.opts(precision=prec)
        x = torch.zeros(0, dtype=torch.float64, device="cuda")
        info = g.bicgstab_solve(A, z, x, tol=1e-8, options=o)
        assert info["conv"] == ib["conv"] == g.CONVERGED and info["iters"] == ib["iters"] == 0
        info = g.gmres_solve(A, z, x, m=20, tol=1e-8, options=o)
        assert info["conv"] == ig["conv"] == g.CONVERGED and info["iters"] == ig["iters"] == 0


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_an_empty_member_of_a_batch(solver):
    """An empty system between ordinary ones: it converges at once and the
    others give bitwise the results of a batch without it."""
    import torch

    g = gsk()
    systems = [configs.c4_system(i) for i in range(3)]
    mk = lambda ss: ([g.Csr.from_host(s.rowptr, s.colidx, s.val) for s in ss],
                     [torch.as_tensor(s.b, device="cuda") for s in ss],
                     [torch.zeros(s.n, dtype=torch.float64, device="cuda") for s in ss])
    As, bs, xs = mk(systems)
    Ae, ze = _empty(g)
    As.insert(1, Ae)
    bs.insert(1, ze)
    xs.insert(1, torch.zeros(0, dtype=torch.float64, device="cuda"))
    if solver == "gmres":
        infos, stat = g.gmres_solve_batched(As, bs, xs, m=20, p=2.0, tol=1e-8, options=g.opts(maxit=1000))
    else:
        infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=2.0, tol=1e-8)
    assert all(st == g.OK for st in stat)
    assert infos[1]["conv"] == g.CONVERGED and infos[1]["iters"] == 0
    A2, b2, x2 = mk(systems)
    if solver == "gmres":
        inf2, _ = g.gmres_solve_batched(A2, b2, x2, m=20, p=2.0, tol=1e-8, options=g.opts(maxit=1000))
    else:
        inf2, _ = g.bicgstab_solve_batched(A2, b2, x2, p=2.0, tol=1e-8)
    for q, i in enumerate((0, 2, 3)):
        assert torch.equal(x2[q], xs[i]) and inf2[q]["iters"] == infos[i]["iters"]


def test_a_single_row_system():
    # n = 1: one equation a x = b.  Bi-CGSTAB takes the cluster path, where
    # fifteen of the sixteen CTAs own no row
    import torch

    g = gsk()
    s = cd.System(1, np.array([0, 1], dtype=np.int32), np.array([0], dtype=np.int32), np.array([-4.0]),
                  np.array([2.0]))
    for solver in ("bicgstab", "gmres"):
        A = g.Csr.from_host(s.rowptr, s.colidx, s.val)
        b = torch.as_tensor(s.b, device="cuda")
        x = torch.zeros(1, dtype=torch.float64, device="cuda")
        info = (g.bicgstab_solve(A, b, x, tol=1e-12) if solver == "bicgstab"
                else g.gmres_solve(A, b, x, m=5, tol=1e-12))
        assert info["conv"] == g.CONVERGED and info["iters"] == 1, (solver, info)
        assert abs(x.item() + 0.5) <= 1e-15
