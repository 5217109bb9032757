"""GPU parity of the two-sided scaling D^1/2 A D^1/2 (Sec. 2) against the CPU
oracle, through the C ABI, and a solve of a scaled system recovered by
x = D^1/2 y that stops on the GS(2)-scaled residual of the original system
(Sec. 2.2)."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import gsk, random_csr, to_dev
from problems import cd, configs

pytestmark = pytest.mark.gpu

# a_ij s_i s_j with s = sqrt(1/||a_i||_p): the norm is summed in another
# order and the square roots round independently, so a few ulp apart
SYM_RTOL = 2e-14


def _sym_case(sys_, p, weights=True):
    g = gsk()
    A, b = to_dev(g, sys_)
    s, w = g.gs_scale_sym(A, b, p=p, weights=weights)
    val_or, b_or, s_or, w_or = oracle.gs_scale_sym(sys_.rowptr, sys_.colidx, sys_.val, sys_.b, p)
    val = A.val.cpu().numpy()
    assert np.all(np.abs(val - val_or) <= SYM_RTOL * np.abs(val_or)), np.max(np.abs(val - val_or) / np.abs(val_or))
    assert np.allclose(b.cpu().numpy(), b_or, rtol=SYM_RTOL, atol=1e-300)
    assert np.allclose(s.cpu().numpy(), s_or, rtol=SYM_RTOL, atol=0)
    if weights:
        assert np.allclose(w.cpu().numpy(), w_or, rtol=SYM_RTOL, atol=0)
    else:
        assert w is None


@pytest.mark.parametrize("p", [1.0, 2.0, math.inf, 3.5])
def test_sym_scaling_c1(p):
    _sym_case(configs.c1(), p)


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_sym_scaling_c2_small_and_random_ragged(p):
    _sym_case(configs.c2(21), p)
    rp, ci, va = random_csr(3000, 5, long_rows=(7, 1500), long_len=400)
    rs = np.random.default_rng(3)
    _sym_case(cd.System(3000, rp, ci, va, rs.normal(size=3000)), p, weights=(p == 1.0))


def test_sym_scaling_errors_leave_the_input():
    import torch

    g = gsk()
    s0 = configs.c1(16)
    bad = s0.colidx.copy()
    bad[10] = s0.n  # a column outside [0, n)
    for rowptr, colidx, val, status in [
        (s0.rowptr, bad, s0.val, g.ERR_ARG),
        (s0.rowptr, s0.colidx, np.where(np.arange(len(s0.val)) == 3, np.nan, s0.val), g.ERR_NONFINITE),
    ]:
        A = g.Csr.from_host(rowptr, colidx, val, device="cuda")
        b = torch.as_tensor(s0.b, device="cuda")
        v_before, b_before = A.val.clone(), b.clone()
        with pytest.raises(g.GskError) as e:
            g.gs_scale_sym(A, b, p=2.0)
        assert e.value.status == status
        assert torch.equal(A.val.isnan(), v_before.isnan())
        assert torch.equal(torch.nan_to_num(A.val), torch.nan_to_num(v_before)) and torch.equal(b, b_before)


def test_solve_through_sym_scaling_meets_the_original_metric():
    """Bi-CGSTAB and GMRES on D^1/2 A D^1/2 y = D^1/2 b with the weights w:
    x = D^1/2 y meets the GS(2)-scaled relative residual of A x = b
    (recomputed by the oracle) and is close to the oracle's GS(2) solution."""
    import torch

    g = gsk()
    s0 = configs.c1()
    val2, b2, _ = oracle.gs_scale(s0.rowptr, s0.colidx, s0.val, s0.b, 2.0)
    x_ref, _ = oracle.bicgstab(s0.rowptr, s0.colidx, val2, b2, tol=1e-12)
    # two tol-accurate solutions differ by at most about cond(A) * tol
    cond = float(np.linalg.cond(cd.System(s0.n, s0.rowptr, s0.colidx, val2, b2).dense()))
    bound = max(1e-6, 4 * cond * 1e-9)
    for solver in ("bicgstab", "gmres"):
        A, b = to_dev(g, s0)
        s, w = g.gs_scale_sym(A, b, p=2.0, weights=True)
        y = torch.zeros(s0.n, dtype=torch.float64, device="cuda")
        # GMRES(20) needs thousands of steps here, a count decided by rounding
        # (the oracle's ensemble: 5,900 .. 9,660), so it gets room beyond
        # the default 10,000
        o = g.opts(weights=w, maxit=40000)
        if solver == "gmres":
            info = g.gmres_solve(A, b, y, m=20, tol=1e-9, options=o)
        else:
            info = g.bicgstab_solve(A, b, y, tol=1e-9, options=o)
        assert info["conv"] == 0, info
        x = g.diag_mul(s, y).cpu().numpy()
        assert oracle.relres(s0.rowptr, s0.colidx, val2, b2, x) < 1e-9
        assert abs(info["relres_true"] - oracle.relres(s0.rowptr, s0.colidx, val2, b2, x)) < 1e-12
        assert np.linalg.norm(x - x_ref) <= bound * np.linalg.norm(x_ref)
