"""GPU parity of GS(p) and SpMV against the CPU oracle, through the C ABI."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import EPS, gsk, random_csr, to_dev
from problems import cd, configs

pytestmark = pytest.mark.gpu

# GS: entries a_ij / ||a_i||_p; the kernel multiplies by the reciprocal of a
# norm summed in another order, so each entry may differ by a few ulp.
GS_RTOL = 1e-14


def _gs_case(sys_, p):
    import torch

    g = gsk()
    A, b = to_dev(g, sys_)
    d = torch.empty(sys_.n, dtype=torch.float64, device="cuda")
    g.gs_scale(A, b, p=p, d_out=d)
    val_or, b_or, d_or = oracle.gs_scale(sys_.rowptr, sys_.colidx, sys_.val, sys_.b, p)
    val = A.val.cpu().numpy()
    bb = b.cpu().numpy()
    assert np.all(np.abs(val - val_or) <= GS_RTOL * np.abs(val_or)), np.max(np.abs(val - val_or) / np.abs(val_or))
    assert np.all(np.abs(bb - b_or) <= GS_RTOL * np.abs(b_or) + 1e-300)
    assert np.allclose(d.cpu().numpy(), d_or, rtol=GS_RTOL, atol=0)


@pytest.mark.parametrize("p", [1.0, 2.0, math.inf, 3.5])
def test_gs_scale_c1(p):
    _gs_case(configs.c1(), p)


@pytest.mark.parametrize("p", [1.0, 2.0, math.inf])
def test_gs_scale_c2_small_ragged_tail(p):
    _gs_case(configs.c2(21), p)  # 9261 rows: 289 full tiles and a 13-row tail


@pytest.mark.parametrize("p", [2.0, 3.5])
def test_gs_scale_random_ragged_and_long_rows(p):
    rp, ci, va = random_csr(1000, 11, min_len=1, max_len=12, long_rows=(3, 500, 999), long_len=400)
    s = cd.System(1000, rp, ci, va, np.random.default_rng(2).normal(size=1000))
    _gs_case(s, p)


def test_gs_scale_extreme_magnitudes():
    s = configs.c1(20)
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    k = np.where(np.arange(s.n) % 3 == 0, 1000, np.where(np.arange(s.n) % 3 == 1, -1000, 0))
    s2 = cd.System(s.n, s.rowptr, s.colidx, np.ldexp(s.val, k[rows]), np.ldexp(s.b, k))
    for p in [1.0, 2.0, math.inf]:
        _gs_case(s2, p)


def _expect_error(sys_, status, p=2.0):
    import torch

    g = gsk()
    A, b = to_dev(g, sys_)
    before = A.val.clone(), b.clone()
    with pytest.raises(g.GskError) as ei:
        g.gs_scale(A, b, p=p)
    assert ei.value.status == status
    # nothing modified (bitwise, so NaN entries compare equal to themselves)
    assert A.val.view(torch.int64).equal(before[0].view(torch.int64))
    assert b.view(torch.int64).equal(before[1].view(torch.int64))


def test_gs_zero_row_is_an_error_and_leaves_input():
    s = configs.c1(10)
    val = s.val.copy()
    val[s.rowptr[37]:s.rowptr[38]] = 0.0
    _expect_error(cd.System(s.n, s.rowptr, s.colidx, val, s.b), gsk().ERR_ZERO_ROW)


def test_gs_nonfinite_is_an_error_and_leaves_input():
    s = configs.c1(10)
    val = s.val.copy()
    val[17] = np.inf
    _expect_error(cd.System(s.n, s.rowptr, s.colidx, val, s.b), gsk().ERR_NONFINITE)
    b = s.b.copy()
    b[5] = np.nan
    _expect_error(cd.System(s.n, s.rowptr, s.colidx, s.val, b), gsk().ERR_NONFINITE)


def test_gs_malformed_rowptr_is_an_error():
    s = configs.c1(10)
    rp = s.rowptr.copy()
    rp[40] = rp[41] + 3  # decreasing extent
    _expect_error(cd.System(s.n, rp, s.colidx, s.val, s.b), gsk().ERR_ARG)


def test_gs_bad_p_rejected():
    g = gsk()
    A, b = to_dev(g, configs.c1(4))
    with pytest.raises(g.GskError):
        g.gs_scale(A, b, p=0.5)


# ------------------------------------------------------------------ SpMV
def _spmv_case(sys_, x):
    import torch

    g = gsk()
    A, _ = to_dev(g, sys_)
    xd = torch.as_tensor(x, device="cuda")
    y = torch.empty(sys_.n, dtype=torch.float64, device="cuda")
    g.gsk_spmv(A, xd, y)
    torch.cuda.synchronize()
    y_or = oracle.spmv(sys_.rowptr, sys_.colidx, sys_.val, x)
    rows = np.repeat(np.arange(sys_.n), np.diff(sys_.rowptr))
    absum = np.zeros(sys_.n)
    np.add.at(absum, rows, np.abs(sys_.val * x[sys_.colidx]))
    lens = np.diff(sys_.rowptr)
    assert np.all(np.abs(y.cpu().numpy() - y_or) <= (lens + 1) * EPS * absum)


def test_spmv_c1_and_c2_small():
    for s in [configs.c1(), configs.c2(21)]:
        _spmv_case(s, np.random.default_rng(3).normal(size=s.n))


def test_spmv_random_with_empty_and_long_rows():
    rp, ci, va = random_csr(777, 5, min_len=1, max_len=7, long_rows=(0, 400), long_len=500)
    # empty a few rows (SpMV allows empty rows)
    lens = np.diff(rp)
    keep = np.ones(len(ci), dtype=bool)
    for i in (10, 11, 776):
        keep[rp[i]:rp[i + 1]] = False
        lens[i] = 0
    rp2 = np.zeros_like(rp)
    rp2[1:] = np.cumsum(lens)
    s = cd.System(777, rp2, ci[keep], va[keep], np.zeros(777))
    _spmv_case(s, np.random.default_rng(4).normal(size=777))


def test_spmv_bad_column_index_is_reported():
    import torch

    g = gsk()
    s = configs.c1(10)
    ci = s.colidx.copy()
    ci[20] = s.n + 5
    A = g.Csr.from_host(s.rowptr, ci, s.val)
    x = torch.ones(s.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    ctx = g.Context(0)
    # the product skips the bad entry and the next solve reports the error
    g.gsk_spmv(A, x, y, ctx=ctx)
    torch.cuda.synchronize()
    with pytest.raises(g.GskError) as ei:
        g.bicgstab_solve(A, torch.ones_like(x), torch.zeros_like(x), tol=1e-8, ctx=ctx)
    assert ei.value.status == g.ERR_ARG
    ctx.close()


def test_spmv_full_c2_sampled_rows():
    """At the 128^3 size the product of sampled rows matches the oracle on
    those rows (rows are independent, so the oracle runs on the sub-matrix)."""
    import torch

    s = configs.c2(128)
    g = gsk()
    A, _ = to_dev(g, s)
    x = np.random.default_rng(8).normal(size=s.n)
    y = torch.empty(s.n, dtype=torch.float64, device="cuda")
    g.gsk_spmv(A, torch.as_tensor(x, device="cuda"), y)
    torch.cuda.synchronize()
    idx = np.unique(np.concatenate([np.random.default_rng(9).choice(s.n, 4000, replace=False), [0, s.n - 1]]))
    lens = s.rowptr[idx + 1] - s.rowptr[idx]
    sub_rp = np.zeros(len(idx) + 1, dtype=np.int32)
    sub_rp[1:] = np.cumsum(lens)
    gather = np.concatenate([np.arange(s.rowptr[i], s.rowptr[i + 1]) for i in idx])
    y_or = oracle.spmv(sub_rp, s.colidx[gather], s.val[gather], x)
    assert np.allclose(y.cpu().numpy()[idx], y_or, rtol=1e-13, atol=1e-12)
