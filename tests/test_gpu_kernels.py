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


def _expect_error(sys_, status, bad_rows, p=2.0):
    """gs_scale reports `status`; the rows that caused it (and their b
    entries) are left bit-for-bit as they were, every other row is scaled as
    the oracle scales it."""
    import torch

    g = gsk()
    A, b = to_dev(g, sys_)
    with pytest.raises(g.GskError) as ei:
        g.gs_scale(A, b, p=p)
    assert ei.value.status == status
    val, bb = A.val.cpu().numpy(), b.cpu().numpy()
    bad = np.zeros(sys_.n, dtype=bool)
    bad[list(bad_rows)] = True
    rows = np.repeat(np.arange(sys_.n), np.diff(sys_.rowptr))
    same = bad[rows]
    # bitwise, so NaN entries compare equal to themselves
    assert np.array_equal(val[same].view(np.int64), sys_.val[same].view(np.int64))
    assert np.array_equal(bb[bad].view(np.int64), sys_.b[bad].view(np.int64))
    # the good rows: as the oracle scales them (it works row by row)
    good = ~bad
    keep = good[rows]
    sub_rp = np.zeros(good.sum() + 1, dtype=np.int32)
    sub_rp[1:] = np.cumsum(np.diff(sys_.rowptr)[good])
    v_or, b_or, _ = oracle.gs_scale(sub_rp, sys_.colidx[keep], sys_.val[keep], sys_.b[good], p)
    assert np.all(np.abs(val[keep] - v_or) <= GS_RTOL * np.abs(v_or))
    assert np.all(np.abs(bb[good] - b_or) <= GS_RTOL * np.abs(b_or) + 1e-300)


def test_gs_zero_row_is_an_error_and_only_that_row_is_left():
    s = configs.c1(10)
    val = s.val.copy()
    val[s.rowptr[37]:s.rowptr[38]] = 0.0
    _expect_error(cd.System(s.n, s.rowptr, s.colidx, val, s.b), gsk().ERR_ZERO_ROW, [37])


def test_gs_nonfinite_is_an_error_and_only_that_row_is_left():
    s = configs.c1(10)
    val = s.val.copy()
    val[17] = np.inf
    row17 = int(np.searchsorted(s.rowptr, 17, side="right") - 1)
    _expect_error(cd.System(s.n, s.rowptr, s.colidx, val, s.b), gsk().ERR_NONFINITE, [row17])
    b = s.b.copy()
    b[5] = np.nan
    _expect_error(cd.System(s.n, s.rowptr, s.colidx, s.val, b), gsk().ERR_NONFINITE, [5])


def test_gs_malformed_rowptr_is_an_error():
    g = gsk()
    s = configs.c1(10)
    rp = s.rowptr.copy()
    rp[40] = rp[41] + 3  # decreasing extent
    A, b = to_dev(g, cd.System(s.n, rp, s.colidx, s.val, s.b))
    with pytest.raises(g.GskError) as ei:
        g.gs_scale(A, b, p=2.0)
    assert ei.value.status == g.ERR_ARG


@pytest.mark.parametrize("p", [1.0, 2.0, math.inf, 3.5])
def test_gs_scale_rows_across_the_exponent_range(p):
    """Rows scaled by 2^k with k spread over [-1000, 1000]: the one-pass
    reciprocal (FP32 seed, FP64 correction) and the rescaled slow path for
    rows near the ends of the range both match the oracle's division."""
    s = configs.c1(24)
    k = np.random.default_rng(12).integers(-1000, 1001, s.n)
    k[:8] = [-1000, -999, -480, -479, 479, 480, 999, 1000]
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    _gs_case(cd.System(s.n, s.rowptr, s.colidx, np.ldexp(s.val, k[rows]), np.ldexp(s.b, k)), p)


def test_gs_bad_p_rejected():
    g = gsk()
    A, b = to_dev(g, configs.c1(4))
    with pytest.raises(g.GskError):
        g.gs_scale(A, b, p=0.5)


def test_profiled_gs_scale_is_gs_scale():
    # the profiling entry runs the same kernel: bitwise the same results, and
    # the kernel's own device time
    import torch

    g = gsk()
    s = configs.c2(21)
    A1, b1 = to_dev(g, s)
    A2, b2 = to_dev(g, s)
    d1 = torch.empty(s.n, dtype=torch.float64, device="cuda")
    d2 = torch.empty_like(d1)
    g.gs_scale(A1, b1, p=2.0, d_out=d1)
    ms = g.profile_gs_scale(A2, b2, p=2.0, d_out=d2)
    assert ms > 0.0
    assert torch.equal(A1.val, A2.val) and torch.equal(b1, b2) and torch.equal(d1, d2)
    val = s.val.copy()
    val[s.rowptr[5]:s.rowptr[6]] = 0.0
    A3, b3 = to_dev(g, cd.System(s.n, s.rowptr, s.colidx, val, s.b))
    with pytest.raises(g.GskError) as ei:
        g.profile_gs_scale(A3, b3, p=2.0)
    assert ei.value.status == g.ERR_ZERO_ROW


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


# The product streams 256-row chunks of the matrix into shared-memory stages
# of 1856 nonzeros; on the matrix's last chunk the copy ends at a 16-byte
# boundary and the last few entries are loaded one by one.  These cases put
# that last chunk at 1855..1859 nonzeros, behind a first chunk of odd length
# (so its start is not aligned either), in FP64 and FP32.
PIPE_CAP = 1856


def _chunk_case(last_nnz, first_nnz, seed):
    rs = np.random.default_rng(seed)
    lens = []
    for total in ([first_nnz] if first_nnz else []) + [last_nnz]:
        base, extra = divmod(total, 256)
        ln = np.full(256, base)
        ln[rs.choice(256, extra, replace=False)] += 1
        lens.append(ln)
    lens = np.concatenate(lens)
    n = len(lens)
    rp = np.zeros(n + 1, dtype=np.int32)
    rp[1:] = np.cumsum(lens)
    ci = np.concatenate([np.sort(rs.choice(n, L, replace=False)) for L in lens]).astype(np.int32)
    va = rs.uniform(-1, 1, len(ci))
    return cd.System(n, rp, ci, va, np.zeros(n))


@pytest.mark.parametrize("last_nnz", [PIPE_CAP - 1, PIPE_CAP, PIPE_CAP + 1, PIPE_CAP + 2, PIPE_CAP + 3])
@pytest.mark.parametrize("first_nnz", [0, 1001])
def test_spmv_last_chunk_at_the_stage_capacity(last_nnz, first_nnz):
    s = _chunk_case(last_nnz, first_nnz, seed=last_nnz + first_nnz)
    assert s.rowptr[-1] == last_nnz + first_nnz
    _spmv_case(s, np.random.default_rng(5).normal(size=s.n))


@pytest.mark.parametrize("last_nnz", [PIPE_CAP - 1, PIPE_CAP + 1, PIPE_CAP + 3])
def test_spmv_fp32_last_chunk_at_the_stage_capacity(last_nnz):
    import torch

    s = _chunk_case(last_nnz, 1001, seed=7 * last_nnz)
    g = gsk()
    A = g.Csr.from_host(s.rowptr, s.colidx, s.val.astype(np.float32), device="cuda", dtype=torch.float32)
    x = np.random.default_rng(6).normal(size=s.n).astype(np.float32)
    y = torch.empty(s.n, dtype=torch.float32, device="cuda")
    g.gsk_spmv(A, torch.as_tensor(x, device="cuda"), y)
    torch.cuda.synchronize()
    v32 = s.val.astype(np.float32).astype(np.float64)
    y_or = oracle.spmv(s.rowptr, s.colidx, v32, x.astype(np.float64))
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    absum = np.zeros(s.n)
    np.add.at(absum, rows, np.abs(v32 * x.astype(np.float64)[s.colidx]))
    lens = np.diff(s.rowptr)
    feps = float(np.finfo(np.float32).eps)
    assert np.all(np.abs(y.cpu().numpy().astype(np.float64) - y_or) <= (lens + 2) * feps * absum)


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
