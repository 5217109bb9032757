"""The allocation-free GS(p) entry point (gs_scale_static), for callers that
may not allocate device memory, against gs_scale through the C ABI.

Collected last on purpose: it checks that repeated calls reuse the library's
built-in scratch array correctly, after (and independently of) every other
test."""
import math

import numpy as np
import pytest

from gpu_util import gsk, to_dev
from problems import cd, configs

pytestmark = pytest.mark.gpu

RTOL = 1e-14  # the GS parity tolerance used by the other GPU tests


def _pair(sys_, p, with_d):
    import torch

    g = gsk()
    A1, b1 = to_dev(g, sys_)
    A2, b2 = to_dev(g, sys_)
    d1 = torch.empty(sys_.n, dtype=torch.float64, device="cuda")
    d2 = torch.empty(sys_.n, dtype=torch.float64, device="cuda") if with_d else None
    g.gs_scale(A1, b1, p=p, d_out=d1)
    g.gs_scale_static(A2, b2, p=p, d_out=d2)
    for got, want in [(A2.val, A1.val), (b2, b1)] + ([(d2, d1)] if with_d else []):
        got, want = got.cpu().numpy(), want.cpu().numpy()
        assert np.all(np.abs(got - want) <= RTOL * np.abs(want))
        # the two entry points share the per-row arithmetic: in fact bit-identical
        assert np.array_equal(got.view(np.int64), want.view(np.int64))


@pytest.mark.parametrize("p", [1.0, 2.0, math.inf, 3.5])
def test_static_matches_gs_scale_twice_in_a_row(p):
    s = configs.c2(21)  # 9261 rows, ragged last tile
    _pair(s, p, with_d=False)
    _pair(s, p, with_d=False)  # second call reuses the array left by the first
    _pair(configs.c1(), p, with_d=True)


def test_static_errors_and_limit():
    import torch

    g = gsk()
    s = configs.c1(10)
    val = s.val.copy()
    val[s.rowptr[5]:s.rowptr[6]] = 0.0
    A, b = to_dev(g, cd.System(s.n, s.rowptr, s.colidx, val, s.b))
    before = A.val.clone(), b.clone()
    with pytest.raises(g.GskError) as ei:
        g.gs_scale_static(A, b, p=2.0)
    assert ei.value.status == g.ERR_ZERO_ROW
    # on error nothing is modified (compared bitwise)
    assert A.val.view(torch.int64).equal(before[0].view(torch.int64))
    assert b.view(torch.int64).equal(before[1].view(torch.int64))
    # a non-finite b entry: ERR_NONFINITE, A and b again untouched
    bad_b = s.b.copy()
    bad_b[3] = np.inf
    A, b = to_dev(g, cd.System(s.n, s.rowptr, s.colidx, s.val, bad_b))
    before = A.val.clone(), b.clone()
    with pytest.raises(g.GskError) as ei:
        g.gs_scale_static(A, b, p=2.0)
    assert ei.value.status == g.ERR_NONFINITE
    assert A.val.view(torch.int64).equal(before[0].view(torch.int64))
    assert b.view(torch.int64).equal(before[1].view(torch.int64))
    # the error word is cleared by the next call: a good matrix scales fine
    _pair(configs.c1(10), 2.0, with_d=False)
    # more rows than the built-in array holds, without d_out: rejected
    n = (1 << 20) + 1
    big = g.Csr(torch.zeros(n + 1, dtype=torch.int32, device="cuda"),
                torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, dtype=torch.float64, device="cuda"))
    with pytest.raises(g.GskError) as ei:
        g.gs_scale_static(big, None, p=2.0)
    assert ei.value.status == g.ERR_ARG
