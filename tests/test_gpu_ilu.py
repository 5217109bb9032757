"""ILU(0) on the GPU (the paper's ILUT with drop tolerance 0 and fill-in 1,
which it found to act as ILU(0), Sec. 2) against the CPU oracle, through the
C ABI: the application z = (LU)^-1 r, the errors of the factorisation, the
right-preconditioned Bi-CGSTAB and GMRES(m), and the paper's ILUT rows of
Tables 1 and 1a (fixture tests/golden/table1_p1_iterations.txt)."""
import numpy as np
import pytest

import oracle
import paper_tables as pt
from gpu_util import gsk, random_csr, to_dev
from problems import cd, configs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["c1", "c2_21", "random"])
def test_ilu0_apply_matches_oracle(case):
    import torch

    g = gsk()
    if case == "c1":
        s = configs.c1()
    elif case == "c2_21":
        s = configs.c2(21)
    else:
        rp, ci, va = random_csr(4000, 11, long_rows=(5, 2000), long_len=200)
        s = cd.System(4000, rp, ci, va, np.ones(4000))
    A, _ = to_dev(g, s)
    M = g.Ilu0(A)
    lu = oracle.ilu0(s.rowptr, s.colidx, s.val)
    for seed in (0, 1):
        r = np.random.default_rng(seed).normal(size=s.n)
        z = M.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
        z_or = oracle.ilu0_apply(s.rowptr, s.colidx, lu, r)
        # the same recurrences, rounded with FMAs on the GPU
        assert np.allclose(z, z_or, rtol=1e-11, atol=1e-13 * np.abs(z_or).max()), np.abs(z - z_or).max()
    M.close()


def test_ilu0_errors():
    g = gsk()
    s = configs.c1(8)
    # a row without its diagonal
    keep = np.ones(len(s.colidx), dtype=bool)
    r0 = slice(s.rowptr[3], s.rowptr[4])
    keep[np.arange(len(s.colidx))[r0][s.colidx[r0] == 3]] = False
    rp = np.concatenate([[0], np.cumsum([np.count_nonzero(keep[s.rowptr[i]:s.rowptr[i + 1]])
                                         for i in range(s.n)])]).astype(np.int32)
    A = g.Csr.from_host(rp, s.colidx[keep], s.val[keep])
    with pytest.raises(g.GskError) as e:
        g.Ilu0(A)
    assert e.value.status == g.ERR_ARG
    # unsorted columns in a row
    ci = s.colidx.copy()
    ci[s.rowptr[2]], ci[s.rowptr[2] + 1] = ci[s.rowptr[2] + 1], ci[s.rowptr[2]]
    with pytest.raises(g.GskError) as e:
        g.Ilu0(g.Csr.from_host(s.rowptr, ci, s.val))
    assert e.value.status == g.ERR_ARG
    # a zero pivot
    val = s.val.copy()
    val[(s.colidx == 0) & (np.arange(len(val)) < s.rowptr[1])] = 0.0
    with pytest.raises(g.GskError) as e:
        g.Ilu0(g.Csr.from_host(s.rowptr, s.colidx, val))
    assert e.value.status == g.ERR_ZERO_ROW
    # FP32 matrices are not factored
    with pytest.raises(g.GskError) as e:
        g.Ilu0(g.Csr.from_host(s.rowptr, s.colidx, s.val, dtype=__import__("torch").float32))
    assert e.value.status == g.ERR_ARG


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
@pytest.mark.parametrize("scaled", [False, True])
def test_preconditioned_solvers_match_oracle(solver, scaled):
    import torch

    g = gsk()
    s = configs.c1()
    if scaled:
        val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
        s = cd.System(s.n, s.rowptr, s.colidx, val, b, s.x_true)
    lu = oracle.ilu0(s.rowptr, s.colidx, s.val)
    A, b = to_dev(g, s)
    M = g.Ilu0(A)
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    o = g.opts(precond=M, refresh=0)
    tol = 1e-10
    if solver == "gmres":
        info = g.gmres_solve(A, b, x, m=20, tol=tol, options=o)
        _, io = oracle.gmres(s.rowptr, s.colidx, s.val, s.b, m=20, tol=tol, lu=lu)
    else:
        info = g.bicgstab_solve(A, b, x, tol=tol, options=o)
        _, io = oracle.bicgstab(s.rowptr, s.colidx, s.val, s.b, tol=tol, refresh=0, lu=lu)
    assert info["conv"] == io["conv"] == 0, (info, io)
    assert abs(info["iters"] - io["iters"]) <= max(2, 0.05 * io["iters"]), (info["iters"], io["iters"])
    xh = x.cpu().numpy()
    assert oracle.relres(s.rowptr, s.colidx, s.val, s.b, xh) < tol
    # ILU(0) needs far fewer iterations than no preconditioner
    x0 = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    plain = (g.gmres_solve(A, b, x0, m=20, tol=tol) if solver == "gmres"
             else g.bicgstab_solve(A, b, x0, tol=tol))
    assert info["iters"] < plain["iters"] / 2
    M.close()


def _table_cases():
    out = []
    for r in pt.load():
        if r["precond"] != "ilut":
            continue
        seen = False
        for tol in pt.TOLS:
            e = r["entries"][tol]
            if not isinstance(e, int):
                if seen:
                    continue
                seen = True
            out.append(pytest.param(r, tol, id=f"{r['table']}-{r['case']}-{r['solver']}-{r['scaling']}-{tol:g}"))
    return out


@pytest.mark.parametrize("row,tol", _table_cases())
def test_gpu_ilu_matches_printed_table(row, tol):
    g = gsk()
    from paper_0812_2769_gb300 import reproduce

    s = configs.p1(128) if row["case"] == "inner1e3" else configs.p1(128, continuous=1000.0)
    conv, iters, relres, _ = reproduce.solve_case(g, s, row["solver"], row["scaling"] == "gs", tol,
                                                  m=row["m"] or 10, precond=True)
    assert pt.matches(row["solver"], row["entries"][tol], conv, iters, relres), (row["entries"][tol], conv, iters,
                                                                                 relres)


@pytest.mark.parametrize("case", ["c1", "c2_21", "random", "p1_128"])
def test_one_block_sweep_is_bit_identical_to_the_grid_sweep(case, monkeypatch):
    """Systems whose z fits in shared memory are swept by one thread block
    (a level ends at a block barrier): the same per-row arithmetic in the
    same order as the grid sweep, so the results are bit-identical."""
    import torch

    g = gsk()
    if case == "c1":
        s = configs.c1()
    elif case == "c2_21":
        s = configs.c2(21)
    elif case == "p1_128":
        s = configs.p1(128)
    else:
        rp, ci, va = random_csr(4000, 11, long_rows=(5, 2000), long_len=200)
        s = cd.System(4000, rp, ci, va, np.ones(4000))
    A, _ = to_dev(g, s)
    monkeypatch.delenv("GSK_ILU_SWEEP", raising=False)
    M1 = g.Ilu0(A)
    monkeypatch.setenv("GSK_ILU_SWEEP", "grid")
    M2 = g.Ilu0(A)
    i1, i2 = M1.info(), M2.info()
    assert i1["one_block"] and not i2["one_block"]
    assert i1["levels_lower"] == i2["levels_lower"] > 1
    for seed in (0, 1):
        r = torch.as_tensor(np.random.default_rng(seed).normal(size=s.n), device="cuda")
        assert torch.equal(M1.apply(r), M2.apply(r))
    M1.close()
    M2.close()


def test_large_systems_take_the_grid_sweep():
    g = gsk()
    s = configs.c2(40)  # z of 64,000 rows does not fit in one block's shared memory
    A, _ = to_dev(g, s)
    M = g.Ilu0(A)
    assert not M.info()["one_block"]
    M.close()
