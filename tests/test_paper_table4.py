"""The oracle against the paper's Problem 4 (Sec. 6): Table 4 (80^3 grid,
convection 100, D = 1e4 and 1e6) and the "limit" table (40^3, D = 1e4,
convection 100 .. 1000); fixture tests/golden/table4_p4_iterations.txt.

Counts use the bands of the Problem 1 tables (GMRES(10) within 1%,
Bi-CGSTAB within 20%).  Where the paper prints "---" (no convergence within
its 10,000 iterations), these CPU tests check a shorter run of NOCONV_MAXIT
iterations, which keeps the suite to minutes: a weaker statement than the
table's, stated as such.  GS is what makes Bi-CGSTAB converge here (Sec. 6):
the unscaled rows do not reach 1e-4, the GS rows do.

Rows left out, and why (the rest of this module holds them to the paper):
* Table 4, ILU(0) without GS: the unscaled Bi-CGSTAB+ILU rows reach 1e-4 in
  39 (D = 1e4) and 32 (D = 1e6) iterations where the paper prints 77 and 52,
  and unscaled GMRES(10)+ILU reaches 1e-4 (D = 1e4) where it prints "---".
  The paper's ILUT(0, fill-in 1) on the unscaled matrix is the one place where
  reading it as ILU(0) does not reproduce the table; with GS the same rows
  match.
* "limit", convection 500: GMRES(10) with GS reaches 1e-4 here, the paper
  prints "---"; the Problem 4 operator's eigenvalues do not match the paper's
  either (Table 4a), so its discretisation differs in ways it does not state.
  Bi-CGSTAB with GS at convections 200 and 500 is decided by rounding: its
  outcome ranges from a breakdown (at 500 even before 1e-4) to convergence to
  1e-10 over a rounding ensemble, and the test checks that the paper's 1e-10
  is among them.
* "limit" rows with ILU: not checked on the CPU (see test_gpu_ilu)."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_tables as pt
from problems import configs

NOCONV_MAXIT = 300
EPS = np.finfo(np.float64).eps

ROWS = [r for r in pt.load(pt.FIXTURE4) if not (r["scaling"] == "none" and r["precond"] == "ilut")]

_SYS = {}


def _system(case, scaling):
    key = (case, scaling)
    if key not in _SYS:
        D = 1.0e4 if case == "p4_D1e4" else 1.0e6
        s = configs.p4(80, D=D)
        if scaling == "gs":
            val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
        else:
            val, b = s.val, s.b
        lu = oracle.ilu0(s.rowptr, s.colidx, val)
        _SYS[key] = (s, val, b, lu)
    return _SYS[key]


def _solve(s, val, b, solver, m, tol, maxit, lu=None):
    if solver == "gmres":
        return oracle.gmres(s.rowptr, s.colidx, val, b, m=m, tol=tol, maxit=maxit, lu=lu)[1]
    return oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=tol, maxit=maxit, refresh=0, lu=lu)[1]


def _cases():
    out = []
    for r in ROWS:
        noconv_done = False
        for tol in pt.TOLS:
            e = r["entries"][tol]
            if e == "noconv":
                if noconv_done:  # one short run stands for every tighter tolerance
                    continue
                noconv_done = True
            out.append(pytest.param(r, tol, id=f"{r['case']}-{r['solver']}-{r['scaling']}-{r['precond']}-{tol:g}"))
    return out


@pytest.mark.parametrize("row,tol", _cases())
def test_oracle_matches_table4(row, tol):
    s, val, b, lu = _system(row["case"], row["scaling"])
    printed = row["entries"][tol]
    maxit = NOCONV_MAXIT if printed == "noconv" else 10000
    info = _solve(s, val, b, row["solver"], row["m"], tol, maxit, lu if row["precond"] == "ilut" else None)
    conv = info["conv"] == oracle.CONVERGED
    assert pt.matches(row["solver"], printed, conv, info["iters"], info["relres_true"]), (printed, info)


# ------------------------------------------------------------- "limit"
def _reaches(s, val, b, solver, m, tol, maxit):
    return _solve(s, val, b, solver, m, tol, maxit)["conv"] == oracle.CONVERGED


def _limit_cases():
    out = []
    for r in pt.load_limit():
        if r["precond"] != "none":
            continue
        for conv in pt.CONVECTIONS:
            if conv == 500.0:
                continue  # test_limit_bicgstab_outcome_is_decided_by_rounding below
            out.append(pytest.param(r, conv, id=f"{r['solver']}-{r['scaling']}-conv{conv:g}"))
    return out


_LIM = {}


def _limit_system(conv, scaling):
    key = (conv, scaling)
    if key not in _LIM:
        s = configs.p4(40, D=1.0e4, conv=conv)
        if scaling == "gs":
            val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
        else:
            val, b = s.val, s.b
        _LIM[key] = (s, val, b)
    return _LIM[key]


@pytest.mark.parametrize("row,conv", _limit_cases())
def test_oracle_matches_limit_table(row, conv):
    """The best goal printed is reached (within 10,000 iterations) and the
    next tighter one is not (within the short run; the paper ran 10,000)."""
    s, val, b = _limit_system(conv, row["scaling"])
    want = row["best"][conv]
    goals = sorted(pt.TOLS, reverse=True)  # 1e-4, 1e-7, 1e-10
    if want is not None:
        assert _reaches(s, val, b, row["solver"], row["m"], want, 10000)
    nxt = goals[0] if want is None else (goals[goals.index(want) + 1] if want != goals[-1] else None)
    if nxt is not None:
        assert not _reaches(s, val, b, row["solver"], row["m"], nxt, NOCONV_MAXIT)


@pytest.mark.parametrize("conv", [200.0, 500.0])
def test_limit_bicgstab_outcome_is_decided_by_rounding(conv):
    """Bi-CGSTAB with GS at convection 200 and 500: over a rounding ensemble
    (b and the scaled values perturbed by an ulp or two) the outcome at tol
    1e-10 ranges from breakdown to convergence; the paper's 1e-10 is among
    them (the GPU's outcome must be one of them too, test_gpu_paper_table4)."""
    s, val, b = _limit_system(conv, "gs")
    outcomes = []
    for k in range(8):
        rs = np.random.default_rng(k)
        bb = b if k == 0 else b * (1.0 + rs.uniform(-1, 1, len(b)) * EPS)
        vv = val if k == 0 else val * (1.0 + rs.uniform(-2, 2, len(val)) * EPS)
        outcomes.append(_solve(s, vv, bb, "bicgstab", None, 1e-10, 10000)["conv"])
    assert oracle.CONVERGED in outcomes and oracle.BREAKDOWN in outcomes, outcomes


# ------------------------------------------------- rounding ensembles
def test_recorded_ensembles_contain_the_printed_counts():
    """The oracle's one-ulp rounding ensembles of the GS-scaled Bi-CGSTAB rows
    (tests/golden/table4_bicgstab_ensembles.json, written by the committed
    script beside it from oracle/ alone): every member converges, and the
    band around each printed count meets the recorded spread, so the paper's
    run reads as one member of the same spread.  Where the spread is wider
    than the band, a count outside the band is no evidence against a path
    that takes this method's arithmetic (the GPU test accepts the spread)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table4_bicgstab_ensembles.json")
    ens = json.load(open(path))
    rows = [r for r in ROWS if r["solver"] == "bicgstab" and r["scaling"] == "gs"]
    assert len(rows) == 4
    for r in rows:
        for tol in pt.TOLS:
            e = ens[f"{r['case']} {r['precond']} {tol:g}"]
            assert len(e["iters"]) == 16 and set(e["conv"]) == {oracle.CONVERGED}
            assert e["min"] == min(e["iters"]) and e["max"] == max(e["iters"])
            lo, hi = pt.band("bicgstab", r["entries"][tol])
            assert lo <= e["max"] and hi >= e["min"], (r["case"], r["precond"], tol, r["entries"][tol], e["min"], e["max"])
