"""The oracle against the paper's printed iteration counts for Problem 1
(Sec. 3, Tables 1 and 1a; fixture tests/golden/table1_p1_iterations.txt):
128x128 grid, b = A (1,...,1)^T, x0 = 0, maxit 10,000, the GS(2)-scaled
relative residual as the stopping metric, GMRES(10) and Bi-CGSTAB without
and with GS(2), without a preconditioner and with ILU(0) (the paper's
ILUT(0, fill-in 1), which it found to act as ILU(0)).

These pin the oracle's whole solve (discretisation of Problem 1, GS,
GMRES(m) with CGS2, Bi-CGSTAB, the stopping rule) to numbers the paper
prints: restarted GMRES reproduces its counts to within 1%, and its
stagnation levels; Bi-CGSTAB within 20% (its counts move by that much under
rounding changes on these systems)."""
import pytest

import oracle
import paper_tables as pt
from problems import configs

ROWS = pt.load()


def _system(case):
    return configs.p1(128) if case == "inner1e3" else configs.p1(128, continuous=1000.0)


_CACHE = {}


def _scaled(case, scaling):
    key = (case, scaling)
    if key not in _CACHE:
        s = _system(case)
        if scaling == "gs":
            val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
        else:
            val, b = s.val, s.b
        _CACHE[key] = (s, val, b)
    return _CACHE[key]


_LU = {}


def _run(row, tol):
    s, val, b = _scaled(row["case"], row["scaling"])
    lu = None
    if row.get("precond", "none") == "ilut":  # ILUT(0, fill 1) acts as ILU(0), Sec. 2
        key = (row["case"], row["scaling"])
        if key not in _LU:
            _LU[key] = oracle.ilu0(s.rowptr, s.colidx, val)
        lu = _LU[key]
    if row["solver"] == "gmres":
        _, info = oracle.gmres(s.rowptr, s.colidx, val, b, m=row["m"], tol=tol, maxit=10000, lu=lu)
    else:
        _, info = oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=tol, maxit=10000, refresh=0, lu=lu)
    return info


def _cases():
    out = []
    for r in ROWS:
        done_stag = False
        for tol in pt.TOLS:
            e = r["entries"][tol]
            # one run stands for every tolerance at which the paper reports
            # no convergence / the same stagnation level
            if not isinstance(e, int):
                if done_stag:
                    continue
                done_stag = True
            out.append(pytest.param(r, tol, id=f"{r['table']}-{r['case']}-{r['solver']}-{r['scaling']}-"
                                              f"{r['precond']}-{tol:g}"))
    return out


@pytest.mark.parametrize("row,tol", _cases())
def test_oracle_matches_printed_table(row, tol):
    info = _run(row, tol)
    printed = row["entries"][tol]
    conv = info["conv"] == 0
    assert pt.matches(row["solver"], printed, conv, info["iters"], info["relres_true"]), (printed, info)


def test_gs_is_what_makes_bicgstab_converge_on_problem_1():
    # Sec. 3: "GS enables the convergence of Bi-CGSTAB without ILUT"
    none = _run({"case": "inner1e3", "scaling": "none", "solver": "bicgstab"}, 1e-4)
    gs = _run({"case": "inner1e3", "scaling": "gs", "solver": "bicgstab"}, 1e-10)
    assert none["conv"] != 0 and gs["conv"] == 0


def test_band_and_match_rules():
    assert pt.band("gmres", 265) == (262, 268)
    assert pt.band("bicgstab", 91) == (73, 109)
    assert pt.matches("gmres", ("stag", 1.1e-5), False, 10000, 1.06e-5)
    assert not pt.matches("gmres", ("stag", 1.1e-5), True, 300, 9e-8)
    assert not pt.matches("bicgstab", "noconv", True, 85, 9e-5)
    assert pt.matches("bicgstab", 299, True, 308, 9e-8)
