"""Test helper: the paper's printed iteration tables for Problem 1 (Sec. 3,
Tables 1 and 1a) and Problem 4 (Sec. 6, Table 4 and the "limit" table),
read from the fixtures tests/golden/table1_p1_iterations.txt and
tests/golden/table4_p4_iterations.txt, and the bands within which a run
counts as matching them.

An entry is an int (iterations to reach the tolerance), "noconv" (no
convergence within 10,000 iterations) or ("stag", r) (restarted GMRES
stagnates at relative residual about r).
"""
from __future__ import annotations

import os

TOLS = (1e-4, 1e-7, 1e-10)
FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_p1_iterations.txt")


def _entry(tok: str):
    if tok == "noconv":
        return "noconv"
    if tok.startswith("stag:"):
        return ("stag", float(tok[5:]))
    return int(tok)


FIXTURE4 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table4_p4_iterations.txt")
CONVECTIONS = (100.0, 200.0, 500.0, 1000.0)


def load(path: str = FIXTURE) -> list[dict]:
    """Iteration-table rows (Tables 1, 1a and 4)."""
    rows = []
    for ln in open(path):
        if not ln.strip() or ln.startswith("#"):
            continue
        t = ln.split()
        if t[0] == "limit":
            continue
        rows.append({"table": t[0], "case": t[1], "solver": t[2], "m": None if t[3] == "-" else int(t[3]),
                     "scaling": t[4], "precond": t[5], "entries": dict(zip(TOLS, (_entry(x) for x in t[6:9])))})
    return rows


def load_limit(path: str = FIXTURE4) -> list[dict]:
    """Rows of the "limit" table (Sec. 6): the best goal reached (a tolerance
    of TOLS, or None) per convection strength."""
    rows = []
    for ln in open(path):
        t = ln.split()
        if not t or t[0] != "limit":
            continue
        rows.append({"solver": t[1], "m": None if t[2] == "-" else int(t[2]), "scaling": t[3], "precond": t[4],
                     "best": dict(zip(CONVECTIONS, (None if x == "none" else float(x) for x in t[5:9])))})
    return rows


def band(solver: str, printed: int) -> tuple[int, int]:
    """Iteration counts that match a printed count: GMRES within 1% (+-3),
    Bi-CGSTAB within 20% (its counts move by that much under 1-ulp changes
    of b on these systems)."""
    if solver == "gmres":
        d = max(3, int(0.01 * printed + 0.5))
    else:
        d = max(5, int(0.20 * printed + 0.5))
    return printed - d, printed + d


def matches(solver: str, printed, conv: bool, iters: int, relres: float) -> bool:
    """Does a run (converged?, iterations, final relative residual) match a
    printed entry?  A stagnation entry matches a run that did not converge
    and ended within a factor 2.5 of the printed residual."""
    if printed == "noconv":
        return not conv
    if isinstance(printed, tuple):
        return (not conv) and printed[1] / 2.5 <= relres <= printed[1] * 2.5
    lo, hi = band(solver, printed)
    return conv and lo <= iters <= hi
