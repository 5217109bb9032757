"""Test helper: the paper's printed iteration tables for Problem 1 (Sec. 3,
Tables 1 and 1a), read from the fixture tests/golden/table1_p1_iterations.txt,
and the bands within which a run counts as matching them.

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


def load(path: str = FIXTURE) -> list[dict]:
    rows = []
    for ln in open(path):
        if not ln.strip() or ln.startswith("#"):
            continue
        t = ln.split()
        rows.append({"table": t[0], "case": t[1], "solver": t[2], "m": None if t[3] == "-" else int(t[3]),
                     "scaling": t[4], "precond": t[5], "entries": dict(zip(TOLS, (_entry(x) for x in t[6:9])))})
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
