"""Writes table4_bicgstab_ensembles.json: the oracle's rounding ensembles of
the GS-scaled Bi-CGSTAB rows of Table 4 (Problem 4, 80^3, D = 1e4 and 1e6,
with and without ILU(0); Sec. 6).

On these systems Bi-CGSTAB's iteration count at a tight tolerance is
decided by rounding: the same method on the same system with b changed by
at most one ulp (b (1 + u eps), u uniform in [-1, 1], seeds 1..15, plus the
unperturbed b) reaches the tolerance after quite different numbers of
iterations.  The GPU test accepts a count inside this recorded spread as
well as inside the band around the printed count.  Calls only oracle/ and
problems/.  16 members per row and tolerance; a few minutes on 8 cores.
"""
import json
import os
import sys
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

SIZE = 16
TOLS = (1e-4, 1e-7, 1e-10)
ROWS = [("p4_D1e4", "none"), ("p4_D1e4", "ilut"), ("p4_D1e6", "none"), ("p4_D1e6", "ilut")]
_SYS = {}


def _system(case, precond):
    import oracle
    from problems import configs

    key = (case, precond)
    if key not in _SYS:
        s = configs.p4(80, D=1.0e4 if case == "p4_D1e4" else 1.0e6)
        val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
        lu = oracle.ilu0(s.rowptr, s.colidx, val) if precond == "ilut" else None
        _SYS[key] = (s, val, b, lu)
    return _SYS[key]


def _member(job):
    import numpy as np

    import oracle

    case, precond, tol, seed = job
    s, val, b, lu = _system(case, precond)
    if seed:
        u = np.random.default_rng(seed).uniform(-1.0, 1.0, s.n)
        b = b * (1.0 + u * np.finfo(np.float64).eps)
    info = oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=tol, maxit=10000, refresh=0, lu=lu)[1]
    return job, int(info["conv"]), int(info["iters"])


def main():
    jobs = [(c, p, t, seed) for c, p in ROWS for t in TOLS for seed in range(SIZE)]
    out = {}
    with get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        for (c, p, t, seed), conv, iters in pool.imap_unordered(_member, jobs):
            e = out.setdefault(f"{c} {p} {t:g}", {"conv": [None] * SIZE, "iters": [None] * SIZE})
            e["conv"][seed] = conv
            e["iters"][seed] = iters
    for k, e in out.items():
        e["min"], e["max"] = min(e["iters"]), max(e["iters"])
    with open(os.path.join(HERE, "table4_bicgstab_ensembles.json"), "w") as f:
        json.dump(dict(sorted(out.items())), f, indent=1)
    for k, e in sorted(out.items()):
        print(k, e["min"], e["max"], sorted(e["iters"]), set(e["conv"]))


if __name__ == "__main__":
    main()
