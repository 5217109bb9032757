"""Writes c2_oracle_counts.json: the oracle's own iteration counts and wall
times for the 128^3 workload (GS(2), tol 1e-8) with Bi-CGSTAB and GMRES(30).

The benchmark's CPU-baseline leg times a bounded sample of oracle iterations
and scales it by these counts to a per-solve time.  Calls only oracle/ and
problems/.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from problems import configs  # noqa: E402


def main():
    s = configs.c2(128)
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    out = {"workload": "c2 128^3 GS(2) tol 1e-8", "n": s.n, "nnz": s.nnz}
    t = time.time()
    _, ib = oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=1e-8)
    out["bicgstab"] = dict(ib, seconds=time.time() - t)
    t = time.time()
    _, ig = oracle.gmres(s.rowptr, s.colidx, val, b, m=30, tol=1e-8)
    out["gmres30"] = dict(ig, seconds=time.time() - t)
    with open(os.path.join(HERE, "c2_oracle_counts.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
