"""Writes c3_oracle_trace.json: the oracle on the 256^3 configuration
(16,777,216 unknowns; a = 10^U[-3,3] on an 8^3 partition, convection
U[-30,30]^3 per cell; GS(2); tol 1e-10), for the GPU parity test of that
configuration:

* GMRES(30), the first two cycles (60 Arnoldi steps): the least-squares
  residual estimate after every step and the true metric after each cycle.
* Bi-CGSTAB to tol 1e-10 (maxit 3,000) on a rounding ensemble of 8 members
  (member k > 0: b and the scaled values perturbed by at most one and two ulp
  per entry, seed k): the outcome, the iteration at which it came and the
  metric reached.

Calls only oracle/ and problems/.  The members run in parallel processes
(about 15 minutes and 30 GB of memory on eight cores).
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

EPS = float(np.finfo(np.float64).eps)
N = 256
TOL = 1e-10
BCG_MEMBERS = 8
GMRES_STEPS = 60


def _job(args):
    import oracle
    from problems import configs

    kind, k = args
    s = configs.c3(N)
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    t = time.time()
    if kind == "gmres":
        _, info, hist, cyc = oracle.gmres(s.rowptr, s.colidx, val, b, m=30, tol=TOL, maxit=GMRES_STEPS,
                                          history=True, trace=True)
        return kind, {"est": [float(v) for v in hist], "cycles": cyc, "info": info, "seconds": time.time() - t}
    if k > 0:
        rs = np.random.default_rng(k)
        b = b * (1.0 + rs.uniform(-1.0, 1.0, s.n) * EPS)
        val = val * (1.0 + rs.uniform(-2.0, 2.0, len(val)) * EPS)
    _, info = oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=TOL, maxit=3000)
    return kind, {"member": k, "conv": info["conv"], "iters": info["iters"], "relres_true": info["relres_true"],
                  "seconds": time.time() - t}


def main():
    jobs = [("gmres", 0)] + [("bicgstab", k) for k in range(BCG_MEMBERS)]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(_job, jobs, chunksize=1)
    out = {"workload": f"c3 {N}^3 GS(2) tol {TOL:g}",
           "perturbation": "member k > 0: b * (1 + U[-1,1] eps), scaled values * (1 + U[-2,2] eps), seed k"}
    out["gmres30"] = next(r for kind, r in res if kind == "gmres")
    out["bicgstab"] = sorted((r for kind, r in res if kind == "bicgstab"), key=lambda r: r["member"])
    with open(os.path.join(HERE, "c3_oracle_trace.json"), "w") as f:
        json.dump(out, f, indent=0)
    print({"gmres_est_60": out["gmres30"]["est"][-1],
           "bicgstab": [(r["conv"], r["iters"]) for r in out["bicgstab"]]})


if __name__ == "__main__":
    main()
