"""Writes c2_oracle_solutions.json: the oracle's solves of the 128^3 benchmark
workload (GS(2), tol 1e-8) that the full-size GPU parity test compares with.

* A rounding ensemble of iteration counts for Bi-CGSTAB (16 members) and
  GMRES(30) (4 members): member 0 solves the oracle's GS(2)-scaled system
  as it is; member k > 0 perturbs b by at most one ulp and the scaled values
  by at most two ulp per entry (seeded), the size of the differences between
  the GPU's GS(2) and the oracle's.
* For member 0 of each solver: the solution on 4,000 seeded sample rows
  (plus the first and last row), its norm, its distance to x_true and its
  metric (Sec. 2.2).

Calls only oracle/ and problems/.  Runs the members in parallel processes
(about ten minutes on eight cores).
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
N = 128
TOL = 1e-8
SAMPLE_SEED = 2026
ENSEMBLE = {"bicgstab": 16, "gmres30": 4}


def sample_rows(n):
    idx = np.random.default_rng(SAMPLE_SEED).choice(n, 4000, replace=False)
    return np.unique(np.concatenate([idx, [0, n - 1]]))


def _member(args):
    import oracle
    from problems import configs

    solver, k = args
    s = configs.c2(N)
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    if k > 0:
        rs = np.random.default_rng(k)
        b = b * (1.0 + rs.uniform(-1.0, 1.0, s.n) * EPS)
        val = val * (1.0 + rs.uniform(-2.0, 2.0, len(val)) * EPS)
    t = time.time()
    if solver == "bicgstab":
        x, info = oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=TOL)
    else:
        x, info = oracle.gmres(s.rowptr, s.colidx, val, b, m=30, tol=TOL)
    out = {"member": k, "iters": info["iters"], "conv": info["conv"], "relres_true": info["relres_true"],
           "seconds": time.time() - t}
    if k == 0:
        idx = sample_rows(s.n)
        out.update(rows=idx.tolist(), x=[float(v) for v in x[idx]], x_norm=float(np.linalg.norm(x)),
                   err_vs_true=float(np.linalg.norm(x - s.x_true) / np.linalg.norm(s.x_true)))
    return solver, out


def main():
    jobs = [(sv, k) for sv, cnt in ENSEMBLE.items() for k in range(cnt)]
    jobs.sort(key=lambda j: j[0] != "gmres30")  # the long GMRES runs first
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        results = pool.map(_member, jobs, chunksize=1)
    out = {"workload": f"c2 {N}^3 GS(2) tol {TOL:g}", "sample_seed": SAMPLE_SEED,
           "perturbation": "member k > 0: b * (1 + U[-1,1] eps), scaled values * (1 + U[-2,2] eps), seed k"}
    for solver in ENSEMBLE:
        ms = sorted((r for sv, r in results if sv == solver), key=lambda r: r["member"])
        out[solver] = {"ensemble_iters": [m["iters"] for m in ms], "ensemble_conv": [m["conv"] for m in ms],
                       "ensemble_relres": [m["relres_true"] for m in ms], "member0": ms[0]}
    with open(os.path.join(HERE, "c2_oracle_solutions.json"), "w") as f:
        json.dump(out, f, indent=0)
    print({sv: out[sv]["ensemble_iters"] for sv in ENSEMBLE})


if __name__ == "__main__":
    main()
