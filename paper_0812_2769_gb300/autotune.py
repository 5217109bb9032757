"""Autotuner for the batched solvers' launch shape.

The batched solvers run one thread block per system (thread per row, block
sizes 128, 256 or 512) and can hand systems above a row count to the
grid-wide solvers (gsk_opts.batch_block, gsk_opts.batch_large_n).  Which
shape is fastest depends on the batch (system sizes, nonzeros per row), the
solver and the precision, so it is measured: the tuner times every candidate
on a sample of the batch and keeps the fastest, caching the choice in a JSON
file under a key built from those properties and the GPU's name.

The sample is solved on copies of the systems (the solvers scale A and b in
place and overwrite x), so tuning leaves the caller's data untouched.  Only
candidates that converge as many sample systems as the best of them are
eligible (a shape must not buy speed with fewer converged systems).

    cfg = autotune.batched_config(As, bs, xs, solver="bicgstab", p=2.0)
    infos, stat = bicgstab_solve_batched(As, bs, xs, p=2.0, options=opts(**cfg))
"""
from __future__ import annotations

import json
import math
import os
import time

BLOCKS = (128, 256, 512)
# The sample has to keep the GPU as busy as the real batch (several waves of
# resident blocks): a small one times how fast one system is solved, not how
# many are solved per second, and favours larger blocks.  Up to this many
# systems are timed per candidate (a one-time cost, cached).
SAMPLE = 4096


def cache_path() -> str:
    return os.environ.get("GSK_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_0812_2769_gb300", "autotune.json"))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, table):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def batch_key(As, solver: str, precision: int, m) -> str:
    """Cache key: solver, precision, restart length, the GPU, and the batch's
    size class (count, median and largest rows on a log2 scale, nonzeros per
    row rounded)."""
    import torch

    ns = sorted(A.n for A in As)
    nnz = sum(A.nnz for A in As)
    rows = max(1, sum(ns))
    med = ns[len(ns) // 2] if ns else 0
    lg = lambda v: int(round(math.log2(max(1, v))))
    mm = m if not isinstance(m, (list, tuple)) else max(m)
    dev = torch.cuda.get_device_name(As[0].val.device) if (As and As[0].val.is_cuda) else "none"
    return (f"{solver}|prec{precision}|m{mm}|{dev}|count{lg(len(ns))}|med{lg(med)}|max{lg(ns[-1] if ns else 0)}|"
            f"nnzrow{round(nnz / rows)}")


def _sample_indices(As, k):
    """Up to k systems spread over the size range (sorted by rows)."""
    order = sorted(range(len(As)), key=lambda i: As[i].n)
    if len(order) <= k:
        return order
    step = len(order) / k
    return [order[int(i * step)] for i in range(k)]


def _clone(g, As, bs, xs, idx):
    out = []
    for i in idx:
        A = As[i]
        out.append((g.Csr(A.rowptr, A.colidx, A.val.clone()), bs[i].clone(), xs[i].clone()))
    return out


def _time_candidate(g, solver, base, p, m, tol, cfg, reps):
    import torch

    best = math.inf
    conv = None
    for _ in range(reps):
        sysv = [(g.Csr(A.rowptr, A.colidx, A.val.clone()), b.clone(), x.clone()) for A, b, x in base]
        As = [s[0] for s in sysv]
        bs = [s[1] for s in sysv]
        xs = [s[2] for s in sysv]
        o = g.opts(**cfg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if solver == "gmres":
            infos, stat = g.gmres_solve_batched(As, bs, xs, m=m, p=p, tol=tol, options=o, check=False)
        else:
            infos, stat = g.bicgstab_solve_batched(As, bs, xs, p=p, tol=tol, options=o, check=False)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
        conv = sum(1 for i, s in zip(infos, stat) if s == g.OK and i["conv"] == 0)
    return best, conv


def batched_config(As, bs, xs, solver: str = "bicgstab", p=2.0, m=30, tol: float = 1e-8, precision: int | None = None,
                   maxit: int = 10000, sample: int = SAMPLE, reps: int = 2, use_cache: bool = True,
                   large_candidates=None) -> dict:
    """The fastest (batch_block, batch_large_n) for this batch, from the cache
    or by timing the candidates on a sample.  Returns keyword arguments for
    opts(): {"batch_block": ..., "batch_large_n": ..., "precision": ...,
    "maxit": ...}."""
    import paper_0812_2769_gb300 as g

    precision = g.PREC_F64 if precision is None else precision
    path = cache_path()
    key = batch_key(As, solver, precision, m)
    table = _load(path) if use_cache else {}
    if key in table:
        hit = table[key]
        return {"batch_block": hit["batch_block"], "batch_large_n": hit["batch_large_n"], "precision": precision,
                "maxit": maxit}
    idx = _sample_indices(As, sample)
    pv = p if not isinstance(p, (list, tuple)) else [p[i] for i in idx]
    mv = m if not isinstance(m, (list, tuple)) else [m[i] for i in idx]
    base = _clone(g, As, bs, xs, idx)
    ns = sorted(As[i].n for i in idx)
    if large_candidates is None:
        # none, or the top tenth / top fortieth of the sample by rows
        large_candidates = sorted({0, ns[int(0.9 * (len(ns) - 1))], ns[int(0.975 * (len(ns) - 1))]} - {ns[-1]})
    results = []
    for blk in BLOCKS:
        for thr in large_candidates:
            if solver == "gmres" and precision != g.PREC_F64 and thr == 0:
                continue  # the one-block GMRES is FP64
            cfg = {"batch_block": blk, "batch_large_n": thr, "precision": precision, "maxit": maxit}
            t, conv = _time_candidate(g, solver, base, pv, mv, tol, cfg, reps)
            results.append({"batch_block": blk, "batch_large_n": thr, "seconds": t, "converged": conv})
    most = max(r["converged"] for r in results)
    best = min((r for r in results if r["converged"] == most), key=lambda r: r["seconds"])
    if use_cache:
        table = _load(path)
        table[key] = {"batch_block": best["batch_block"], "batch_large_n": best["batch_large_n"],
                      "sample": len(idx), "candidates": results}
        _store(path, table)
    return {"batch_block": best["batch_block"], "batch_large_n": best["batch_large_n"], "precision": precision,
            "maxit": maxit}
