"""Eigenvalue-distribution analysis (Sec. 3, Table 1b; Sec. 6, Table 4a).

The paper explains what GS does to a matrix through its spectrum: the
smallest and largest eigenvalue moduli, their ratio, and how many
eigenvalues fall into the first of 100 equal intervals of a histogram of
the real parts (Table 1b), or into the interval that holds the origin
(Table 4a).  GS leaves the ratio about where it was but empties the crowded
region next to zero.

Two routes to the eigenvalues:

* ``dense_eigenvalues``: all of them, for the paper's small grids (40 x 40,
  12 x 12 x 12).  A dense nonsymmetric eigensolver has no data-parallel
  form worth a GPU kernel at these sizes, so the CSR matrix (scaled on the
  device by ``gs_scale`` where GS is studied) is copied to the host and
  LAPACK's general eigensolver (numpy.linalg.eigvals) runs there.
* ``ritz_values``: the eigenvalues of the Hessenberg matrix of m Arnoldi
  steps run on the device by ``gsk_arnoldi`` (the GMRES basis kernels),
  for matrices far beyond a dense solver.  They approximate the extreme
  eigenvalues (the largest modulus first), not the crowd near zero.

``summary`` turns a set of eigenvalues into the statistics of the tables.
"""
from __future__ import annotations

import numpy as np

BINS = 100  # the paper's histogram has 100 intervals
MAX_DENSE = 8192


def summary(ev, bins: int = BINS) -> dict:
    """Table 1b / 4a statistics of the eigenvalues ev: lambda_min and
    lambda_max (smallest and largest modulus), their ratio, the count in the
    first of `bins` equal intervals of [min Re, max Re] (Table 1b) and the
    count in the interval containing Re = 0, or the nearest end interval when
    0 lies outside the range (Table 4a)."""
    ev = np.asarray(ev)
    if ev.size == 0:
        raise ValueError("no eigenvalues")
    mag = np.abs(ev)
    re = ev.real
    lo, hi = float(re.min()), float(re.max())
    hist, _ = np.histogram(re, bins, (lo, hi))
    width = (hi - lo) / bins
    k0 = 0 if width == 0 else int(np.clip(np.floor((0.0 - lo) / width), 0, bins - 1))
    lmin, lmax = float(mag.min()), float(mag.max())
    return {"lambda_min": lmin, "lambda_max": lmax, "ratio": lmax / lmin if lmin > 0 else float("inf"),
            "first_interval": int(hist[0]), "origin_interval": int(hist[k0]), "n": int(ev.size)}


def dense_eigenvalues(A, max_n: int = MAX_DENSE) -> np.ndarray:
    """All eigenvalues of the CSR matrix A (a library Csr on the device, or
    any object with rowptr/colidx/val arrays): copied to the host, densified,
    LAPACK's general eigensolver."""
    import torch

    rp, ci, va = (t.cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)
                  for t in (A.rowptr, A.colidx, A.val))
    n = len(rp) - 1
    if n > max_n:
        raise ValueError(f"n = {n} is too large for the dense eigensolver (max {max_n}); use ritz_values")
    D = np.zeros((n, n))
    D[np.repeat(np.arange(n), np.diff(rp)), ci] = va
    return np.linalg.eigvals(D)


def ritz_values(A, m: int = 64, v0=None, seed: int = 0, ctx=None, stream=None):
    """Ritz values of m Arnoldi steps on the device from v0 (a seeded normal
    vector when None); returns (ritz values, H, steps)."""
    import torch

    import paper_0812_2769_gb300 as g

    n = A.n
    if v0 is None:
        v0 = torch.as_tensor(np.random.default_rng(seed).normal(size=n), device=A.val.device)
    H, k = g.arnoldi(A, v0, m, ctx=ctx, stream=stream)
    return (np.linalg.eigvals(H[:k, :k]) if k else np.zeros(0)), H, k
