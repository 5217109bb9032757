"""Helpers shared by the GPU parity tests (marshalling only)."""
import numpy as np

EPS = np.finfo(np.float64).eps


def gsk():
    from paper_0812_2769_gb300 import build

    build.build()
    import paper_0812_2769_gb300 as g

    return g


def to_dev(g, sys_, dtype=None):
    import torch

    A = g.Csr.from_host(sys_.rowptr, sys_.colidx, sys_.val, device="cuda", dtype=dtype)
    b = torch.as_tensor(sys_.b, device="cuda")
    if dtype is not None:
        b = b.to(dtype)
    return A, b


def random_csr(n, seed, min_len=1, max_len=9, long_rows=(), long_len=300, diag_boost=4.0):
    """Random sparse matrix with ragged rows (sorted unique columns, diagonal
    present), optional very long rows; returns (rowptr, colidx, val)."""
    rs = np.random.default_rng(seed)
    rows_c, rows_v = [], []
    for i in range(n):
        L = long_len if i in long_rows else int(rs.integers(min_len, max_len + 1))
        L = min(L, n)
        cols = np.unique(np.concatenate([[i], rs.choice(n, size=max(L - 1, 0), replace=False)]))
        vals = rs.uniform(-1, 1, size=len(cols))
        vals[cols == i] = diag_boost * (1 + rs.uniform()) * np.sqrt(len(cols))
        rows_c.append(cols)
        rows_v.append(vals)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(c) for c in rows_c])
    return rowptr, np.concatenate(rows_c).astype(np.int32), np.concatenate(rows_v)
