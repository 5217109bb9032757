"""Inputs that drive the solvers into their rarely taken branches, shared by
the oracle pins (test_oracle_branches) and the GPU parity tests
(test_gpu_branches).  Seeded and synthetic; no solver arithmetic here."""
import numpy as np

import oracle
from problems import configs


def ill_posed_c1():
    """The GS(2)-scaled C1 matrix (cond ~1.9e5) with the right-hand side of
    its smallest singular vector: ||b|| is then cond(A) times smaller than
    ||A|| ||x||, so the true residual cannot fall much below eps cond(A)
    (~5e-11 here) while the recursive residual keeps falling."""
    s = configs.c1()
    v, _, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    A = np.zeros((s.n, s.n))
    for i in range(s.n):
        A[i, s.colidx[s.rowptr[i]:s.rowptr[i + 1]]] = v[s.rowptr[i]:s.rowptr[i + 1]]
    _, _, vt = np.linalg.svd(A)
    x_true = vt[-1]
    return s.rowptr, s.colidx, v, A @ x_true


def row_scaled_system(seed=11, n=300, density=0.03, spread=1.0):
    """A well-conditioned nonsymmetric matrix whose rows are multiplied by
    10^U[-spread, spread]: GMRES minimises the unweighted residual, so its
    estimate can meet tol while the GS(2)-weighted metric of Sec. 2.2 does
    not."""
    import scipy.sparse as sp

    rs = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=seed + 1, format="csr")
    A = (A + sp.diags(rs.uniform(2, 3, n) * (1 + density * n))).tocsr()
    lam = 10.0 ** rs.uniform(-spread, spread, n)
    A = (sp.diags(lam) @ A).tocsr()
    A.sort_indices()
    b = lam * rs.normal(size=n)
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data, b
