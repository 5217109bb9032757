"""The oracle's Krylov solvers against SciPy's independent implementations
of the same methods (scipy.sparse.linalg.gmres with restart m and bicgstab),
on well-conditioned nonsymmetric systems where the iteration counts do not
depend on rounding: the same iterates (solutions equal to a few ulp) and the
same counts -- GMRES(m) Arnoldi steps exactly; Bi-CGSTAB iterations equal,
or one more in the oracle, which counts an exit at the half step (s small
enough) as an iteration where SciPy's callback does not run."""
import numpy as np
import pytest

import oracle

sp = pytest.importorskip("scipy.sparse")
spla = pytest.importorskip("scipy.sparse.linalg")


def _system(seed, n=300, density=0.03):
    rs = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=seed + 1, format="csr")
    A = (A + sp.diags(rs.uniform(2, 3, n) * (1 + density * n))).tocsr()
    A.sort_indices()
    return A, rs.normal(size=n)


def _csr(A):
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data


@pytest.mark.parametrize("seed", [3, 11, 29])
@pytest.mark.parametrize("tol", [1e-6, 1e-10])
@pytest.mark.parametrize("m", [5, 20])
def test_gmres_matches_scipy(seed, tol, m):
    A, b = _system(seed)
    steps = [0]
    x_sp, info = spla.gmres(A, b, rtol=tol, atol=0.0, restart=m, maxiter=1000,
                            callback=lambda _: steps.__setitem__(0, steps[0] + 1), callback_type="pr_norm")
    # the metric ||b - Ax|| / ||b|| (x0 = 0): unit weights
    x_or, io = oracle.gmres(*_csr(A), b, m=m, tol=tol, w=np.ones(len(b)))
    assert info == 0 and io["conv"] == oracle.CONVERGED
    assert io["iters"] == steps[0]
    assert np.abs(x_or - x_sp).max() <= 1e-13 * np.abs(x_or).max()


@pytest.mark.parametrize("seed", [3, 11, 29])
@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_bicgstab_matches_scipy(seed, tol):
    A, b = _system(seed)
    its = [0]
    x_sp, info = spla.bicgstab(A, b, rtol=tol, atol=0.0, maxiter=1000,
                               callback=lambda _: its.__setitem__(0, its[0] + 1))
    x_or, io = oracle.bicgstab(*_csr(A), b, tol=tol, refresh=0, w=np.ones(len(b)))
    assert info == 0 and io["conv"] == oracle.CONVERGED
    assert io["iters"] in (its[0], its[0] + 1), (io["iters"], its[0])
    assert np.abs(x_or - x_sp).max() <= 1e-13 * np.abs(x_or).max()
