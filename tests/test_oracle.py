"""Pins for the CPU oracle against facts fixed by the paper and by mathematics
(no GPU).  Each test is chosen so that a plausible slip in the oracle (a
dropped term, a wrong sign or index, a transposed operand) breaks it."""
import math

import numpy as np
import pytest

import oracle
from problems import cd, configs

EPS = np.finfo(np.float64).eps


def _random_csr(n, seed, density=0.3, zero_row=None):
    rs = np.random.default_rng(seed)
    A = rs.uniform(-1, 1, (n, n)) * (rs.uniform(size=(n, n)) < density)
    A += np.diag(rs.uniform(2, 3, n) * n * density)
    if zero_row is not None:
        A[zero_row] = 0.0
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(A[i])[0]
        cols.extend(nz)
        vals.extend(A[i, nz])
        rowptr[i + 1] = len(cols)
    return A, rowptr, np.array(cols, dtype=np.int32), np.array(vals)


# ------------------------------------------------------------------ GS(p)
@pytest.mark.parametrize("p", [1.0, 2.0, math.inf, 3.5])
def test_gs_rows_have_unit_norm(p):
    """Sec. 1: after GS(p) every row has unit L_p norm."""
    s = configs.c1()
    val, b, d = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, p)
    for i in range(0, s.n, 7):
        row = val[s.rowptr[i]:s.rowptr[i + 1]]
        assert abs(oracle.lp_norm_def(row, p) - 1.0) <= 8 * EPS


def test_gs_closed_form_rows():
    rowptr = np.array([0, 2], dtype=np.int32)
    colidx = np.array([0, 1], dtype=np.int32)
    for p, want in [(2.0, [0.6, -0.8]), (1.0, [3 / 7, -4 / 7]), (math.inf, [0.75, -1.0])]:
        val, b, d = oracle.gs_scale(rowptr, colidx, np.array([3.0, -4.0]), np.array([10.0]), p)
        assert np.allclose(val, want, rtol=2 * EPS, atol=0)
        assert np.isclose(b[0], 10.0 * d[0], rtol=2 * EPS)


@pytest.mark.parametrize("p", [1.0, 2.0, math.inf, 3.5])
def test_gs_invariant_under_row_scaling(p):
    """GS(p)(Lambda A) = sign(Lambda) GS(p)(A) for any nonzero diagonal Lambda."""
    s = configs.c1()
    rs = np.random.default_rng(1)
    lam = 10.0 ** rs.uniform(-6, 6, s.n) * np.where(rs.uniform(size=s.n) < 0.3, -1, 1)
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    v1, b1, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, p)
    v2, b2, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val * lam[rows], s.b * lam, p)
    sg = np.sign(lam)
    assert np.allclose(v2, sg[rows] * v1, rtol=8 * EPS, atol=0)
    assert np.allclose(b2, sg * b1, rtol=8 * EPS, atol=1e-300)


def test_gs_power_of_two_scaling_is_exact_even_near_overflow():
    """Scaling a row by 2^k is exact in binary floating point, so GS must give
    bit-identical output for rows of size ~1e300 (no overflow of |a|^p)."""
    s = configs.c1()
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    k = np.where(np.arange(s.n) % 2 == 0, 990, -990)
    for p in [1.0, 2.0, math.inf, 3.5]:
        v1, _, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, None, p)
        v2, _, _ = oracle.gs_scale(s.rowptr, s.colidx, np.ldexp(s.val, k[rows]), None, p)
        assert np.array_equal(v1, v2)


def test_gs_norm_inequalities():
    s = configs.c2(10)
    _, _, d1 = oracle.gs_scale(s.rowptr, s.colidx, s.val, None, 1.0)
    _, _, d2 = oracle.gs_scale(s.rowptr, s.colidx, s.val, None, 2.0)
    _, _, di = oracle.gs_scale(s.rowptr, s.colidx, s.val, None, math.inf)
    nnz = np.diff(s.rowptr)
    n1, n2, ni = 1 / d1, 1 / d2, 1 / di
    assert np.all(ni <= n2 * (1 + 4 * EPS)) and np.all(n2 <= n1 * (1 + 4 * EPS))
    assert np.all(n1 <= nnz * ni * (1 + 4 * EPS))


def test_gs_same_solution_dense():
    """Eq. (2): DAx = Db has the solution of Ax = b."""
    s = configs.c1(12)
    x0 = np.linalg.solve(s.dense(), s.b)
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    sc = cd.System(s.n, s.rowptr, s.colidx, val, b)
    x1 = np.linalg.solve(sc.dense(), b)
    assert np.allclose(x0, x1, rtol=1e-12, atol=1e-12)
    assert np.allclose(x0, s.x_true, rtol=0, atol=1e-10)


def test_gs_errors():
    A, rp, ci, va = _random_csr(6, 0, zero_row=3)
    with pytest.raises(oracle.OracleError, match="zero row"):
        oracle.gs_scale(rp, ci, va, None, 2.0)
    A, rp, ci, va = _random_csr(6, 0)
    va[2] = np.nan
    with pytest.raises(oracle.OracleError, match="non-finite"):
        oracle.gs_scale(rp, ci, va, None, 2.0)
    with pytest.raises(oracle.OracleError):
        oracle.gs_scale(rp, ci, np.abs(va), None, 0.5)


# ------------------------------------------------- two-sided D^(1/2) scaling
def _dense_of(rp, ci, va, n):
    M = np.zeros((n, n))
    for i in range(n):
        M[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    return M


@pytest.mark.parametrize("p", [1.0, 2.0, math.inf])
def test_sym_scaling_solves_the_original_system(p):
    """Sec. 2: D^1/2 A D^1/2 y = D^1/2 b and x = D^1/2 y solve A x = b."""
    s = configs.c1(12)
    x0 = np.linalg.solve(s.dense(), s.b)
    val, b, sv, _ = oracle.gs_scale_sym(s.rowptr, s.colidx, s.val, s.b, p)
    y = np.linalg.solve(_dense_of(s.rowptr, s.colidx, val, s.n), b)
    assert np.allclose(sv * y, x0, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("p", [1.0, 2.0, math.inf])
def test_sym_scaling_is_similar_to_gs(p):
    """D^1/2 A D^1/2 = D^-1/2 (D A) D^1/2: the same eigenvalues as GS(p)(A)."""
    A, rp, ci, va = _random_csr(16, 7)
    v_gs, _, _ = oracle.gs_scale(rp, ci, va, None, p)
    v_sym, _, _, _ = oracle.gs_scale_sym(rp, ci, va, None, p)
    e_gs = np.sort_complex(np.linalg.eigvals(_dense_of(rp, ci, v_gs, 16)))
    e_sym = np.sort_complex(np.linalg.eigvals(_dense_of(rp, ci, v_sym, 16)))
    assert np.allclose(e_gs, e_sym, rtol=1e-10, atol=1e-12)


def test_sym_scaling_closed_forms():
    # a diagonal matrix becomes its sign pattern; a symmetric one stays symmetric
    n = 5
    d = np.array([3.0, -0.5, 7.0, -2.0, 1e-3])
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    for p in (1.0, 2.0, math.inf):
        v, _, sv, _ = oracle.gs_scale_sym(rp, ci, d, None, p)
        assert np.allclose(v, np.sign(d), rtol=4 * EPS, atol=0)  # d * s * s rounds within a few ulp
        assert np.allclose(sv, 1.0 / np.sqrt(np.abs(d)), rtol=2 * EPS)
    A, rp, ci, va = _random_csr(12, 9)
    S = A + A.T
    rp2 = np.zeros(13, dtype=np.int32)
    cols, vals = [], []
    for i in range(12):
        nz = np.nonzero(S[i])[0]
        cols.extend(nz)
        vals.extend(S[i, nz])
        rp2[i + 1] = len(cols)
    v, _, _, _ = oracle.gs_scale_sym(rp2, np.array(cols, dtype=np.int32), np.array(vals), None, 2.0)
    M = _dense_of(rp2, np.array(cols, dtype=np.int32), v, 12)
    assert np.allclose(M, M.T, rtol=4 * EPS, atol=0)


def test_sym_scaling_metric_weights_give_the_gs2_residual():
    """Sec. 2.2: the stopping test is the GS(2)-scaled residual of the
    original system; with the weights w, the scaled system's residual norm
    is exactly that for x = D^1/2 y."""
    A, rp, ci, va = _random_csr(20, 11)
    b = np.random.default_rng(1).normal(size=20)
    val, bs, sv, w = oracle.gs_scale_sym(rp, ci, va, b, 1.0)
    y = np.random.default_rng(2).normal(size=20)
    r_scaled = bs - _dense_of(rp, ci, val, 20) @ y
    r_orig = b - A @ (sv * y)
    d2 = 1.0 / np.linalg.norm(A, axis=1)
    assert np.allclose(w * r_scaled, d2 * r_orig, rtol=1e-12, atol=1e-13)


def test_sym_scaling_errors():
    A, rp, ci, va = _random_csr(6, 0, zero_row=3)
    with pytest.raises(oracle.OracleError, match="zero row"):
        oracle.gs_scale_sym(rp, ci, va, None, 2.0)
    A, rp, ci, va = _random_csr(6, 0)
    bad = ci.copy()
    bad[4] = 6
    with pytest.raises(oracle.OracleError, match="invalid"):
        oracle.gs_scale_sym(rp, bad, va, None, 2.0)
    va2 = va.copy()
    va2[1] = np.inf
    with pytest.raises(oracle.OracleError, match="non-finite"):
        oracle.gs_scale_sym(rp, ci, va2, None, 2.0)


# ------------------------------------------------------------------ ILU(0)
def _pattern_dense(rp, ci, v, n):
    M = np.zeros((n, n))
    for i in range(n):
        M[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    return M


def _split_lu(rp, ci, lu, n):
    F = _pattern_dense(rp, ci, lu, n)
    return np.tril(F, -1) + np.eye(n), np.triu(F)


def test_ilu0_is_exact_lu_on_a_tridiagonal_matrix():
    """No fill-in arises for a tridiagonal matrix, so ILU(0) = LU: the
    preconditioned system is the identity and GMRES needs one step."""
    n = 50
    rs = np.random.default_rng(5)
    T = np.diag(rs.uniform(3, 4, n)) + np.diag(rs.uniform(-1, 1, n - 1), 1) + np.diag(rs.uniform(-1, 1, n - 1), -1)
    rp = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(T[i])[0]
        cols.extend(nz)
        vals.extend(T[i, nz])
        rp[i + 1] = len(cols)
    ci, va = np.array(cols, dtype=np.int32), np.array(vals)
    lu = oracle.ilu0(rp, ci, va)
    L, U = _split_lu(rp, ci, lu, n)
    assert np.allclose(L @ U, T, rtol=0, atol=1e-14)
    b = rs.normal(size=n)
    x, info = oracle.gmres(rp, ci, va, b, m=10, tol=1e-12, lu=lu)
    assert info["iters"] == 1 and info["conv"] == 0
    assert np.allclose(T @ x, b, atol=1e-12)


def test_ilu0_matches_a_on_its_pattern():
    """The defining property of ILU(0): (LU)_ij = a_ij wherever a_ij is in
    the pattern (the fill-in outside it is what is dropped)."""
    s = configs.c1(9)
    lu = oracle.ilu0(s.rowptr, s.colidx, s.val)
    L, U = _split_lu(s.rowptr, s.colidx, lu, s.n)
    A = s.dense()
    mask = _pattern_dense(s.rowptr, s.colidx, np.ones_like(s.val), s.n) != 0
    assert np.allclose((L @ U)[mask], A[mask], rtol=1e-13, atol=1e-12)
    assert np.abs((L @ U)[~mask]).max() > 1e-3  # fill-in was dropped
    r = np.random.default_rng(6).normal(size=s.n)
    z = oracle.ilu0_apply(s.rowptr, s.colidx, lu, r)
    assert np.allclose(L @ (U @ z), r, rtol=1e-12, atol=1e-12)


def test_ilu0_is_row_scaling_equivariant():
    """For a positive diagonal D, ILU(0)(DA) = (D L D^-1, D U): the GS-scaled
    system's preconditioned operator is similar to the original one."""
    s = configs.c1(8)
    d = np.random.default_rng(7).uniform(0.5, 3.0, s.n)
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    lu1 = oracle.ilu0(s.rowptr, s.colidx, s.val)
    lu2 = oracle.ilu0(s.rowptr, s.colidx, s.val * d[rows])
    L1, U1 = _split_lu(s.rowptr, s.colidx, lu1, s.n)
    L2, U2 = _split_lu(s.rowptr, s.colidx, lu2, s.n)
    assert np.allclose(L2, np.diag(d) @ L1 @ np.diag(1 / d), rtol=1e-12, atol=1e-14)
    assert np.allclose(U2, np.diag(d) @ U1, rtol=1e-12, atol=1e-14)


def test_ilu0_errors():
    s = configs.c1(6)
    nodiag_rp = s.rowptr.copy()
    with pytest.raises(oracle.OracleError):  # no diagonal entry in row 0
        keep = np.ones(len(s.colidx), dtype=bool)
        keep[np.nonzero(s.colidx[s.rowptr[0]:s.rowptr[1]] == 0)[0][0]] = False
        rp = np.concatenate([[0], np.cumsum([np.count_nonzero(keep[s.rowptr[i]:s.rowptr[i + 1]])
                                             for i in range(s.n)])]).astype(np.int32)
        oracle.ilu0(rp, s.colidx[keep], s.val[keep])
    bad = s.colidx.copy()
    bad[0], bad[1] = bad[1], bad[0]  # unsorted row
    with pytest.raises(oracle.OracleError):
        oracle.ilu0(nodiag_rp, bad, s.val)


# ------------------------------------------------------------------ SpMV
def test_spmv_matches_dense():
    A, rp, ci, va = _random_csr(37, 3)
    x = np.random.default_rng(4).normal(size=37)
    assert np.allclose(oracle.spmv(rp, ci, va, x), A @ x, rtol=1e-14, atol=1e-13)


def test_metric_weights_are_gs2_scales():
    s = configs.c1(8)
    w = oracle.metric_weights(s.rowptr, s.val)
    A = s.dense()
    assert np.allclose(w, 1 / np.sqrt((A**2).sum(1)), rtol=4 * EPS)


# ---------------------------------------------------------------- Arnoldi
def test_arnoldi_relation_and_orthogonality():
    s = configs.c1(10)
    A = s.dense()
    v0 = np.random.default_rng(5).normal(size=s.n)
    k = 12
    V, H, steps = oracle.arnoldi(s.rowptr, s.colidx, s.val, v0, k)
    assert steps == k
    assert np.abs(A @ V[:, :k] - V @ H).max() <= 1e-12 * np.abs(A).sum(1).max()
    assert np.abs(np.eye(k + 1) - V.T @ V).max() <= 1e-13
    assert np.allclose(V[:, 0], v0 / np.linalg.norm(v0), rtol=1e-15, atol=1e-16)
    assert np.allclose(np.tril(H, -2), 0.0)  # Hessenberg
    assert np.all(np.diag(H, -1) > 0)


@pytest.mark.parametrize("k", [1, 4, 7])
def test_arnoldi_finite_termination_gives_the_eigenvalues(k):
    """A diagonal matrix with k distinct eigenvalues has a grade-k Krylov space:
    the Arnoldi process stops after exactly k steps (h_{k+1,k} ~ rounding), and
    the Ritz values of H(0:k, 0:k) are those k eigenvalues."""
    n = 90
    vals = np.array([0.5 + 1.3 * j for j in range(k)])
    rp, ci, va = _diag_csr(vals[np.arange(n) % k])
    v0 = np.random.default_rng(7).uniform(1, 2, n)
    _, H, steps = oracle.arnoldi(rp, ci, va, v0, 12)
    assert steps == k
    ritz = np.sort(np.linalg.eigvals(H[:k, :k]).real)
    assert np.allclose(ritz, vals, rtol=1e-12)
    assert np.all(H[:, k:] == 0.0)


def test_arnoldi_full_length_ritz_values_are_the_eigenvalues():
    """n steps on an n x n matrix: H(0:n, 0:n) = V^T A V is similar to A, so
    its eigenvalues equal LAPACK's eigenvalues of A."""
    A, rp, ci, va = _random_csr(30, 11, density=0.3)
    v0 = np.random.default_rng(12).normal(size=30)
    _, H, steps = oracle.arnoldi(rp, ci, va, v0, 30)
    assert steps == 30
    ea = np.sort_complex(np.linalg.eigvals(A))
    eh = np.sort_complex(np.linalg.eigvals(H[:30, :30]))
    assert np.allclose(ea, eh, rtol=1e-9, atol=1e-10 * np.abs(ea).max())


def test_arnoldi_symmetric_matrix_gives_a_symmetric_tridiagonal_h():
    """For symmetric A, H = V^T A V is symmetric and so tridiagonal (Lanczos)."""
    A, rp, ci, va = _random_csr(40, 13, density=0.2)
    As = A + A.T
    rows, cols = np.nonzero(As)
    rp = np.searchsorted(rows, np.arange(41)).astype(np.int32)
    _, H, steps = oracle.arnoldi(rp, cols.astype(np.int32), As[rows, cols], np.ones(40), 10)
    T = H[:10, :10]
    scale = np.abs(T).max()
    assert np.abs(np.triu(T, 2)).max() <= 1e-12 * scale
    assert np.allclose(np.diag(T, 1), np.diag(T, -1), rtol=1e-10)


def test_arnoldi_zero_start_takes_no_step():
    s = configs.c1(6)
    _, H, steps = oracle.arnoldi(s.rowptr, s.colidx, s.val, np.zeros(s.n), 5)
    assert steps == 0 and np.all(H == 0.0)


# ------------------------------------------------------------------ GMRES
def _diag_csr(d):
    n = len(d)
    return np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(d, dtype=np.float64)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_gmres_finite_termination_on_k_distinct_eigenvalues(k):
    """A diagonal matrix with k distinct eigenvalues has a grade-k Krylov space:
    GMRES(m >= k) converges in exactly k steps (to rounding)."""
    n = 60
    vals = np.array([1.0 + 0.7 * j for j in range(k)])
    d = vals[np.arange(n) % k]
    rp, ci, va = _diag_csr(d)
    b = np.random.default_rng(6).uniform(1, 2, n)
    x, info = oracle.gmres(rp, ci, va, b, m=10, tol=1e-12, w=np.ones(n))
    assert info["conv"] == oracle.CONVERGED
    assert info["iters"] == k
    assert np.allclose(x, b / d, rtol=1e-11)


def test_gmres_full_equals_dense_lu():
    A, rp, ci, va = _random_csr(25, 7, density=0.4)
    b = np.random.default_rng(8).normal(size=25)
    x, info = oracle.gmres(rp, ci, va, b, m=25, tol=1e-13, w=np.ones(25))
    assert info["conv"] == oracle.CONVERGED and info["restarts"] == 0
    assert np.allclose(x, oracle.dense_solve(A, b), rtol=1e-10, atol=1e-12)


def test_gmres_estimate_monotone_and_matches_true_residual():
    s = configs.c1()
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    n = s.n
    x, info, hist = oracle.gmres(s.rowptr, s.colidx, val, b, m=40, tol=1e-9, maxit=40,
                                 w=np.ones(n), history=True)
    # within one cycle the least-squares residual never increases
    assert np.all(np.diff(hist) <= 1e-15)
    r = b - oracle.spmv(s.rowptr, s.colidx, val, x)
    true = np.linalg.norm(r) / np.linalg.norm(b)
    assert abs(true - hist[-1]) <= 1e-10 * max(true, 1e-300) + 1e-14
    assert abs(info["relres_true"] - true) <= 1e-13


def test_gmres_restarted_reaches_tolerance_and_reports_metric():
    s = configs.c1(16)
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    x, info = oracle.gmres(s.rowptr, s.colidx, val, b, m=20, tol=1e-8)
    assert info["conv"] == oracle.CONVERGED
    assert info["restarts"] >= 1
    assert info["relres_true"] < 1e-8
    assert abs(oracle.relres(s.rowptr, s.colidx, val, b, x) - info["relres_true"]) < 1e-15
    # forward error is bounded by cond(A) times the relative residual
    sc = cd.System(s.n, s.rowptr, s.colidx, val, b)
    kappa = np.linalg.cond(sc.dense())
    assert np.linalg.norm(x - s.x_true) / np.linalg.norm(s.x_true) <= 2 * kappa * info["relres_true"]


def test_gmres_maxit_is_respected():
    s = configs.c1()
    x, info = oracle.gmres(s.rowptr, s.colidx, s.val, s.b, m=20, tol=1e-12, maxit=55)
    assert info["iters"] == 55 and info["conv"] == oracle.MAXIT


# -------------------------------------------------------------- Bi-CGSTAB
def test_bicgstab_scalar_multiple_of_identity_one_iteration():
    n = 40
    rp, ci, va = _diag_csr(np.full(n, 3.5))
    b = np.random.default_rng(9).normal(size=n)
    x, info = oracle.bicgstab(rp, ci, va, b, tol=1e-12)
    assert info["conv"] == oracle.CONVERGED and info["iters"] == 1
    assert np.allclose(x, b / 3.5, rtol=1e-15)


@pytest.mark.parametrize("N", [4, 7, 12])
def test_bicgstab_matches_dense_lu_on_small_grids(N):
    s = configs.c1(N)
    A = s.dense()
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    x, info = oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=1e-12)
    assert info["conv"] == oracle.CONVERGED
    xd = oracle.dense_solve(A, s.b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


def test_bicgstab_recovers_manufactured_solution_c1():
    s = configs.c1()
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    x, info = oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=1e-8)
    assert info["conv"] == oracle.CONVERGED and info["relres_true"] < 1e-8
    sc = cd.System(s.n, s.rowptr, s.colidx, val, b)
    kappa = np.linalg.cond(sc.dense())
    assert np.linalg.norm(x - s.x_true) / np.linalg.norm(s.x_true) <= 2 * kappa * info["relres_true"]
    assert abs(oracle.relres(s.rowptr, s.colidx, val, b, x) - info["relres_true"]) < 1e-15


def test_bicgstab_history_and_scaling_helps_c1():
    """GS(2) cuts the Bi-CGSTAB iteration count on the discontinuous C1 system
    (the effect reported throughout Sec. 3-6)."""
    s = configs.c1()
    _, i0 = oracle.bicgstab(s.rowptr, s.colidx, s.val, s.b, tol=1e-8)
    val, b, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    _, i2 = oracle.bicgstab(s.rowptr, s.colidx, val, b, tol=1e-8)
    assert i2["conv"] == oracle.CONVERGED
    assert i2["iters"] * 4 < i0["iters"]


def test_metric_is_the_gs2_scaled_residual_whatever_the_scaling():
    """Sec. 2.2: the test is made on the GS(2)-scaled system.  The metric of a
    GS(1)-scaled solve must equal the plain residual ratio of the GS(2) system."""
    s = configs.c1(12)
    v1, b1, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 1.0)
    x, info = oracle.bicgstab(s.rowptr, s.colidx, v1, b1, tol=1e-6)
    v2, b2, _ = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)
    r = b2 - oracle.spmv(s.rowptr, s.colidx, v2, x)
    assert abs(np.linalg.norm(r) / np.linalg.norm(b2) - info["relres_true"]) < 1e-14


def test_bicgstab_breakdown_is_reported():
    # rh = r orthogonal to A r: the rotation [[0, 1], [-1, 0]] gives sigma = 0
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([1, 0], dtype=np.int32)
    va = np.array([1.0, -1.0])
    x, info = oracle.bicgstab(rp, ci, va, np.array([1.0, 0.0]), tol=1e-10)
    assert info["conv"] == oracle.BREAKDOWN and info["iters"] == 0


def test_the_empty_system_is_solved_at_x0():
    """n = 0: the residual is the empty vector, of norm 0, so both solvers
    stop at x0 before any step -- the same outcome as for b = 0 on a
    non-empty system (Sec. 2.2's test with a zero initial residual)."""
    rp = np.zeros(1, dtype=np.int32)
    e = (rp, np.zeros(0, dtype=np.int32), np.zeros(0), np.zeros(0))
    for x, info in (oracle.bicgstab(*e, tol=1e-8), oracle.gmres(*e, m=10, tol=1e-8)):
        assert info["conv"] == oracle.CONVERGED and info["iters"] == 0 and info["relres_true"] == 0.0
        assert len(x) == 0
    s = configs.c1(6)
    z = np.zeros(s.n)
    for x, info in (oracle.bicgstab(s.rowptr, s.colidx, s.val, z, tol=1e-8),
                    oracle.gmres(s.rowptr, s.colidx, s.val, z, m=10, tol=1e-8)):
        assert info["conv"] == oracle.CONVERGED and info["iters"] == 0 and not x.any()
    with pytest.raises(oracle.OracleError):
        oracle.gmres(rp, e[1], e[2], e[3], m=0, tol=1e-8)
