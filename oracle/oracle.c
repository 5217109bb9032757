/*
 * Plain CPU FP64 oracle for geometric scaling and the two Krylov solvers.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA library, and the product path never calls
 * it.
 *
 * Everything is written for clarity, not speed: one thread, row-order loops,
 * sequential sums, no blocking or fusion beyond what the algorithms state.
 *
 * Sources (section / equation of the paper, Gordon & Gordon 2009):
 *   GS(p)      Sec. 1 and Sec. 2, Eq. (2): D = diag(1/||a_i||_p), solve DAx = Db.
 *   D^(1/2)    Sec. 2 (two-sided variant): D^(1/2) A D^(1/2) y = D^(1/2) b.
 *   L_p norm   Sec. 2 (read with absolute values; p = inf is max |a_ij|).
 *   GMRES(m)   Sec. 2: restarted GMRES (Saad & Schultz 1986) with double
 *              classical Gram-Schmidt; Givens rotations for the least-squares
 *              problem.
 *   Bi-CGSTAB  Sec. 2 and 2.2 (van der Vorst 1992); breakdown tolerance
 *              1e-16 * DBL_EPSILON relative to the vector norms (Sec. 2.2).
 *   ILU(0)     Sec. 2 (ILUT with drop tolerance 0 and fill-in 1 behaves as
 *              ILU(0)); Saad's IKJ algorithm; right preconditioning.
 *   Stopping   Sec. 2.2: ||b - Ax|| / ||b - Ax0|| < eps measured on the
 *              GS(2)-scaled system, i.e. with weights w_i = 1/||a_i||_2 of the
 *              matrix being solved; 10,000-iteration cap; x0 = 0 (Sec. 2.1).
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_ZERO_ROW 2
#define OR_ERR_NONFINITE 3
#define OR_ERR_OOM 4

/* convergence outcomes */
#define OR_CONVERGED 0
#define OR_MAXIT 1
#define OR_BREAKDOWN 2
#define OR_STAGNATED 3

typedef struct {
  int iters;         /* GMRES: Arnoldi steps; Bi-CGSTAB: iterations */
  int restarts;      /* GMRES cycles after the first */
  int refreshes;     /* Bi-CGSTAB true-residual restarts */
  int conv;          /* OR_CONVERGED ... */
  double relres_true;/* ||W(b - Ax)|| / ||W(b - Ax0)|| for the returned x */
  double relres_rec; /* last recursive / estimated value the solver saw */
} or_info;

/* ------------------------------------------------------------------ GS(p) */

/* ||a_i||_p of one row.  The row is divided by its largest magnitude m first
 * so that |a|^p cannot overflow or underflow; (sum (|a|/m)^p)^(1/p) * m is the
 * same quantity.  p = 1 and p = 2 are written out; p = inf is the max. */
static double row_norm(const double* a, int len, double p) {
  double m = 0.0;
  for (int k = 0; k < len; ++k) {
    double v = fabs(a[k]);
    if (v > m) m = v;
  }
  if (m == 0.0 || isinf(p)) return m;
  double s = 0.0;
  for (int k = 0; k < len; ++k) {
    double q = fabs(a[k]) / m;
    if (p == 1.0) s += q;
    else if (p == 2.0) s += q * q;
    else s += pow(q, p);
  }
  if (p == 1.0) return m * s;
  if (p == 2.0) return m * sqrt(s);
  return m * pow(s, 1.0 / p);
}

/* GS(p), Eq. (2): a_ij <- a_ij / ||a_i||_p and b_i <- b_i / ||a_i||_p.
 * s_out (optional) receives d_i = 1/||a_i||_p, the diagonal of D.
 * A row of zeros is an error (the paper assumes none). */
int or_gs_scale(int n, const int* rowptr, const int* colidx, double* val,
                double* b, double p, double* s_out) {
  (void)colidx;
  if (n < 0 || !(p >= 1.0)) return OR_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    int r0 = rowptr[i], len = rowptr[i + 1] - rowptr[i];
    for (int k = 0; k < len; ++k)
      if (!isfinite(val[r0 + k])) return OR_ERR_NONFINITE;
    if (b && !isfinite(b[i])) return OR_ERR_NONFINITE;
  }
  for (int i = 0; i < n; ++i)
    if (row_norm(val + rowptr[i], rowptr[i + 1] - rowptr[i], p) == 0.0)
      return OR_ERR_ZERO_ROW;
  for (int i = 0; i < n; ++i) {
    int r0 = rowptr[i], len = rowptr[i + 1] - rowptr[i];
    double nrm = row_norm(val + r0, len, p);
    for (int k = 0; k < len; ++k) val[r0 + k] = val[r0 + k] / nrm;
    if (b) b[i] = b[i] / nrm;
    if (s_out) s_out[i] = 1.0 / nrm;
  }
  return OR_OK;
}

/* Two-sided variant of GS (Sec. 2, the paragraph after the experimental
 * set-up): with D = diag(1/||a_i||_p), the system becomes
 * D^(1/2) A D^(1/2) y = D^(1/2) b, and x = D^(1/2) y.
 *   s_out[i] = (1/||a_i||_p)^(1/2), the diagonal of D^(1/2) (required);
 *   w_out[i] = (1/||a_i||_2) / s_out[i] (optional): stopping-metric weights
 *   for the scaled system.  Its residual is D^(1/2)(b - A x), so these
 *   weights turn its norm into the GS(2)-scaled residual of the original
 *   system, the paper's stopping test (Sec. 2.2).
 * The whole input is checked (finite values, column indices, no zero row)
 * before anything is written. */
int or_gs_scale_sym(int n, const int* rowptr, const int* colidx, double* val,
                    double* b, double p, double* s_out, double* w_out) {
  if (n < 0 || !(p >= 1.0) || !s_out) return OR_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (colidx[k] < 0 || colidx[k] >= n) return OR_ERR_ARG;
      if (!isfinite(val[k])) return OR_ERR_NONFINITE;
    }
    if (b && !isfinite(b[i])) return OR_ERR_NONFINITE;
  }
  for (int i = 0; i < n; ++i) {
    int r0 = rowptr[i], len = rowptr[i + 1] - rowptr[i];
    double nrm = row_norm(val + r0, len, p);
    if (nrm == 0.0) return OR_ERR_ZERO_ROW;
    s_out[i] = sqrt(1.0 / nrm);
    if (w_out) w_out[i] = (1.0 / row_norm(val + r0, len, 2.0)) / s_out[i];
  }
  for (int i = 0; i < n; ++i) {
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) val[k] = val[k] * s_out[i] * s_out[colidx[k]];
    if (b) b[i] = b[i] * s_out[i];
  }
  return OR_OK;
}

/* ------------------------------------------------------------ basic ops */

void or_spmv(int n, const int* rowptr, const int* colidx, const double* val,
             const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[colidx[k]];
    y[i] = s;
  }
}

static double dot(int n, const double* x, const double* y) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

static double wnorm(int n, const double* w, const double* x) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += (w[i] * x[i]) * (w[i] * x[i]);
  return sqrt(s);
}

/* r = b - A x */
static void residual(int n, const int* rp, const int* ci, const double* va,
                     const double* b, const double* x, double* r) {
  or_spmv(n, rp, ci, va, x, r);
  for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
}

/* Stopping-test weights: w_i = 1/||a_i||_2, the GS(2) scales of the matrix
 * being solved (Sec. 2.2: the test is made on the GS(2)-scaled system; since
 * GS(2) of D A equals GS(2) of A for any positive diagonal D, these weights
 * turn any row scaling of the system into its GS(2) form). */
int or_metric_weights(int n, const int* rowptr, const double* val, double* w) {
  for (int i = 0; i < n; ++i) {
    double nrm = row_norm(val + rowptr[i], rowptr[i + 1] - rowptr[i], 2.0);
    if (nrm == 0.0) return OR_ERR_ZERO_ROW;
    w[i] = 1.0 / nrm;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ GMRES */

/* One Arnoldi step with classical Gram-Schmidt applied twice (Sec. 2:
 * "double classical Gram-Schmidt").  On entry V holds the orthonormal
 * columns v_0..v_j (column-major, leading dimension n).  Computes
 * w = A v_j, h1 = V^T w, w -= V h1, h2 = V^T w, w -= V h2, and returns in
 * hcol[0..j] the sum h1 + h2 and in hcol[j+1] = ||w||.  w is left in wout.
 * *aw_norm receives ||A v_j|| (used by the breakdown test). */
/* ------------------------------------------------------------ ILU(0) */

/* ILU(0) (Sec. 2: the paper's ILUT with drop tolerance 0 and fill-in 1 acted
 * as ILU(0)), in the IKJ form of Saad, Iterative Methods for Sparse Linear
 * Systems, Alg. 10.4: L (unit lower) and U share A's sparsity pattern and
 * are stored together in lu (A's layout).  For each row i and each k < i in
 * its pattern, in column order: l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj
 * for every j > k present in both rows i and k.
 * Rows must hold their diagonal and sorted column indices; a zero pivot is an
 * error. */
int or_ilu0(int n, const int* rp, const int* ci, const double* va, double* lu) {
  if (n <= 0) return OR_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    int has_diag = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] < 0 || ci[k] >= n) return OR_ERR_ARG;
      if (k > rp[i] && ci[k] <= ci[k - 1]) return OR_ERR_ARG;
      if (ci[k] == i) has_diag = 1;
      lu[k] = va[k];
    }
    if (!has_diag) return OR_ERR_ARG;
  }
  for (int i = 0; i < n; ++i) {
    for (int kk = rp[i]; kk < rp[i + 1] && ci[kk] < i; ++kk) {
      const int k = ci[kk];
      double ukk = 0.0;
      for (int q = rp[k]; q < rp[k + 1]; ++q)
        if (ci[q] == k) ukk = lu[q];
      if (ukk == 0.0) return OR_ERR_ZERO_ROW;
      lu[kk] = lu[kk] / ukk;
      for (int jj = kk + 1; jj < rp[i + 1]; ++jj) {
        const int j = ci[jj];
        for (int q = rp[k]; q < rp[k + 1]; ++q)
          if (ci[q] == j) lu[jj] -= lu[kk] * lu[q];
      }
    }
    double uii = 0.0;
    for (int q = rp[i]; q < rp[i + 1]; ++q)
      if (ci[q] == i) uii = lu[q];
    if (uii == 0.0 || !isfinite(uii)) return OR_ERR_ZERO_ROW;
  }
  return OR_OK;
}

/* z = (LU)^-1 r: forward substitution with the unit lower factor, then
 * backward substitution with the upper factor, rows in order. */
void or_ilu0_apply(int n, const int* rp, const int* ci, const double* lu, const double* r, double* z) {
  for (int i = 0; i < n; ++i) {
    double s = r[i];
    for (int k = rp[i]; k < rp[i + 1] && ci[k] < i; ++k) s -= lu[k] * z[ci[k]];
    z[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = z[i], d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] > i) s -= lu[k] * z[ci[k]];
      else if (ci[k] == i) d = lu[k];
    }
    z[i] = s / d;
  }
}

/* y = A M^-1 x with M = LU from or_ilu0 (right preconditioning), or y = A x
 * when lu is NULL; tmp is scratch [n]. */
static void precond_spmv(int n, const int* rp, const int* ci, const double* va, const double* lu,
                         const double* x, double* y, double* tmp) {
  if (lu) {
    or_ilu0_apply(n, rp, ci, lu, x, tmp);
    or_spmv(n, rp, ci, va, tmp, y);
  } else {
    or_spmv(n, rp, ci, va, x, y);
  }
}

static void arnoldi_step(int n, const int* rp, const int* ci, const double* va, const double* lu,
                         const double* V, int j, double* hcol, double* wout,
                         double* h2, double* aw_norm, double* tmp) {
  precond_spmv(n, rp, ci, va, lu, V + (size_t)j * n, wout, tmp);
  *aw_norm = sqrt(dot(n, wout, wout));
  for (int k = 0; k <= j; ++k) hcol[k] = dot(n, V + (size_t)k * n, wout);
  for (int k = 0; k <= j; ++k) {
    const double* vk = V + (size_t)k * n;
    for (int i = 0; i < n; ++i) wout[i] -= hcol[k] * vk[i];
  }
  for (int k = 0; k <= j; ++k) h2[k] = dot(n, V + (size_t)k * n, wout);
  for (int k = 0; k <= j; ++k) {
    const double* vk = V + (size_t)k * n;
    for (int i = 0; i < n; ++i) wout[i] -= h2[k] * vk[i];
  }
  for (int k = 0; k <= j; ++k) hcol[k] += h2[k];
  hcol[j + 1] = sqrt(dot(n, wout, wout));
}

/* k Arnoldi steps from v0 (normalised here), exposing V (n x (k+1)) and the
 * Hessenberg matrix H ((k+1) x k, column-major) built by arnoldi_step.
 * Returns the number of steps completed: fewer than k when the Krylov space
 * is numerically invariant (h_{j+1,j} <= 1e-14 ||A v_j||, GMRES's rule), 0
 * for v0 = 0.  The eigenvalues of the leading square block are the Ritz
 * values used for the eigenvalue analysis of Sec. 3. */
int or_arnoldi(int n, const int* rp, const int* ci, const double* va,
               const double* v0, int k, double* V, double* H) {
  double* h2 = (double*)malloc(sizeof(double) * (k + 1));
  if (!h2) return -1;
  double beta = sqrt(dot(n, v0, v0));
  memset(H, 0, sizeof(double) * (size_t)(k + 1) * k);
  if (beta == 0.0) { free(h2); return 0; }
  for (int i = 0; i < n; ++i) V[i] = v0[i] / beta;
  int done = 0;
  for (int j = 0; j < k; ++j) {
    double awn;
    double* hcol = H + (size_t)j * (k + 1);
    double* w = V + (size_t)(j + 1) * n;
    arnoldi_step(n, rp, ci, va, NULL, V, j, hcol, w, h2, &awn, NULL);
    done = j + 1;
    if (hcol[j + 1] <= 1e-14 * awn) break;
    for (int i = 0; i < n; ++i) w[i] /= hcol[j + 1];
  }
  free(h2);
  return done;
}

/* Restarted GMRES(m) (Saad & Schultz 1986) as described in Sec. 2.
 *
 * Per cycle: beta = ||r||, v_0 = r / beta, g = beta e_1; for j = 0..m-1 an
 * Arnoldi step (CGS2), then the earlier Givens rotations are applied to the
 * new column of H, a new rotation (c, s) = (h_jj, h_j+1,j) / hypot(...) zeroes
 * h_j+1,j, and g_j+1 = -s g_j, g_j = c g_j, so |g_j+1| is ||b - A x_j||.
 * The cycle ends when |g_j+1| < tau * ||r0||, at (near) exact breakdown
 * h_j+1,j <= 1e-14 ||A v_j||, after m steps, or at maxit.  Then H y = g is
 * solved by back substitution and x += V y; the true residual is formed and
 * the weighted metric ||W r|| / ||W r0|| decides convergence.  If the
 * estimate said "converged" but the weighted metric did not, tau is tightened
 * by tol / metric and the method restarts.
 *
 * hist (optional, length maxit) receives |g_j+1| / ||r0|| per step.
 * trace (optional, 4 * trace_cap doubles) receives one record per cycle:
 * the steps it took, the tau it ran with, its last estimate |g_j+1| / ||r0||
 * and the weighted metric after its update of x (records past trace_cap are
 * dropped).  Neither output changes the arithmetic. */
int or_gmres(int n, const int* rp, const int* ci, const double* va,
             const double* b, double* x, int m, double tol, int maxit,
             const double* w_in, const double* lu, or_info* info, double* hist,
             double* trace, int trace_cap) {
  memset(info, 0, sizeof(*info));
  if (n < 0 || m < 1 || maxit < 0 || !(tol >= 0.0)) return OR_ERR_ARG;
  /* the empty system: its residual is the empty vector, of norm 0 -- the
   * case mu0 = 0 below, converged at x0 without a step */
  if (n == 0) { info->conv = OR_CONVERGED; return OR_OK; }
  size_t nn = (size_t)n;
  double* V = (double*)malloc(sizeof(double) * nn * (m + 1));
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* g = (double*)calloc(m + 1, sizeof(double));
  double* cs = (double*)calloc(m, sizeof(double));
  double* sn = (double*)calloc(m, sizeof(double));
  double* y = (double*)calloc(m, sizeof(double));
  double* h2 = (double*)calloc(m + 1, sizeof(double));
  double* r = (double*)malloc(sizeof(double) * nn);
  double* wv = (double*)malloc(sizeof(double) * nn);
  double* tmp = (double*)malloc(sizeof(double) * nn);
  double* u = (double*)malloc(sizeof(double) * nn);
  if (!V || !H || !g || !cs || !sn || !y || !h2 || !r || !wv || !tmp || !u) {
    free(V); free(H); free(g); free(cs); free(sn); free(y); free(h2); free(r); free(wv); free(tmp); free(u);
    return OR_ERR_OOM;
  }
  const double* w = w_in;
  if (!w) {
    if (or_metric_weights(n, rp, va, wv) != OR_OK) { free(V); free(H); free(g); free(cs); free(sn); free(y); free(h2); free(r); free(wv); free(tmp); free(u); return OR_ERR_ZERO_ROW; }
    w = wv;
  }

  residual(n, rp, ci, va, b, x, r);
  double mu0 = wnorm(n, w, r);
  double rho0 = sqrt(dot(n, r, r));
  info->conv = OR_MAXIT;
  if (mu0 == 0.0) {
    info->conv = OR_CONVERGED;
    goto out;
  }
  double tau = tol;
  int cycle = 0;
  for (;;) {
    double beta = sqrt(dot(n, r, r));
    for (size_t i = 0; i < nn; ++i) V[i] = r[i] / beta;
    for (int k = 0; k <= m; ++k) g[k] = 0.0;
    g[0] = beta;
    int kcols = 0, est_hit = 0;
    for (int j = 0; j < m && info->iters < maxit; ++j) {
      double* hcol = H + (size_t)j * (m + 1);
      double* wj = V + (size_t)(j + 1) * nn;
      double awn;
      arnoldi_step(n, rp, ci, va, lu, V, j, hcol, wj, h2, &awn, tmp);
      info->iters++;
      kcols = j + 1;
      double hnext = hcol[j + 1];
      for (int k = 0; k < j; ++k) {
        double t0 = cs[k] * hcol[k] + sn[k] * hcol[k + 1];
        double t1 = -sn[k] * hcol[k] + cs[k] * hcol[k + 1];
        hcol[k] = t0;
        hcol[k + 1] = t1;
      }
      double rho = hypot(hcol[j], hnext);
      if (rho == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
      else { cs[j] = hcol[j] / rho; sn[j] = hnext / rho; }
      hcol[j] = rho;
      hcol[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      double est = fabs(g[j + 1]) / rho0;
      info->relres_rec = est;
      if (hist) hist[info->iters - 1] = est;
      if (est < tau) { est_hit = 1; break; }
      if (hnext <= 1e-14 * awn) break; /* the Krylov space is (numerically) invariant */
      for (size_t i = 0; i < nn; ++i) wj[i] /= hnext;
    }
    /* back substitution H(0:k,0:k) y = g(0:k) */
    for (int i = kcols - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < kcols; ++k) s -= H[(size_t)k * (m + 1) + i] * y[k];
      y[i] = s / H[(size_t)i * (m + 1) + i];
    }
    if (lu) { /* x += M^-1 (V y) */
      for (size_t i = 0; i < nn; ++i) u[i] = 0.0;
      for (int k = 0; k < kcols; ++k) {
        const double* vk = V + (size_t)k * nn;
        for (size_t i = 0; i < nn; ++i) u[i] += y[k] * vk[i];
      }
      or_ilu0_apply(n, rp, ci, lu, u, tmp);
      for (size_t i = 0; i < nn; ++i) x[i] += tmp[i];
    } else { /* x += V y */
      for (int k = 0; k < kcols; ++k) {
        const double* vk = V + (size_t)k * nn;
        for (size_t i = 0; i < nn; ++i) x[i] += y[k] * vk[i];
      }
    }
    residual(n, rp, ci, va, b, x, r);
    double mu = wnorm(n, w, r) / mu0;
    info->relres_true = mu;
    if (trace && cycle < trace_cap) {
      trace[4 * cycle + 0] = kcols;
      trace[4 * cycle + 1] = tau;
      trace[4 * cycle + 2] = info->relres_rec;
      trace[4 * cycle + 3] = mu;
    }
    if (mu < tol) { info->conv = OR_CONVERGED; break; }
    if (info->iters >= maxit || kcols == 0) { info->conv = OR_MAXIT; break; }
    if (est_hit) tau = tau * (tol / mu);
    cycle++;
    info->restarts = cycle;
  }
out:
  if (info->conv == OR_CONVERGED && info->iters == 0) info->relres_true = 0.0;
  free(V); free(H); free(g); free(cs); free(sn); free(y); free(h2); free(r); free(wv); free(tmp); free(u);
  return OR_OK;
}

/* --------------------------------------------------------------- Bi-CGSTAB */

/* Bi-CGSTAB (van der Vorst 1992) as used in Sec. 2, in the usual form:
 *   r = b - Ax, rh = r, p = r, rho = <rh, r>
 *   loop: v = Ap; sigma = <rh, v>; alpha = rho / sigma; s = r - alpha v;
 *         if ||W s|| / ||W r0|| < tol: x += alpha p, stop (half step);
 *         t = As; omega = <t, s> / <t, t>; x += alpha p + omega s;
 *         r = s - omega t; if ||W r|| / ||W r0|| < tol: stop;
 *         rho' = <rh, r>; beta = (rho' / rho)(alpha / omega);
 *         p = r + beta (p - omega v); rho = rho'.
 * Breakdown (Sec. 2.2): |sigma| <= brk ||rh|| ||v|| or |rho'| <= brk ||rh|| ||r||
 * with brk = 1e-16 * DBL_EPSILON, or <t, t> = 0, or omega = 0.
 * When the recursive residual meets tol the true residual b - Ax is formed;
 * if it does not meet tol and refreshes remain, r is replaced by the true
 * residual (rh = p = r) and the iteration continues; otherwise the outcome is
 * OR_STAGNATED.  An iteration is one pass with two products by A; a half-step
 * exit counts as one iteration.
 *
 * hist (optional, length maxit) receives the recursive metric per iteration.
 * trace (optional, 2 * trace_cap doubles) receives one record per
 * true-residual confirmation: the iteration count at that point and the
 * true metric found (records past trace_cap are dropped).  Neither output
 * changes the arithmetic. */
int or_bicgstab(int n, const int* rp, const int* ci, const double* va,
                const double* b, double* x, double tol, int maxit, int refresh,
                const double* w_in, const double* lu, or_info* info, double* hist,
                double* trace, int trace_cap) {
  memset(info, 0, sizeof(*info));
  if (n < 0 || maxit < 0 || !(tol >= 0.0) || refresh < 0) return OR_ERR_ARG;
  /* the empty system: converged at x0, as for mu0 = 0 below */
  if (n == 0) { info->conv = OR_CONVERGED; return OR_OK; }
  size_t nn = (size_t)n;
  double* r = (double*)malloc(sizeof(double) * nn);
  double* rh = (double*)malloc(sizeof(double) * nn);
  double* p = (double*)malloc(sizeof(double) * nn);
  double* v = (double*)malloc(sizeof(double) * nn);
  double* s = (double*)malloc(sizeof(double) * nn);
  double* t = (double*)malloc(sizeof(double) * nn);
  double* wv = (double*)malloc(sizeof(double) * nn);
  double* ph = (double*)malloc(sizeof(double) * nn); /* M^-1 p */
  double* sh = (double*)malloc(sizeof(double) * nn); /* M^-1 s */
  if (!r || !rh || !p || !v || !s || !t || !wv || !ph || !sh) {
    free(r); free(rh); free(p); free(v); free(s); free(t); free(wv); free(ph); free(sh);
    return OR_ERR_OOM;
  }
  /* with a preconditioner M = LU (right preconditioning) the products are
   * A M^-1 p and A M^-1 s, and x moves along M^-1 p and M^-1 s; without one
   * ph and sh are p and s themselves */
  const double* pp = lu ? ph : p;
  const double* ss = lu ? sh : s;
  const double brk = 1e-16 * DBL_EPSILON;
  const double* w = w_in;
  if (!w) {
    if (or_metric_weights(n, rp, va, wv) != OR_OK) { free(r); free(rh); free(p); free(v); free(s); free(t); free(wv); free(ph); free(sh); return OR_ERR_ZERO_ROW; }
    w = wv;
  }
  residual(n, rp, ci, va, b, x, r);
  double mu0 = wnorm(n, w, r);
  info->conv = OR_MAXIT;
  if (mu0 == 0.0) { info->conv = OR_CONVERGED; goto out; }
  int refresh_left = refresh, nconfirm = 0;
  for (;;) { /* (re)start from the current r */
    memcpy(rh, r, sizeof(double) * nn);
    memcpy(p, r, sizeof(double) * nn);
    double rho = dot(n, rh, r);
    double rhn = sqrt(dot(n, rh, rh));
    int check_true = 0;
    while (!check_true) {
      if (info->iters >= maxit) { info->conv = OR_MAXIT; goto final; }
      if (lu) or_ilu0_apply(n, rp, ci, lu, p, ph);
      or_spmv(n, rp, ci, va, pp, v);
      double sigma = dot(n, rh, v);
      double vn = sqrt(dot(n, v, v));
      if (fabs(sigma) <= brk * rhn * vn) { info->conv = OR_BREAKDOWN; goto final; }
      double alpha = rho / sigma;
      for (size_t i = 0; i < nn; ++i) s[i] = r[i] - alpha * v[i];
      double mus = wnorm(n, w, s) / mu0;
      if (mus < tol) {
        for (size_t i = 0; i < nn; ++i) x[i] += alpha * pp[i];
        info->iters++;
        info->relres_rec = mus;
        if (hist) hist[info->iters - 1] = mus;
        check_true = 1;
        break;
      }
      if (lu) or_ilu0_apply(n, rp, ci, lu, s, sh);
      or_spmv(n, rp, ci, va, ss, t);
      double tt = dot(n, t, t);
      double ts = dot(n, t, s);
      if (tt == 0.0) { info->conv = OR_BREAKDOWN; goto final; }
      double omega = ts / tt;
      for (size_t i = 0; i < nn; ++i) x[i] += alpha * pp[i] + omega * ss[i];
      for (size_t i = 0; i < nn; ++i) r[i] = s[i] - omega * t[i];
      info->iters++;
      double mur = wnorm(n, w, r) / mu0;
      info->relres_rec = mur;
      if (hist) hist[info->iters - 1] = mur;
      if (mur < tol) { check_true = 1; break; }
      if (omega == 0.0) { info->conv = OR_BREAKDOWN; goto final; }
      double rho1 = dot(n, rh, r);
      double rn = sqrt(dot(n, r, r));
      if (fabs(rho1) <= brk * rhn * rn) { info->conv = OR_BREAKDOWN; goto final; }
      double beta = (rho1 / rho) * (alpha / omega);
      for (size_t i = 0; i < nn; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
      rho = rho1;
    }
    /* the recursive residual met tol: confirm with the true residual */
    residual(n, rp, ci, va, b, x, t);
    double mu = wnorm(n, w, t) / mu0;
    if (trace && nconfirm < trace_cap) {
      trace[2 * nconfirm + 0] = info->iters;
      trace[2 * nconfirm + 1] = mu;
    }
    nconfirm++;
    if (mu < tol) { info->conv = OR_CONVERGED; info->relres_true = mu; goto out; }
    if (refresh_left == 0) { info->conv = OR_STAGNATED; info->relres_true = mu; goto out; }
    refresh_left--;
    info->refreshes++;
    memcpy(r, t, sizeof(double) * nn);
  }
final:
  residual(n, rp, ci, va, b, x, t);
  info->relres_true = wnorm(n, w, t) / mu0;
out:
  free(r); free(rh); free(p); free(v); free(s); free(t); free(wv); free(ph); free(sh);
  return OR_OK;
}
