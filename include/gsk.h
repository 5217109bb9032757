/*
 * gsk.h -- C ABI of the GB300 library for geometric scaling (GS(p)) and the
 * restarted GMRES(m) / Bi-CGSTAB solvers of
 *   D. Gordon, R. Gordon, "Geometric scaling: a simple preconditioner for
 *   certain linear systems with discontinuous coefficients" (2009).
 *
 * Conventions for every entry point:
 *  - Matrices are CSR with int32 row pointers and column indices (columns in
 *    any order within a row, each index in [0, n)), values FP64 or FP32.
 *  - Every array pointer that names matrix or vector data is a DEVICE pointer
 *    owned by the caller; the library never frees it.  The library owns only
 *    the workspace held by a gsk_ctx.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Work is ordered on that stream.
 *  - Every kernel bounds-checks the CSR structure it reads (rowptr extents,
 *    column indices); a malformed matrix yields GSK_ERR_ARG, never an
 *    out-of-range access.
 *  - No C++ exception crosses the ABI.  Every call returns a gsk_status; the
 *    text of the last error of a context is available from gsk_last_error.
 *  - Non-convergence is not an error: a solve returns GSK_OK with
 *    info->conv != GSK_CONVERGED (a run that misses the goal within maxit,
 *    which the paper's tables mark as not converged, Sec. 2.2).
 *  - One context runs one solve at a time: calls that share a context must be
 *    issued on the same stream (or be serialised by the caller).  Use one
 *    context per concurrent stream.
 */
#ifndef GSK_H
#define GSK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GSK_OK = 0,
  GSK_ERR_ARG = 1,        /* invalid size, pointer, parameter or CSR structure */
  GSK_ERR_ZERO_ROW = 2,   /* a row of A is all zeros (Sec. 2 assumes none) */
  GSK_ERR_NONFINITE = 3,  /* NaN or Inf in A or b */
  GSK_ERR_OOM = 4,        /* workspace allocation failed */
  GSK_ERR_CUDA = 5,       /* a CUDA runtime call failed (see gsk_last_error) */
  GSK_ERR_TIMEOUT = 6     /* a bounded device-side wait gave up */
} gsk_status;

typedef enum { GSK_F64 = 0, GSK_F32 = 1 } gsk_dtype;

typedef enum {
  GSK_CONVERGED = 0,  /* the stopping metric fell below tol */
  GSK_MAXIT = 1,      /* the iteration cap was reached first */
  GSK_BREAKDOWN = 2,  /* a Bi-CGSTAB breakdown test fired (Sec. 2.2) */
  GSK_STAGNATED = 3   /* the recursive residual met tol, the true one did not */
} gsk_conv;

typedef enum {
  GSK_METRIC_GS2 = 0,   /* Sec. 2.2: ||W(b-Ax)||/||W(b-Ax0)||, W = GS(2) scales of A */
  GSK_METRIC_PLAIN = 1  /* ||b-Ax||/||b-Ax0|| of the system as given */
} gsk_metric;

typedef enum {
  GSK_PREC_F64 = 0,   /* every vector and product in FP64 */
  GSK_PREC_MIXED = 1  /* FP32 inner Krylov solves inside FP64 iterative refinement;
                         when a refinement step stops paying off (less than 10x
                         for Bi-CGSTAB, no progress for a GMRES cycle) the solve
                         is finished by the FP64 solver from the current x */
} gsk_precision;

typedef struct gsk_ctx gsk_ctx;

/* A sparse n x n matrix.  rowptr has n+1 entries with rowptr[0] = 0 and
 * rowptr[n] = nnz, non-decreasing; colidx and val have nnz entries. */
typedef struct {
  int32_t n;
  int32_t nnz;
  const int32_t* rowptr; /* device [n+1] */
  const int32_t* colidx; /* device [nnz] */
  void* val;             /* device [nnz], FP64 or FP32 per dtype */
  int32_t dtype;         /* gsk_dtype */
} gsk_csr;

/* ILU(0) factors of a matrix on the device (gsk_ilu0_create). */
typedef struct gsk_ilu0 gsk_ilu0;

/* Solver options; gsk_opts_default() fills the paper's settings. */
typedef struct {
  int32_t maxit;          /* iteration cap, default 10000 (Sec. 2.2) */
  int32_t refresh;        /* Bi-CGSTAB: true-residual restarts allowed after
                             the recursive residual met tol, default 3 */
  int32_t precision;      /* gsk_precision, default GSK_PREC_F64 */
  int32_t metric;         /* gsk_metric, default GSK_METRIC_GS2 */
  const double* weights;  /* optional device [n] metric weights W (overrides
                             metric); NULL = derive them from `metric` */
  double inner_tol;       /* mixed precision: relative tolerance of each FP32
                             inner solve, default 1e-5 */
  int32_t inner_maxit;    /* mixed precision: iterations per inner solve; 0 (the
                             default) means m for GMRES (one cycle) and maxit
                             for Bi-CGSTAB */
  int32_t max_refinements;/* mixed precision: cap on outer FP64 refinement steps
                             (for GMRES one step is one inner cycle); 0, the
                             default, means no cap beyond maxit, which always
                             bounds the total inner iterations */
  const gsk_ilu0* precond;/* optional ILU(0) preconditioner of the matrix being
                             solved, applied on the right (x = M^-1 u), so the
                             residual and the stopping metric stay those of
                             A x = b; NULL (the default) = none.  FP64 solvers
                             only (GSK_ERR_ARG with GSK_PREC_MIXED) */
  int32_t batch_block;    /* batched solvers: threads per block, one block per
                             system: 128, 256 or 512; 0 (the default) = 256.
                             The autotuner (paper_0812_2769_gb300.autotune)
                             picks it by timing candidates */
  int32_t batch_large_n;  /* batched solvers: systems with more rows than
                             this are solved one at a time by the grid-wide
                             solvers instead of by one block; 0 (the default)
                             = every system takes one block */
} gsk_opts;

/* Result of a solve (host memory). */
typedef struct {
  int32_t iters;        /* GMRES: Arnoldi steps over all cycles; Bi-CGSTAB:
                           iterations (two products by A each); for mixed
                           precision the sum over inner solves */
  int32_t restarts;     /* GMRES cycles after the first */
  int32_t refreshes;    /* Bi-CGSTAB true-residual restarts taken */
  int32_t refinements;  /* mixed precision: outer FP64 steps */
  int32_t conv;         /* gsk_conv */
  double relres_true;   /* metric of the returned x, from a true residual */
  double relres_rec;    /* last recursive / least-squares estimate seen */
  float ms;             /* device time of the solve (CUDA events) */
} gsk_info;

/* Library version string. */
const char* gsk_version(void);

/* Create a context on `device` (owns workspace, cached graphs, streams). */
gsk_status gsk_ctx_create(gsk_ctx** ctx, int device);
/* Destroy a context and free its workspace; NULL is accepted. */
gsk_status gsk_ctx_destroy(gsk_ctx* ctx);
/* Text describing the last error on this context ("" if none). */
const char* gsk_last_error(gsk_ctx* ctx);

/* Default options: maxit 10000, refresh 3, FP64, GS(2) metric. */
void gsk_opts_default(gsk_opts* opts);

/*
 * gs_scale -- geometric scaling GS(p) (Sec. 1; Sec. 2, Eq. (2)).
 * Divides row i of A, and b_i, by ||a_i||_p, the L_p norm of the row's
 * coefficients (sum |a_ij|^p)^(1/p); p = INFINITY gives max_j |a_ij|.
 * Afterwards every row of A has unit L_p norm; the solution is unchanged.
 *   A      in/out: values scaled in place (FP64 or FP32)
 *   b      in/out: device [n], same dtype as A, scaled in place; may be NULL
 *   p      >= 1, or INFINITY
 *   d_out  optional device FP64 [n]: receives d_i = 1/||a_i||_p (the diagonal
 *          of D), 0 for a row in error; NULL to skip
 * One pass over the matrix: each row's norm is formed and the row scaled as
 * it is read, so its values are read once and written once.
 * Accuracy: d_i is within a few ulp of the exact 1/||a_i||_p.  For FP64
 * values and p = 1 or 2, on rows whose largest magnitude lies within
 * 2^+-1000 (p = 1) or 2^+-480 (p = 2, rows of at most 4,095 entries), the
 * sum of |a_ij|^p is formed in integer arithmetic on the aligned
 * significands and rounded once (within an ulp of the exact sum, whatever
 * the order of the row's entries); other rows are summed in FP64 after an
 * exact power-of-two rescaling.
 * Errors: GSK_ERR_ARG (p < 1, bad sizes/pointers, row pointers out of
 * range), GSK_ERR_ZERO_ROW (a row is all zero, or its norm is below 2^-1024),
 * GSK_ERR_NONFINITE (NaN or Inf in a row or in b).  On error the rows that
 * caused it (with their b entries), and every row of a 32-row tile whose row
 * pointers are out of range, are left unmodified; the other rows are scaled.
 * gs_scale_static checks every row before it scales any, and leaves A and b
 * entirely unmodified on error.
 * Synchronises `stream` to read the error flags back.
 */
gsk_status gs_scale(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* d_out, void* stream);

/*
 * gs_scale_static -- the same GS(p) scaling as gs_scale for callers that may
 * not allocate device memory: code running where the memory is owned by
 * someone else (a host application with a fixed device-memory budget or its
 * own pool, a plugin that must not touch the allocator) and so cannot create
 * a gsk_ctx, whose workspace is allocated.  The paper has no counterpart; it
 * is an interface variant of gs_scale.
 * It takes no context and calls no allocating CUDA routine.  Its scratch (an
 * error word and, when d_out is NULL, the per-row scales) is a fixed array of
 * 8 MiB + 256 B compiled into the library, which every GPU that loads the
 * library holds until the process exits.
 *   A, b, p, d_out, stream   as for gs_scale (device pointers, caller-owned)
 * It checks every row before it scales any (two passes over the values), and
 * on valid input its result is bit-identical to gs_scale's.
 * Limits and errors: with d_out == NULL, at most 1,048,576 rows (larger n
 * returns GSK_ERR_ARG; pass d_out to scale larger systems, then only the
 * error word is used); also GSK_ERR_ARG / GSK_ERR_ZERO_ROW / GSK_ERR_NONFINITE
 * as gs_scale, but here A and b are left entirely unmodified on error;
 * GSK_ERR_CUDA if a CUDA call fails.  No error text is kept (there is no
 * context).  The scratch array lives on the device that is current when the
 * call is made, which must be the device holding A and b.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the array and clears the
 * error word itself; calls whose work overlaps on the GPU (other streams, other
 * threads) race on the array, so serialise them.  Synchronises `stream`.
 */
gsk_status gs_scale_static(gsk_csr* A, void* b, double p, double* d_out, void* stream);

/*
 * gs_scale_sym -- the two-sided variant of geometric scaling the paper also
 * tried (Sec. 2, after the description of the experiments): with
 * D = diag(1/||a_i||_p), A becomes D^(1/2) A D^(1/2) and b becomes
 * D^(1/2) b.  The scaled system's solution is y = D^(-1/2) x; recover x with
 * gsk_diag_mul(s_out, y).
 *   A      in/out: values scaled in place (FP64 or FP32): a_ij s_i s_j
 *   b      in/out: device [n], A's dtype, scaled in place (b_i s_i); may be NULL
 *   p      >= 1, or INFINITY
 *   s_out  required device FP64 [n]: s_i = (1/||a_i||_p)^(1/2)
 *   w_out  optional device FP64 [n]: w_i = (1/||a_i||_2) / s_i.  Passed as
 *          gsk_opts.weights to a solver of the scaled system, it makes the
 *          stopping metric the GS(2)-scaled residual of the ORIGINAL system
 *          (Sec. 2.2), since the scaled residual is D^(1/2)(b - A x).
 * Errors: GSK_ERR_ARG (p < 1, bad sizes/pointers, a column index outside
 * [0, n)), GSK_ERR_ZERO_ROW, GSK_ERR_NONFINITE; on error A and b are left
 * unmodified.  Synchronises `stream` to read the error flags back.
 */
gsk_status gs_scale_sym(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* s_out, double* w_out, void* stream);

/*
 * gsk_diag_mul -- x_i <- s_i x_i for i < n (x of dtype, s FP64; device
 * pointers).  With s from gs_scale_sym it turns the scaled system's solution
 * y into x = D^(1/2) y (Sec. 2).  Asynchronous on `stream`.
 */
gsk_status gsk_diag_mul(gsk_ctx* ctx, int n, const double* s, void* x, gsk_dtype dtype, void* stream);

/*
 * gsk_ilu0_create -- ILU(0) factors of A for right preconditioning (Sec. 2:
 * the paper's ILUT with drop tolerance 0 and fill-in 1 acted as ILU(0)).
 * L (unit lower) and U have A's sparsity pattern (Saad's IKJ form: for each
 * row i and k < i in its pattern, l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj
 * for the j > k present in both rows).  The rows are processed by level sets
 * of their dependency graph, computed on the host from A's structure (one
 * copy of rowptr and colidx to the host); the factorisation and every later
 * application run on the device, one cooperative launch each.
 *   A    FP64, every row holding its diagonal, columns sorted within a row.
 *        The handle keeps A's rowptr and colidx pointers: they must stay
 *        valid and unchanged while the handle is used (its values are
 *        copied).
 *   out  receives the handle (owns device memory; free with gsk_ilu0_destroy)
 * Errors: GSK_ERR_ARG (FP32 matrix, missing diagonal, unsorted or
 * out-of-range columns), GSK_ERR_ZERO_ROW (a zero pivot), GSK_ERR_OOM,
 * GSK_ERR_CUDA; GSK_ERR_TIMEOUT if a bounded wait between levels gave up.
 * Synchronises `stream`.  One solve at a time may use a handle.
 */
gsk_status gsk_ilu0_create(gsk_ctx* ctx, const gsk_csr* A, gsk_ilu0** out, void* stream);
gsk_status gsk_ilu0_destroy(gsk_ilu0* ilu);

/*
 * gsk_ilu0_apply -- z = (LU)^-1 r: forward substitution with L, backward with
 * U, by level sets.  r, z: device FP64 [n], distinct.  Asynchronous on
 * `stream`; a timed-out wait is reported by the next gsk_ilu0_create or by
 * the solve that uses the handle.
 */
gsk_status gsk_ilu0_apply(gsk_ctx* ctx, const gsk_ilu0* ilu, const double* r, double* z, void* stream);

/*
 * gsk_ilu0_info -- the handle's level schedule: the number of levels of the
 * forward (L) and backward (U) sweeps, and whether the sweeps run in one
 * thread block with z in shared memory (1: systems whose z fits there) or
 * across the grid with a barrier between levels (0).  Host pointers; any
 * may be NULL.  GSK_ERR_ARG for a NULL handle.
 */
gsk_status gsk_ilu0_info(const gsk_ilu0* ilu, int* levels_lower, int* levels_upper, int* one_block);

/*
 * gsk_spmv -- y = A x, the product every Krylov step performs (Sec. 2).
 *   x, y   device [n] of A's dtype; x and y must not overlap.
 * Asynchronous on `stream`.
 */
gsk_status gsk_spmv(gsk_ctx* ctx, const gsk_csr* A, const void* x, void* y, void* stream);

/*
 * gmres_solve -- restarted GMRES(m) with classical Gram-Schmidt applied twice
 * (Sec. 2) on the system as given (apply gs_scale first for GS).
 *   b      device [n], A's dtype
 *   x      in: initial guess x0 (zeros = the paper's u0 = 0, Sec. 2.1);
 *          out: solution.  Device [n], A's dtype.
 *   m      Krylov dimension per cycle, 1..64
 *   tol    stop when ||W(b-Ax)||/||W(b-Ax0)|| < tol (Sec. 2.2)
 *   opts   NULL for defaults
 *   info   host pointer or NULL; when non-NULL the call synchronises `stream`
 *          and fills it.
 * The whole solve runs on the device: no host round trip per iteration.
 * Small systems (FP64, no preconditioner, at most
 * gsk_gmres_small_system_rows rows for this m) run on one thread-block
 * cluster; the decisions are the same, the sums are added in another order.
 */
gsk_status gmres_solve(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                       const gsk_opts* opts, gsk_info* info, void* stream);

/*
 * gsk_arnoldi -- the Arnoldi process of GMRES (Sec. 2: classical Gram-Schmidt
 * applied twice) on A from v0, for the eigenvalue-distribution diagnostic of
 * Sec. 3 (Tables 1b and 4a): the Ritz values, eigenvalues of the leading
 * k x k block of H, approximate A's extreme eigenvalues.
 *   A      FP64 CSR (device); apply gs_scale first to study the scaled matrix
 *   v0     device [n] FP64, the starting vector (normalised here; not modified)
 *   m      number of steps, 1..64
 *   H      host [(m+1) * m] FP64, column-major with leading dimension m+1:
 *          A V_k = V_{k+1} H(0:k+1, 0:k) for the orthonormal basis V; entries
 *          beyond the k steps taken are zero
 *   steps  host: k = m, or fewer when the Krylov space becomes invariant
 *          (h_{k+1,k} <= 1e-14 ||A v_k||, the breakdown rule of gmres_solve);
 *          0 when v0 = 0
 * Runs the solver's basis kernels as one CUDA graph launch (recorded on the
 * first call for this matrix, v0 and m, then reused) and synchronises
 * `stream` before returning.  GSK_ERR_ARG for a non-FP64
 * matrix, m outside 1..64 or a NULL pointer; GSK_ERR_NONFINITE when v0 or A
 * v_j is not finite.
 */
gsk_status gsk_arnoldi(gsk_ctx* ctx, const gsk_csr* A, const double* v0, int m, double* H, int* steps,
                       void* stream);

/*
 * bicgstab_solve -- Bi-CGSTAB (Sec. 2; van der Vorst 1992) with breakdown
 * tolerance 1e-16 * DBL_EPSILON relative to the vector norms (Sec. 2.2) and
 * true-residual confirmation.  Arguments as for gmres_solve.  Systems of at
 * most gsk_small_system_rows rows (FP64, no preconditioner) run on one
 * thread-block cluster; the decisions are the same, the dot products are
 * summed in another order.
 */
gsk_status bicgstab_solve(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, double tol,
                          const gsk_opts* opts, gsk_info* info, void* stream);

/*
 * gsk_small_system_rows -- the largest system (rows) that bicgstab_solve runs
 * on one thread-block cluster of this context's device: 16 CTAs holding the
 * iteration vectors in their shared memory, the whole solve in one launch
 * with no kernel boundary per iteration.  FP64 solves without a
 * preconditioner of systems this small take that path; larger ones, and every
 * other solve, the grid-wide solver.  0 when the device cannot launch the
 * cluster.  The environment variable GSK_SMALL_N, read when a context is
 * created, lowers the limit (0 turns the path off).  Host pointer; GSK_ERR_ARG
 * for a NULL argument.
 */
gsk_status gsk_small_system_rows(gsk_ctx* ctx, int* rows);

/*
 * gsk_gmres_small_system_rows -- the largest system (rows, for matrices of
 * about 7 nonzeros per row) that gmres_solve with restart length m runs on
 * one thread-block cluster: 16 CTAs holding the m + 1 basis vectors, x and
 * the metric weights of their rows in shared memory (so the limit falls as
 * m grows), the whole solve in one launch.  Whether a given system takes
 * that path also depends on its nonzeros fitting the CTAs' stages.  0 when
 * the path is off (GSK_SMALL_N=0) or the device cannot launch the cluster.
 * m in 1..64; host pointer; GSK_ERR_ARG otherwise.
 */
gsk_status gsk_gmres_small_system_rows(gsk_ctx* ctx, int m, int* rows);

/*
 * bicgstab_solve_batched -- GS(p) then Bi-CGSTAB (Sec. 2) on nsys independent
 * systems in one persistent kernel launch: each thread block takes the next
 * system from a work queue (largest first), scales it, solves it with
 * block-level reductions and takes another.  A system's result does not
 * depend on the rest of the batch (bit-identical alone and in any batch).
 *   A       host array [nsys] of FP64 CSR descriptors (device data)
 *   b, x    host arrays [nsys] of device pointers (FP64 [n_i]); x holds x0 on
 *           entry and the solution on exit
 *   p       host array [nsys]: GS(p_i) is applied in place to A[i] and b[i]
 *           first (p_i >= 1 or INFINITY); NaN means no scaling; NULL = NaN for all
 *   tol     stopping tolerance of the metric of Sec. 2.2 (GS(2)-scaled residual)
 *   opts    maxit, refresh, metric; precision GSK_PREC_MIXED runs FP32 inner
 *           solves (relative tolerance inner_tol, at most inner_maxit
 *           iterations each, 40 when 0) in FP64 refinement; a system whose
 *           refinement step gains less than 10x in the FP64 metric is
 *           finished by FP64 Bi-CGSTAB from its current x;
 *           batch_block (threads per block: 128, 256, 512; 0 = 256) and
 *           batch_large_n (systems with more rows are solved one at a
 *           time by gs_scale and the grid-wide solver with the same
 *           options, beside the persistent launch: on a second stream with
 *           a child context of ctx, which keeps its own workspace; `stream`
 *           waits for them before the call returns; 0 = none) shape the
 *           launch
 *   infos   host array [nsys] or NULL; status host array [nsys] or NULL
 *           (per-system gsk_status: GSK_ERR_ZERO_ROW / NONFINITE / ARG).
 * When infos or status is given the call synchronises `stream`; it returns
 * the first failing system's status (the others are still solved).
 */
gsk_status bicgstab_solve_batched(gsk_ctx* ctx, int nsys, const gsk_csr* A, void* const* b, void* const* x,
                                  const double* p, double tol, const gsk_opts* opts, gsk_info* infos,
                                  int32_t* status, void* stream);

/*
 * gmres_solve_batched -- GS(p) then restarted GMRES(m_i) with classical
 * Gram-Schmidt applied twice (Sec. 2) on nsys independent systems in one
 * persistent launch, one thread block per system (the basis in the block's
 * scratch), with the cycle and stopping rules of gmres_solve.  Arguments as
 * bicgstab_solve_batched, plus
 *   m       host array [nsys]: restart length of each system, 1..64
 * The one-block path is FP64; precision GSK_PREC_MIXED is accepted only for
 * systems routed to the grid-wide solver by batch_large_n (GSK_ERR_ARG
 * otherwise).  Bit-identical alone and in any batch for a given batch_block.
 */
gsk_status gmres_solve_batched(gsk_ctx* ctx, int nsys, const gsk_csr* A, void* const* b, void* const* x,
                               const double* p, const int* m, double tol, const gsk_opts* opts, gsk_info* infos,
                               int32_t* status, void* stream);

/* One timed kernel launch of gsk_profile_solve. */
typedef struct {
  int32_t kernel;  /* kernel id, named by gsk_kernel_name */
  int32_t step;    /* Bi-CGSTAB: iteration; GMRES: Arnoldi index j (or -1) */
  float ms;        /* device time between CUDA events around the launch */
} gsk_launch_record;

/* Name of a kernel id of gsk_launch_record ("" if unknown). */
const char* gsk_kernel_name(int kernel);

/*
 * gsk_profile_solve -- runs the same kernels as gmres_solve (solver 0) or
 * bicgstab_solve (solver 1) from a host loop on `stream` instead of one
 * graph launch, with a CUDA event pair around every kernel launch, for at
 * most max_iters iterations (Arnoldi steps for GMRES).  Up to `cap` records
 * are written to recs (host) and their number to *nrec; `info` (host,
 * optional) receives the outcome.  A profiling aid (the paper has no
 * counterpart): the host reads the device state between launches, so the
 * wall time is not that of a solve; the per-launch device times are.
 */
gsk_status gsk_profile_solve(gsk_ctx* ctx, int solver, const gsk_csr* A, const void* b, void* x, int m,
                             double tol, const gsk_opts* opts, int max_iters, gsk_launch_record* recs, int cap,
                             int* nrec, gsk_info* info, void* stream);

/*
 * gsk_profile_gs_scale -- gs_scale (same arguments, same kernel, same
 * results and errors), and the device time of the GS(p) kernel alone in
 * *kernel_ms (host), from a CUDA event pair around its launch on `stream`.
 * A profiling aid: gs_scale's own time also holds the clearing of the error
 * word and the read-back that synchronises the stream.
 */
gsk_status gsk_profile_gs_scale(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* d_out, void* stream,
                                float* kernel_ms);

/* Device workspace a solve of this shape needs (solver: 0 = GMRES, 1 =
 * Bi-CGSTAB), so that callers can budget HBM before admitting work. */
gsk_status gsk_workspace_bytes(int n, int nnz, int solver, int m, int precision, size_t* bytes);

#ifdef __cplusplus
}
#endif
#endif /* GSK_H */
