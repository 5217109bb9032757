// Mixed precision: FP32 inner Krylov solves inside FP64 iterative refinement.
//
// GS keeps every row of the scaled system at unit L_2 norm, which is what
// lets the inner solves run in FP32.  Let W2 = diag(1/||a_i||_2) (the GS(2)
// scales of A).  The inner matrix is (W2 A) rounded to FP32, made once per
// solve.  Each refinement step, all on the device:
//   r = b - A x                      FP64 product, FP64 residual
//   metric ||W r|| / ||W r0||        FP64 (W as for the FP64 solvers)
//   r32 = W2 r / ||W2 r||            scaled to unit norm, rounded to FP32
//   (W2 A)_32 d = r32                FP32 Bi-CGSTAB to a relative tolerance
//                                    inner_tol, or one FP32 GMRES cycle of at
//                                    most m steps (Hessenberg, Givens and the
//                                    least-squares solve stay FP64)
//   x += ||W2 r|| d                  FP64 update
// until the FP64 metric is below tol, maxit inner iterations or
// max_refinements steps.  A (W2 A) d = W2 r step solves A (||W2 r|| d) = r,
// so the FP64 residual, the solution update and the Hessenberg least squares
// are the only FP64 work, as the FP32 kernels accumulate in FP32.
//
// Graph: [weights, convert, residual] -> WHILE_outer{ prep -> inner solve ->
// update -> residual }, the inner solve being the Bi-CGSTAB WHILE/IF body or
// the GMRES Arnoldi WHILE body of the FP64 solvers instantiated for float.
// A correction that is not finite is never applied.  A refinement step that
// gains less than 10x (Bi-CGSTAB) or nothing (a GMRES cycle) ends the FP32
// loop as STAGNATED: FP32 is too coarse for the system's conditioning, and the
// solve is finished by the FP64 solver from the current x (one host decision,
// only on that path), with the tolerance rescaled to the first residual.
#include <cfloat>
#include <cmath>

#include "bicgstab_kernels.cuh"
#include "gmres_kernels.cuh"
#include "graph.hpp"

namespace gsk {

struct MxState {
  double mu0, mu, rnorm, tol, mu_prev, stag;
  int refinements, max_ref, total_iters, maxit, conv, stop, w_identity, solver, skip, skipped;
};

struct MxArgs {
  int n, nnz, solver;  // solver 0 = GMRES, 1 = Bi-CGSTAB
  const int* rowptr;
  const int* colidx;
  const double* val;
  float* val32;
  const double* b;
  double* x;
  double* r;
  const double* w2;  // GS(2) scales of A (inner scaling)
  const double* wm;  // metric weights, nullptr when S->w_identity
  MxState* S;
  BcgState* Sb;
  GmState* Sg;
  GridRed red;
  unsigned* cnt;
  int* err;
  cudaGraphConditionalHandle h_outer, h_inner;
  // inner Bi-CGSTAB vectors (x32 is the correction d)
  float *x32, *r32, *rh32, *p32;
  // inner GMRES basis
  float* V32;
  long long ldv;
  int m;
  double *sig, *g, *y;
};

#define MX_ROW_LOOP(a) for (int i = blockIdx.x * kBlock + threadIdx.x; i < (a).n; i += gridDim.x * kBlock)

// (W2 A) in FP32: every nonzero of row i times w2_i, rounded once.
__global__ void __launch_bounds__(kBlock) mx_convert(MxArgs a) {
  MX_ROW_LOOP(a) {
    const int rs = __ldg(a.rowptr + i), re = __ldg(a.rowptr + i + 1);
    if (rs < 0 || re < rs || re > a.nnz) {
      atomicOr(a.err, kErrIndex);
      continue;
    }
    const double wi = __ldg(a.w2 + i);
    for (int k = rs; k < re; ++k) a.val32[k] = (float)(__ldg(a.val + k) * wi);
  }
}

// r = b - A x (FP64); metric and scaling norms; start, continue or stop.
template <bool INIT>
__global__ void __launch_bounds__(kBlock) mx_residual(MxArgs a) {
  __shared__ PipeSmem<double> pipe;
  __shared__ double blk[2], tot[2];
  double* sm = reinterpret_cast<double*>(&pipe);  // reduction scratch after the product
  MxState* S = a.S;
  const bool wid = S->w_identity;
  double acc[2] = {0.0, 0.0};
  spmv_rows_tma(a.rowptr, a.colidx, a.val, a.x, a.n, a.nnz, pipe, a.err, [&](int i, double ax) {
    const double r = a.b[i] - ax;
    a.r[i] = r;
    const double wr = (wid ? 1.0 : __ldg(a.wm + i)) * r;
    const double w2r = __ldg(a.w2 + i) * r;
    acc[0] = fma(wr, wr, acc[0]);
    acc[1] = fma(w2r, w2r, acc[1]);
  });
  block_sum<2, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    const int e = *(volatile int*)a.err;
    const double mw = sqrt(tot[0]);
    S->rnorm = sqrt(tot[1]);
    int stop = 0;
    if (INIT) {
      S->mu0 = mw;
      S->mu = 1.0;
      S->mu_prev = 1.0;
      S->refinements = 0;
      S->total_iters = 0;
      S->conv = GSK_MAXIT;
      if (e) {
        stop = 1;
      } else if (!isfinite(mw)) {
        atomicOr(a.err, kErrNonFinite);
        stop = 1;
      } else if (mw == 0.0) {
        S->conv = GSK_CONVERGED;
        S->mu = 0.0;
        stop = 1;
      } else if (S->maxit <= 0) {
        stop = 1;
      }
    } else {
      S->refinements += 1;
      S->total_iters += a.solver == 1 ? a.Sb->iters : a.Sg->iters;
      const double mu = mw / S->mu0;
      S->mu = mu;
      if (e) {
        stop = 1;
      } else if (mu < S->tol) {
        S->conv = GSK_CONVERGED;
        stop = 1;
      } else if (S->total_iters >= S->maxit || (S->max_ref > 0 && S->refinements >= S->max_ref) ||
                 !(mu == mu)) {
        S->conv = GSK_MAXIT;
        stop = 1;
      } else if (mu > S->stag * S->mu_prev) {
        // the FP32 step no longer gains enough: hand over to FP64 (host side)
        S->conv = GSK_STAGNATED;
        stop = 1;
      }
      S->mu_prev = mu;
    }
    S->stop = stop;
    cudaGraphSetConditional(a.h_outer, (unsigned)!stop);
  }
}

// Inner Bi-CGSTAB start: r32 = rh32 = p32 = W2 r / ||W2 r||, x32 = 0.
__global__ void __launch_bounds__(kBlock) mx_prep_bcg(MxArgs a) {
  __shared__ double sm[kBlock], blk[1], tot[1];
  const double inv = 1.0 / a.S->rnorm;
  float acc = 0.f;
  MX_ROW_LOOP(a) {
    const float v = (float)(__ldg(a.w2 + i) * a.r[i] * inv);
    a.r32[i] = v;
    a.rh32[i] = v;
    a.p32[i] = v;
    a.x32[i] = 0.f;
    acc = fmaf(v, v, acc);
  }
  const double accd[1] = {(double)acc};
  block_sum<1, kBlock>(accd, sm, blk);
  if (grid_sum(blk, 1, a.red, tot) && threadIdx.x == 0) {
    BcgState* Sb = a.Sb;
    Sb->rho = tot[0];
    Sb->rhn = sqrt(tot[0]);
    Sb->mu0 = sqrt(tot[0]);
    Sb->mu_rec = 1.0;
    Sb->iters = 0;
    Sb->halfexit = 0;
    Sb->check = 0;
    Sb->stop = 0;
    Sb->active = 1;
    Sb->conv = GSK_MAXIT;
    cudaGraphSetConditional(a.h_inner, 1u);
  }
}

// After a round of inner Bi-CGSTAB iterations: go on unless one of them met
// the inner tolerance, broke down or hit the cap.
__global__ void mx_inner_next(MxArgs a) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(a.h_inner, (a.Sb->check || a.Sb->stop) ? 0u : 1u);
}

// Counts non-finite entries of the FP32 correction; a correction that is not
// finite is not applied (S->skip), so x only ever takes finite steps.
__global__ void __launch_bounds__(kBlock) mx_check_bcg(MxArgs a) {
  __shared__ double sm[kBlock], blk[1], tot[1];
  int bad = 0;
  MX_ROW_LOOP(a) bad |= !isfinite(a.x32[i]);
  const double accd[1] = {(double)bad};
  block_sum<1, kBlock>(accd, sm, blk);
  if (grid_sum(blk, 1, a.red, tot) && threadIdx.x == 0) {
    a.S->skip = tot[0] != 0.0;
    a.S->skipped += a.S->skip;
  }
}

// x += ||W2 r|| x32 (FP64), unless the correction was not finite.
__global__ void __launch_bounds__(kBlock) mx_update_bcg(MxArgs a) {
  if (a.S->skip) return;
  const double s = a.S->rnorm;
  MX_ROW_LOOP(a) a.x[i] = fma(s, (double)a.x32[i], a.x[i]);
}

// Inner GMRES cycle start: V32[:, 0] = W2 r / ||W2 r||.
__global__ void __launch_bounds__(kBlock) mx_prep_gm(MxArgs a) {
  __shared__ double sm[kBlock], blk[1], tot[1];
  const double inv = 1.0 / a.S->rnorm;
  float acc = 0.f;
  MX_ROW_LOOP(a) {
    const float v = (float)(__ldg(a.w2 + i) * a.r[i] * inv);
    a.V32[i] = v;
    acc = fmaf(v, v, acc);
  }
  const double accd[1] = {(double)acc};
  block_sum<1, kBlock>(accd, sm, blk);
  if (grid_sum(blk, 1, a.red, tot) && threadIdx.x == 0) {
    const double beta = sqrt(tot[0]);
    GmState* Sg = a.Sg;
    a.sig[0] = 1.0 / beta;
    a.g[0] = beta;
    for (int q = 1; q <= a.m; ++q) a.g[q] = 0.0;
    Sg->rho0 = beta;
    Sg->inv_rho0 = 1.0 / beta;
    Sg->j = 0;
    Sg->iters = 0;
    Sg->kcols = 0;
    Sg->est_hit = 0;
    Sg->est = 1.0;
    Sg->cont = 1;
  }
}

// x += ||W2 r|| V32_k (sig .* y) with FP64 accumulation.
template <int KP>
__global__ void __launch_bounds__(kBlock) mx_update_gm(MxArgs a) {
  __shared__ double coef[KP];
  const int k = a.Sg->kcols;
  const double s = a.S->rnorm;
  for (int c = threadIdx.x; c < k; c += kBlock) coef[c] = s * a.sig[c] * a.y[c];
  __syncthreads();
  // a least-squares solution that is not finite (singular H) is not applied
  for (int c = 0; c < k; ++c)
    if (!isfinite(coef[c])) return;
  MX_ROW_LOOP(a) {
    double x = a.x[i];
#pragma unroll
    for (int c0 = 0; c0 < KP; c0 += 4)
      if (c0 < k) {
#pragma unroll
        for (int c = c0; c < c0 + 4; ++c)
          if (c < k) x = fma((double)a.V32[(long long)c * a.ldv + i], coef[c], x);
      }
    a.x[i] = x;
  }
}

// ------------------------------------------------------------------ host

struct MxPlan {
  int solver, wmode, KP, g_tile, g_vec, g_vec2, m;
  // inner GMRES: grids of the basis kernels per column class (as the FP64
  // solver: the step with k columns runs the instance of class gm_kclass(k))
  int nclass, g_gd[kGmClasses], g_gb[kGmClasses], g_gc[kGmClasses];
  MxArgs a;
  BcgArgs<float> bi;
  GmArgs<float> gi;
  double* wmbuf;
  MxState hs;
  BcgState hb;
  GmState hg;
};

template <int KP>
static void mx_grids_class(gsk_ctx* ctx, MxPlan& P, int c, int n);

static gsk_status mx_prepare(gsk_ctx* ctx, int solver, const gsk_csr* A, const void* b, void* x, int m,
                             double tol, const gsk_opts& opts, MxPlan& P) {
  if (A->dtype != GSK_F64) return ctx->fail(GSK_ERR_ARG, "mixed precision needs an FP64 matrix");
  if (!(tol >= 0.0) || opts.maxit < 0 || !(opts.inner_tol > 0.0) || opts.inner_maxit < 0)
    return ctx->fail(GSK_ERR_ARG, "bad tol/maxit/inner_tol/inner_maxit");
  if (A->n > 0 && (!b || !x)) return ctx->fail(GSK_ERR_ARG, "NULL b or x");
  const int n = A->n;
  P.solver = solver;
  P.m = solver == 0 ? m : 1;
  P.wmode = opts.weights ? 2 : (opts.metric == GSK_METRIC_PLAIN ? 1 : 0);
  P.KP = m <= 16 ? 16 : (m <= 32 ? 32 : 64);
  P.g_tile = ctx->spmv_grid(n);
  P.g_vec = ctx->grid_for(n, kBlock, 4);
  P.g_vec2 = ctx->occ_grid((const void*)bcg_k3<float>, (n + 3) / 4, kBlock);  // four FP32 rows per thread
  int gmax = P.g_tile;
  for (int g : {P.g_vec, P.g_vec2, ctx->grid_for(n, kBlock, 8)}) gmax = g > gmax ? g : gmax;
  P.nclass = 0;
  if (solver == 0) {
    P.nclass = gm_kclass(m) + 1;
    for (int c = 0; c < kGmClasses; ++c) P.g_gd[c] = P.g_gb[c] = P.g_gc[c] = 1;
    mx_grids_class<4>(ctx, P, 0, n);
    if (P.nclass > 1) mx_grids_class<8>(ctx, P, 1, n);
    if (P.nclass > 2) mx_grids_class<16>(ctx, P, 2, n);
    if (P.nclass > 3) mx_grids_class<32>(ctx, P, 3, n);
    if (P.nclass > 4) mx_grids_class<64>(ctx, P, 4, n);
    for (int c = 0; c < P.nclass; ++c)
      for (int g : {P.g_gd[c], P.g_gb[c], P.g_gc[c]}) gmax = g > gmax ? g : gmax;
  }
  const long long ldv = ((long long)n + 63) / 64 * 64;
  MxArgs& a = P.a;
  std::memset(&a, 0, sizeof(a));
  std::memset(&P.bi, 0, sizeof(P.bi));
  std::memset(&P.gi, 0, sizeof(P.gi));
  float *v32 = nullptr, *s32 = nullptr, *t32 = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *h1 = nullptr, *h2 = nullptr;
  auto layout = [&](Arena& ar) {
    a.err = ar.take<int>(64);
    a.cnt = ar.take<unsigned>(64);
    a.red = take_red(ar, gmax, solver == 0 ? m + 2 : 4);
    a.S = ar.take<MxState>(1);
    a.Sb = ar.take<BcgState>(1);
    a.Sg = ar.take<GmState>(1);
    a.val32 = ar.take<float>(A->nnz);
    double* w2 = ar.take<double>(n);
    a.w2 = w2;
    a.r = ar.take<double>(n);
    if (solver == 1) {
      a.x32 = ar.take<float>(n);
      a.r32 = ar.take<float>(n);
      a.rh32 = ar.take<float>(n);
      a.p32 = ar.take<float>(n);
      v32 = ar.take<float>(n);
      s32 = ar.take<float>(n);
      t32 = ar.take<float>(n);
    } else {
      a.V32 = ar.take<float>((size_t)ldv * (m + 1));
      H = ar.take<double>((size_t)(m + 1) * m);
      a.g = ar.take<double>(m + 1);
      cs = ar.take<double>(m);
      sn = ar.take<double>(m);
      a.y = ar.take<double>(m);
      h1 = ar.take<double>(m + 1);
      h2 = ar.take<double>(m + 1);
      a.sig = ar.take<double>(m + 1);
    }
  };
  Arena sizing;
  layout(sizing);
  gsk_status s = ctx->reserve(sizing.off);
  if (s != GSK_OK) return s;
  Arena ar{(char*)ctx->ws, ctx->ws_bytes, 0};
  layout(ar);
  a.n = n;
  a.nnz = A->nnz;
  a.solver = solver;
  a.rowptr = A->rowptr;
  a.colidx = A->colidx;
  a.val = (const double*)A->val;
  a.b = (const double*)b;
  a.x = (double*)x;
  a.wm = P.wmode == 0 ? a.w2 : (P.wmode == 2 ? opts.weights : nullptr);
  a.ldv = ldv;
  a.m = m;

  std::memset(&P.hs, 0, sizeof(P.hs));
  P.hs.tol = tol;
  P.hs.maxit = opts.maxit;
  P.hs.max_ref = opts.max_refinements;
  P.hs.w_identity = P.wmode == 1 ? 1 : 0;
  P.hs.solver = solver;
  // a refinement step must gain 10x (Bi-CGSTAB solve) or make some progress
  // (one GMRES cycle) to continue in FP32
  P.hs.stag = solver == 1 ? 0.1 : 0.99;
  const int inner_maxit = opts.inner_maxit > 0 ? opts.inner_maxit : (solver == 0 ? m : opts.maxit);

  if (solver == 1) {
    BcgArgs<float>& bi = P.bi;
    bi.n = n;
    bi.nnz = A->nnz;
    bi.rowptr = A->rowptr;
    bi.colidx = A->colidx;
    bi.val = a.val32;
    bi.x = a.x32;
    bi.r = a.r32;
    bi.rh = a.rh32;
    bi.p = a.p32;
    bi.v = v32;
    bi.s = s32;
    bi.t = t32;
    bi.p_in = bi.p;
    bi.s_in = bi.s;
    bi.w = nullptr;
    bi.S = a.Sb;
    bi.red = a.red;
    bi.cnt = a.cnt;
    bi.err = a.err;
    bi.in_graph = 1;
    bi.vec_ok = 1;  // every FP32 vector is workspace (256-byte aligned)
    std::memset(&P.hb, 0, sizeof(P.hb));
    P.hb.tol = opts.inner_tol;
    // FP32 rounding noise swamps |<rh, v>| below about FLT_EPSILON ||rh|| ||v||:
    // the inner solve stops there and the refinement restarts it
    P.hb.brk = FLT_EPSILON;
    P.hb.maxit = inner_maxit;
    P.hb.w_identity = 1;
  } else {
    GmArgs<float>& gi = P.gi;
    gi.n = n;
    gi.nnz = A->nnz;
    gi.m = m;
    gi.ldv = ldv;
    gi.rowptr = A->rowptr;
    gi.colidx = A->colidx;
    gi.val = a.val32;
    gi.V = a.V32;
    gi.H = H;
    gi.g = a.g;
    gi.cs = cs;
    gi.sn = sn;
    gi.y = a.y;
    gi.h1 = h1;
    gi.h2 = h2;
    gi.sig = a.sig;
    gi.w = nullptr;
    gi.S = a.Sg;
    gi.red = a.red;
    gi.cnt = a.cnt;
    gi.err = a.err;
    gi.in_graph = 1;
    gi.unrolled = 1;
    std::memset(&P.hg, 0, sizeof(P.hg));
    P.hg.tau = opts.inner_tol;
    P.hg.tol = opts.inner_tol;
    P.hg.hbrk = 1e-6;
    P.hg.m = m;
    P.hg.maxit = inner_maxit;
    P.hg.w_identity = 1;
  }
  return GSK_OK;
}

constexpr int kMxUnroll = 4;  // inner Bi-CGSTAB iterations per loop-body pass

template <int KP>
static void mx_launch_gm(MxPlan& P, int which, cudaStream_t s) {
  switch (which) {
    case 4: gm_gy<float><<<1, kBlock, 0, s>>>(P.gi); break;
    case 5: mx_update_gm<KP><<<P.g_vec, kBlock, 0, s>>>(P.a); break;
  }
}

static void mx_gm(MxPlan& P, int which, cudaStream_t s) {
  if (P.KP == 16) mx_launch_gm<16>(P, which, s);
  else if (P.KP == 32) mx_launch_gm<32>(P, which, s);
  else mx_launch_gm<64>(P, which, s);
}

// One inner Arnoldi step with k = j + 1 basis columns: the product, then the
// CGS passes of the column class of k.
template <int KP>
static void mx_step_kp(MxPlan& P, int c, cudaStream_t s) {
  gm_gd<float, KP><<<P.g_gd[c], kBlock, 0, s>>>(P.gi);
  gm_gb<float, KP><<<P.g_gb[c], kBlock, 0, s>>>(P.gi);
  gm_gc<float, (KP <= 32 ? 32 : 64)><<<P.g_gc[c], kBlock, 0, s>>>(P.gi);
}

static void mx_step(MxPlan& P, int j, cudaStream_t s) {
  gm_ga<float><<<P.g_tile, kBlock, 0, s>>>(P.gi);
  const int c = gm_kclass(j + 1);
  switch (c) {
    case 0: mx_step_kp<4>(P, c, s); break;
    case 1: mx_step_kp<8>(P, c, s); break;
    case 2: mx_step_kp<16>(P, c, s); break;
    case 3: mx_step_kp<32>(P, c, s); break;
    default: mx_step_kp<64>(P, c, s); break;
  }
}

// Grids of the FP32 basis kernels (four rows per thread): as many blocks as
// are resident at each kernel's occupancy.  The FP32 passes are bound by
// memory, not by the FP64 pipe, so no cap below the occupancy.
template <int KP>
static void mx_grids_class(gsk_ctx* ctx, MxPlan& P, int c, int n) {
  const long long rows4 = ((long long)n + 3) / 4;
  P.g_gd[c] = ctx->occ_grid((const void*)gm_gd<float, KP>, rows4, kBlock);
  P.g_gb[c] = ctx->occ_grid((const void*)gm_gb<float, KP>, rows4, kBlock);
  P.g_gc[c] = ctx->occ_grid((const void*)gm_gc<float, (KP <= 32 ? 32 : 64)>, rows4, kBlock);
}

static gsk_status mx_record(gsk_ctx* ctx, MxPlan& P, cudaGraphExec_t* exec_out) {
  cudaStream_t cs = ctx->capture;
  cudaGraph_t top = nullptr;
  GSK_CK(cudaGraphCreate(&top, 0));
  struct Guard {
    cudaGraph_t g;
    ~Guard() { if (g) cudaGraphDestroy(g); }
  } guard{top};
  MxArgs& a = P.a;
  GSK_CK(cudaGraphConditionalHandleCreate(&a.h_outer, top, 1u, cudaGraphCondAssignDefault));
  cudaGraphNode_t onode;
  cudaGraph_t obody;
  GSK_CK(add_conditional(top, {}, a.h_outer, cudaGraphCondTypeWhile, 1, &onode, &obody));
  if (P.solver == 1) {
    GSK_CK(cudaGraphConditionalHandleCreate(&a.h_inner, obody, 1u, 0));
    P.bi.h_while = a.h_inner;
  }

  // init: scales W2 (GS(2) of A), the identity test of the metric weights,
  // (W2 A) in FP32, the first FP64 residual
  Capture c0;
  GSK_CK(c0.begin(cs, top));
  launch_gs_norm(ctx, a.n, a.nnz, a.rowptr, a.val, 2.0, const_cast<double*>(a.w2), a.err, cs);
  if (P.wmode == 0) launch_unit_check(ctx, a.n, a.w2, a.red, &a.S->w_identity, cs);
  mx_convert<<<P.g_vec, kBlock, 0, cs>>>(a);
  mx_residual<true><<<P.g_tile, kBlock, 0, cs>>>(a);
  GSK_CK(c0.end());
  {
    std::vector<cudaGraphNode_t> to(c0.tail.size(), onode);
    GSK_CK(cudaGraphAddDependencies(top, c0.tail.data(), to.data(), nullptr, c0.tail.size()));
  }

  Capture cp;
  GSK_CK(cp.begin(cs, obody));
  if (P.solver == 0) {
    // GMRES: the cycle start, then the inner cycle's m steps unrolled (no
    // inner WHILE node; the steps after the cycle has ended return at entry)
    mx_prep_gm<<<P.g_vec, kBlock, 0, cs>>>(a);
    for (int j = 0; j < P.m; ++j) mx_step(P, j, cs);
    mx_gm(P, 4, cs);
    mx_gm(P, 5, cs);
    mx_residual<false><<<P.g_tile, kBlock, 0, cs>>>(a);
    GSK_CK(cp.end());
  } else {
    mx_prep_bcg<<<P.g_vec, kBlock, 0, cs>>>(a);
    GSK_CK(cp.end());
    cudaGraphNode_t inode;
    cudaGraph_t ibody;
    GSK_CK(add_conditional(obody, cp.tail, a.h_inner, cudaGraphCondTypeWhile, 1, &inode, &ibody));
    // inner body: kMxUnroll iterations in a row (kernels after the iteration
    // that set check or stop return at entry), then the loop condition; no
    // conditional node per iteration
    Capture c1;
    GSK_CK(c1.begin(cs, ibody));
    for (int u = 0; u < kMxUnroll; ++u) {
      bcg_k1<float><<<P.g_tile, kBlock, 0, cs>>>(P.bi);
      bcg_k2a<float><<<P.g_vec2, kBlock, 0, cs>>>(P.bi);
      bcg_k2b<float><<<P.g_tile, kBlock, 0, cs>>>(P.bi);
      bcg_k3<float><<<P.g_vec2, kBlock, 0, cs>>>(P.bi);
      bcg_k4<float><<<P.g_vec2, kBlock, 0, cs>>>(P.bi);
    }
    mx_inner_next<<<1, 32, 0, cs>>>(a);
    GSK_CK(c1.end());
    Capture c4;
    GSK_CK(c4.begin(cs, obody, {inode}));
    mx_check_bcg<<<P.g_vec, kBlock, 0, cs>>>(a);
    mx_update_bcg<<<P.g_vec, kBlock, 0, cs>>>(a);
    mx_residual<false><<<P.g_tile, kBlock, 0, cs>>>(a);
    GSK_CK(c4.end());
  }
  GSK_CK(cudaGraphInstantiate(exec_out, top, 0));
  return GSK_OK;
}

static gsk_status mx_solve(gsk_ctx* ctx, int solver, const gsk_csr* A, const void* b, void* x, int m, double tol,
                           const gsk_opts* opts, gsk_info* info, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  MxPlan P;
  gsk_status s = mx_prepare(ctx, solver, A, b, x, m, tol, *opts, P);
  if (s != GSK_OK) return s;
  if (A->n == 0) {
    if (info) *info = gsk_info{0, 0, 0, 0, GSK_CONVERGED, 0.0, 0.0, 0.f};
    return GSK_OK;
  }
  std::vector<uint64_t> key = {2 + (uint64_t)solver, (uint64_t)A->n, (uint64_t)A->nnz, (uint64_t)m,
                               (uint64_t)A->rowptr, (uint64_t)A->colidx, (uint64_t)A->val, (uint64_t)b,
                               (uint64_t)x, (uint64_t)P.wmode, (uint64_t)P.a.wm, (uint64_t)ctx->ws};
  GraphEntry* ge = ctx->find_graph(key);
  if (!ge) {
    cudaGraphExec_t ex = nullptr;
    if ((s = mx_record(ctx, P, &ex)) != GSK_OK) return s;
    ge = ctx->add_graph(key, ex);
  }
  GSK_CK(cudaEventRecord(ctx->ev0, st));
  const char* end = (const char*)(P.a.red.counters + 1);
  GSK_CK(cudaMemsetAsync(ctx->ws, 0, end - (const char*)ctx->ws, st));
  GSK_CK(cudaMemcpyAsync(P.a.S, &P.hs, sizeof(MxState), cudaMemcpyHostToDevice, st));
  if (solver == 1) GSK_CK(cudaMemcpyAsync(P.a.Sb, &P.hb, sizeof(BcgState), cudaMemcpyHostToDevice, st));
  else GSK_CK(cudaMemcpyAsync(P.a.Sg, &P.hg, sizeof(GmState), cudaMemcpyHostToDevice, st));
  GSK_CK(cudaGraphLaunch(ge->exec, st));
  GSK_CK(cudaEventRecord(ctx->ev1, st));
  if (!info) return GSK_OK;
  char* hp = (char*)ctx->host_pinned;
  GSK_CK(cudaMemcpyAsync(hp, P.a.S, sizeof(MxState), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaMemcpyAsync(hp + 512, P.a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaMemcpyAsync(hp + 1024, P.a.Sb, sizeof(BcgState), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaMemcpyAsync(hp + 2048, P.a.Sg, sizeof(GmState), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  MxState out;
  BcgState ob;
  GmState og;
  int bits;
  std::memcpy(&out, hp, sizeof(out));
  std::memcpy(&bits, hp + 512, sizeof(int));
  std::memcpy(&ob, hp + 1024, sizeof(ob));
  std::memcpy(&og, hp + 2048, sizeof(og));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  const double inner_rec = solver == 1 ? ob.mu_rec : og.est;
  *info = gsk_info{out.total_iters, (solver == 0 && out.refinements > 0) ? out.refinements - 1 : 0, 0,
                   out.refinements, out.conv, out.mu,
                   inner_rec, ms};
  gsk_status st_bits = err_bits_status(ctx, bits);
  if (st_bits != GSK_OK || out.conv != GSK_STAGNATED || !(out.mu > 0.0) || !std::isfinite(out.mu) ||
      out.total_iters >= opts->maxit)
    return st_bits;
  // The refinement stopped short of tol (FP32 too coarse for this system):
  // finish in FP64 from the current x, the tolerance rescaled so that it is
  // still relative to the first residual.
  gsk_opts o64 = *opts;
  o64.precision = GSK_PREC_F64;
  o64.maxit = opts->maxit - out.total_iters;
  gsk_info i64;
  gsk_status s64 = solver == 1 ? bicgstab_solve(ctx, A, b, x, tol / out.mu, &o64, &i64, stream)
                               : gmres_solve(ctx, A, b, x, m, tol / out.mu, &o64, &i64, stream);
  if (s64 != GSK_OK) return s64;
  info->iters += i64.iters;
  info->refreshes = i64.refreshes;
  info->conv = i64.conv;
  info->relres_true = i64.relres_true * out.mu;
  info->relres_rec = i64.relres_rec * out.mu;
  info->ms += i64.ms;
  return GSK_OK;
}

}  // namespace gsk

gsk_status gmres_solve_mixed(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                             const gsk_opts* opts, gsk_info* info, void* stream) {
  if (opts && opts->precond) return ctx->fail(GSK_ERR_ARG, "no preconditioner with mixed precision");
  return gsk::mx_solve(ctx, 0, A, b, x, m, tol, opts, info, stream);
}

gsk_status bicgstab_solve_mixed(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, double tol,
                                const gsk_opts* opts, gsk_info* info, void* stream) {
  if (opts && opts->precond) return ctx->fail(GSK_ERR_ARG, "no preconditioner with mixed precision");
  return gsk::mx_solve(ctx, 1, A, b, x, 30, tol, opts, info, stream);
}
