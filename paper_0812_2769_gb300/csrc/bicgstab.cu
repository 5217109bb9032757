// Bi-CGSTAB (Sec. 2; van der Vorst 1992) with every scalar and every
// stopping decision on the device.
//
// One iteration is the kernel chain
//   k1  v = A p,           sigma = <rh, v>, ||v||         -> alpha or breakdown
//   k2a s = r - alpha v,   ||W s||                         -> half-step exit?
//   k2b t = A s,           <t, s>, <t, t>                  -> omega or breakdown
//   k3  x += alpha p + omega s, r = s - omega t,
//                          <rh, r>, ||W r||, ||r||         -> beta, flags
//   then either k4  p = r + beta (p - omega v)             (keep iterating)
//   or          kt  t = b - A x, ||W t||, ||t||            (true residual)
//               kr  finish, or refresh r = rh = p = t
// The chain is recorded once into a CUDA graph: a WHILE node repeats the
// iteration and an IF/ELSE node picks k4 or kt+kr, both driven by values the
// kernels set on the device, so a solve is one graph launch.  The same
// kernels can also be driven from a host loop with a CUDA event around each
// launch (gsk_profile_solve); every kernel then checks the device flags
// itself, which the graph's conditional nodes make redundant.
//
// The breakdown tolerance is 1e-16 * DBL_EPSILON relative to the vector
// norms (Sec. 2.2).  The stopping metric is ||W(b - Ax)|| / ||W(b - Ax0)||
// with W the GS(2) scales of A (Sec. 2.2); when W is the identity to within
// 4 ulp (an already GS(2)-scaled system) the weight loads are skipped and
// ||r|| is taken from ||W r||.
#include <cfloat>

#include "graph.hpp"
#include "internal.hpp"

namespace gsk {

struct BcgState {
  double rho, alpha, omega, beta, rhn, mu0, mu_s, mu_rec, mu_true, tt_true, tol, brk;
  int maxit, refresh_left, iters, refreshes, conv, stop, halfexit, check, active, w_identity;
};

template <typename T>
struct BcgArgs {
  int n, nnz;
  const int* rowptr;
  const int* colidx;
  const T* val;
  const T* b;
  T* x;
  T *r, *rh, *p, *v, *s, *t;
  const double* w;
  BcgState* S;
  GridRed red;
  unsigned* cnt;
  int* err;
  cudaGraphConditionalHandle h_while, h_if;
  int in_graph;
};

template <typename T>
__device__ __forceinline__ void set_cond(const BcgArgs<T>& a, cudaGraphConditionalHandle h, unsigned v) {
  if (a.in_graph) cudaGraphSetConditional(h, v);
}

#define BCG_TILE_LOOP(a) \
  for (int tile = blockIdx.x * kWarpsPerBlock + warp_id(), ntiles_ = ((a).n + 31) / 32; tile < ntiles_; \
       tile += gridDim.x * kWarpsPerBlock)

// Two rows per thread per trip (i and i + stride) so that each thread keeps
// twice the loads in flight; the row-to-thread map depends only on the grid.
#define BCG_ROW2_LOOP(a)                                                        \
  for (int i = blockIdx.x * kBlock + threadIdx.x, stride_ = gridDim.x * kBlock; \
       i < (a).n; i += 2 * stride_)

__device__ __forceinline__ double wgt(const double* w, bool wid, int i) { return wid ? 1.0 : __ldg(w + i); }

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_init(BcgArgs<T> a) {
  __shared__ TileStage<T, kStageCap> stage[kWarpsPerBlock];
  __shared__ double blk[2], tot[2];
  double* sm = reinterpret_cast<double*>(stage);  // reduction scratch after the tile loop
  BcgState* S = a.S;
  const bool wid = S->w_identity;
  double acc[2] = {0.0, 0.0};
  BCG_TILE_LOOP(a) {
    const int i = tile * 32 + lane_id();
    const T ax = csr_tile_row<T, T, kStageCap>(a.rowptr, a.colidx, a.val, a.x, a.n, a.nnz, tile * 32,
                                                 stage[warp_id()], a.err);
    if (i < a.n) {
      const T r = a.b[i] - ax;
      a.r[i] = r;
      a.rh[i] = r;
      a.p[i] = r;
      const double wr = wgt(a.w, wid, i) * (double)r;
      acc[0] = fma(wr, wr, acc[0]);
      acc[1] = fma((double)r, (double)r, acc[1]);
    }
  }
  block_sum<2, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    const int e = *(volatile int*)a.err;
    const double mu0 = sqrt(tot[0]);
    S->iters = 0;
    S->refreshes = 0;
    S->halfexit = 0;
    S->check = 0;
    S->mu0 = mu0;
    S->rho = tot[1];
    S->rhn = sqrt(tot[1]);
    S->mu_rec = 1.0;
    S->mu_true = 1.0;
    S->conv = GSK_MAXIT;
    int active = 1;
    if (e) {
      active = 0;
    } else if (!isfinite(mu0)) {
      atomicOr(a.err, kErrNonFinite);
      active = 0;
    } else if (mu0 == 0.0) {
      S->conv = GSK_CONVERGED;
      S->mu_true = 0.0;
      S->mu_rec = 0.0;
      active = 0;
    } else if (S->maxit <= 0) {
      active = 0;
    }
    S->stop = !active;
    S->active = active;
    set_cond(a, a.h_while, active);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k1(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop) return;
  __shared__ TileStage<T, kStageCap> stage[kWarpsPerBlock];
  __shared__ double blk[2], tot[2];
  double* sm = reinterpret_cast<double*>(stage);  // reduction scratch after the tile loop
  const T* __restrict__ rh = a.rh;
  T* __restrict__ vout = a.v;
  double acc[2] = {0.0, 0.0};
  BCG_TILE_LOOP(a) {
    const int i = tile * 32 + lane_id();
    const T v = csr_tile_row<T, T, kStageCap>(a.rowptr, a.colidx, a.val, a.p, a.n, a.nnz, tile * 32,
                                                stage[warp_id()], a.err);
    if (i < a.n) {
      vout[i] = v;
      acc[0] = fma((double)rh[i], (double)v, acc[0]);
      acc[1] = fma((double)v, (double)v, acc[1]);
    }
  }
  block_sum<2, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    const double sigma = tot[0], vn = sqrt(tot[1]);
    if (*(volatile int*)a.err) {
      S->stop = 1;
    } else if (!(fabs(sigma) > S->brk * S->rhn * vn)) {
      S->conv = GSK_BREAKDOWN;
      S->stop = 1;
    } else {
      S->alpha = S->rho / sigma;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k2a(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop) return;
  __shared__ double sm[1 * kBlock], blk[1], tot[1];
  const double alpha = S->alpha;
  const bool wid = S->w_identity;
  const T* __restrict__ r = a.r;
  const T* __restrict__ v = a.v;
  T* __restrict__ s = a.s;
  double acc[1] = {0.0};
  BCG_ROW2_LOOP(a) {
    const int i2 = i + stride_;
    const bool two = i2 < a.n;
    const double r1 = (double)r[i], v1 = (double)v[i];
    const double r2 = two ? (double)r[i2] : 0.0, v2 = two ? (double)v[i2] : 0.0;
    const T s1 = (T)fma(-alpha, v1, r1);
    s[i] = s1;
    double w1 = (double)s1;
    if (!wid) w1 *= __ldg(a.w + i);
    acc[0] = fma(w1, w1, acc[0]);
    if (two) {
      const T s2 = (T)fma(-alpha, v2, r2);
      s[i2] = s2;
      double w2 = (double)s2;
      if (!wid) w2 *= __ldg(a.w + i2);
      acc[0] = fma(w2, w2, acc[0]);
    }
  }
  block_sum<1, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 1, a.red, tot) && threadIdx.x == 0) {
    const double mus = sqrt(tot[0]) / S->mu0;
    S->mu_s = mus;
    if (mus < S->tol) S->halfexit = 1;
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k2b(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop || S->halfexit) return;
  __shared__ TileStage<T, kStageCap> stage[kWarpsPerBlock];
  __shared__ double blk[2], tot[2];
  double* sm = reinterpret_cast<double*>(stage);  // reduction scratch after the tile loop
  const T* __restrict__ sv = a.s;
  T* __restrict__ tout = a.t;
  double acc[2] = {0.0, 0.0};
  BCG_TILE_LOOP(a) {
    const int i = tile * 32 + lane_id();
    const T t = csr_tile_row<T, T, kStageCap>(a.rowptr, a.colidx, a.val, a.s, a.n, a.nnz, tile * 32,
                                                stage[warp_id()], a.err);
    if (i < a.n) {
      tout[i] = t;
      acc[0] = fma((double)t, (double)sv[i], acc[0]);
      acc[1] = fma((double)t, (double)t, acc[1]);
    }
  }
  block_sum<2, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    if (*(volatile int*)a.err) {
      S->stop = 1;
    } else if (!(tot[1] > 0.0)) {
      S->conv = GSK_BREAKDOWN;
      S->stop = 1;
    } else {
      S->omega = tot[0] / tot[1];
    }
  }
}

template <typename T>
__device__ __forceinline__ void bcg_k3_row(const BcgArgs<T>& a, int i, double alpha, double omega, bool wid,
                                           double (&acc)[3]) {
  const double s = (double)a.s[i];
  const double x = fma(alpha, (double)a.p[i], (double)a.x[i]);
  a.x[i] = (T)fma(omega, s, x);
  const T r = (T)fma(-omega, (double)a.t[i], s);
  a.r[i] = r;
  const double rd = (double)r;
  acc[0] = fma((double)a.rh[i], rd, acc[0]);
  if (wid) {
    acc[1] = fma(rd, rd, acc[1]);
  } else {
    const double wr = __ldg(a.w + i) * rd;
    acc[1] = fma(wr, wr, acc[1]);
    acc[2] = fma(rd, rd, acc[2]);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k3(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a, a.h_if, 1u);
    return;
  }
  const double alpha = S->alpha;
  if (S->halfexit) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < a.n; i += gridDim.x * kBlock)
      a.x[i] = (T)fma(alpha, (double)a.p[i], (double)a.x[i]);
    if (grid_last(a.cnt) && threadIdx.x == 0) {
      S->iters += 1;
      S->mu_rec = S->mu_s;
      S->check = 1;
      set_cond(a, a.h_if, 1u);
    }
    return;
  }
  __shared__ double sm[3 * kBlock], blk[3], tot[3];
  const double omega = S->omega;
  const bool wid = S->w_identity;
  double acc[3] = {0.0, 0.0, 0.0};
  BCG_ROW2_LOOP(a) {
    bcg_k3_row(a, i, alpha, omega, wid, acc);
    if (i + stride_ < a.n) bcg_k3_row(a, i + stride_, alpha, omega, wid, acc);
  }
  block_sum<3, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 3, a.red, tot) && threadIdx.x == 0) {
    S->iters += 1;
    const double mur = sqrt(tot[1]) / S->mu0;
    S->mu_rec = mur;
    int check = 0, stop = 0;
    if (mur < S->tol) {
      check = 1;
    } else if (omega == 0.0) {
      S->conv = GSK_BREAKDOWN;
      stop = 1;
    } else {
      const double rho1 = tot[0], rn = sqrt(wid ? tot[1] : tot[2]);
      if (!(fabs(rho1) > S->brk * S->rhn * rn)) {
        S->conv = GSK_BREAKDOWN;
        stop = 1;
      } else {
        S->beta = (rho1 / S->rho) * (alpha / omega);
        S->rho = rho1;
      }
    }
    if (!check && !stop && S->iters >= S->maxit) {
      S->conv = GSK_MAXIT;
      stop = 1;
    }
    S->check = check;
    S->stop = stop;
    set_cond(a, a.h_if, (unsigned)(check | stop));
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k4(BcgArgs<T> a) {
  const BcgState* S = a.S;
  if (S->check || S->stop) return;  // the graph's IF node already excludes this
  const double beta = S->beta, omega = S->omega;
  const T* __restrict__ r = a.r;
  const T* __restrict__ v = a.v;
  T* __restrict__ p = a.p;
  BCG_ROW2_LOOP(a) {
    const int i2 = i + stride_;
    const bool two = i2 < a.n;
    const double p1 = (double)p[i], v1 = (double)v[i], r1 = (double)r[i];
    const double p2 = two ? (double)p[i2] : 0.0, v2 = two ? (double)v[i2] : 0.0, r2 = two ? (double)r[i2] : 0.0;
    p[i] = (T)fma(beta, fma(-omega, v1, p1), r1);
    if (two) p[i2] = (T)fma(beta, fma(-omega, v2, p2), r2);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a, a.h_while, 1u);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_kt(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (!(S->check || S->stop)) return;  // the graph's IF node already excludes this
  __shared__ TileStage<T, kStageCap> stage[kWarpsPerBlock];
  __shared__ double blk[2], tot[2];
  double* sm = reinterpret_cast<double*>(stage);  // reduction scratch after the tile loop
  const bool wid = S->w_identity;
  double acc[2] = {0.0, 0.0};
  BCG_TILE_LOOP(a) {
    const int i = tile * 32 + lane_id();
    const T ax = csr_tile_row<T, T, kStageCap>(a.rowptr, a.colidx, a.val, a.x, a.n, a.nnz, tile * 32,
                                                 stage[warp_id()], a.err);
    if (i < a.n) {
      const T t = a.b[i] - ax;
      a.t[i] = t;
      const double wt = wgt(a.w, wid, i) * (double)t;
      acc[0] = fma(wt, wt, acc[0]);
      acc[1] = fma((double)t, (double)t, acc[1]);
    }
  }
  block_sum<2, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    S->mu_true = sqrt(tot[0]) / S->mu0;
    S->tt_true = tot[1];
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_kr(BcgArgs<T> a) {
  BcgState* S = a.S;
  const int stop = S->stop, check = S->check;
  if (!(check || stop)) return;  // the graph's IF node already excludes this
  const bool met = S->mu_true < S->tol;
  const bool refresh = !stop && check && !met && S->refresh_left > 0 && *(volatile int*)a.err == 0;
  if (refresh) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < a.n; i += gridDim.x * kBlock) {
      const T t = a.t[i];
      a.r[i] = t;
      a.rh[i] = t;
      a.p[i] = t;
    }
  }
  if (grid_last(a.cnt) && threadIdx.x == 0) {
    int active = 0;
    if (!stop && check) {
      if (met) {
        S->conv = GSK_CONVERGED;
      } else if (refresh) {
        S->refresh_left -= 1;
        S->refreshes += 1;
        S->rho = S->tt_true;
        S->rhn = sqrt(S->tt_true);
        S->check = 0;
        S->halfexit = 0;
        if (S->iters >= S->maxit) {
          S->conv = GSK_MAXIT;
        } else {
          active = 1;
        }
      } else {
        S->conv = GSK_STAGNATED;
      }
    }
    S->stop = !active;
    S->active = active;
    set_cond(a, a.h_while, (unsigned)active);
  }
}

// ------------------------------------------------------------------ host

struct BcgPlan {
  int g_tile, g_vec, wmode;
  BcgArgs<double> a;
  double* wbuf;  // weights computed by the solver (or nullptr)
  BcgState host_state;
};

static void bcg_launch(gsk_ctx* ctx, BcgPlan& P, int k, cudaStream_t s) {
  BcgArgs<double>& a = P.a;
  switch (k) {
    case kKWeights: launch_gs_norm(ctx, a.n, a.nnz, a.rowptr, a.val, 2.0, P.wbuf, a.err, s); break;
    case kKUnitCheck: launch_unit_check(ctx, a.n, P.wbuf, a.red, &a.S->w_identity, s); break;
    case kKBcgInit: bcg_init<double><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKBcgK1: bcg_k1<double><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKBcgK2a: bcg_k2a<double><<<P.g_vec, kBlock, 0, s>>>(a); break;
    case kKBcgK2b: bcg_k2b<double><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKBcgK3: bcg_k3<double><<<P.g_vec, kBlock, 0, s>>>(a); break;
    case kKBcgK4: bcg_k4<double><<<P.g_vec, kBlock, 0, s>>>(a); break;
    case kKBcgKt: bcg_kt<double><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKBcgKr: bcg_kr<double><<<P.g_vec, kBlock, 0, s>>>(a); break;
  }
}

static gsk_status bcg_record(gsk_ctx* ctx, BcgPlan& P, cudaGraphExec_t* exec_out) {
  cudaStream_t cs = ctx->capture;
  cudaGraph_t top = nullptr;
  GSK_CK(cudaGraphCreate(&top, 0));
  struct Guard {
    cudaGraph_t g;
    ~Guard() { if (g) cudaGraphDestroy(g); }
  } guard{top};
  BcgArgs<double>& a = P.a;
  a.in_graph = 1;
  GSK_CK(cudaGraphConditionalHandleCreate(&a.h_while, top, 1u, cudaGraphCondAssignDefault));

  Capture c0;
  GSK_CK(c0.begin(cs, top));
  if (P.wmode == 0) {  // GS(2) metric: w = 1/||a_i||_2, then test for the identity
    bcg_launch(ctx, P, kKWeights, cs);
    bcg_launch(ctx, P, kKUnitCheck, cs);
  }
  bcg_launch(ctx, P, kKBcgInit, cs);
  GSK_CK(c0.end());

  cudaGraphNode_t wnode;
  cudaGraph_t wbody;
  GSK_CK(add_conditional(top, c0.tail, a.h_while, cudaGraphCondTypeWhile, 1, &wnode, &wbody));
  GSK_CK(cudaGraphConditionalHandleCreate(&a.h_if, wbody, 0u, 0));

  Capture c1;
  GSK_CK(c1.begin(cs, wbody));
  for (int k : {kKBcgK1, kKBcgK2a, kKBcgK2b, kKBcgK3}) bcg_launch(ctx, P, k, cs);
  GSK_CK(c1.end());

  cudaGraphNode_t inode;
  cudaGraph_t ib[2];
  GSK_CK(add_conditional(wbody, c1.tail, a.h_if, cudaGraphCondTypeIf, 2, &inode, ib));
  Capture c2;
  GSK_CK(c2.begin(cs, ib[0]));
  bcg_launch(ctx, P, kKBcgKt, cs);
  bcg_launch(ctx, P, kKBcgKr, cs);
  GSK_CK(c2.end());
  Capture c3;
  GSK_CK(c3.begin(cs, ib[1]));
  bcg_launch(ctx, P, kKBcgK4, cs);
  GSK_CK(c3.end());

  GSK_CK(cudaGraphInstantiate(exec_out, top, 0));
  return GSK_OK;
}

// Validates the call, lays out the workspace and fills P.
static gsk_status bcg_prepare(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, double tol,
                              const gsk_opts& opts, BcgPlan& P) {
  if (A->dtype != GSK_F64) return ctx->fail(GSK_ERR_ARG, "the FP64 solver needs an FP64 matrix");
  if (!(tol >= 0.0) || opts.maxit < 0 || opts.refresh < 0) return ctx->fail(GSK_ERR_ARG, "bad tol/maxit/refresh");
  if (A->n > 0 && (!b || !x)) return ctx->fail(GSK_ERR_ARG, "NULL b or x");
  const int n = A->n;
  P.wmode = opts.weights ? 2 : (opts.metric == GSK_METRIC_PLAIN ? 1 : 0);
  P.g_tile = ctx->grid_for((n + 31) / 32, kWarpsPerBlock, 8);
  // vector kernels: 4 blocks per SM, so that each thread sums many rows
  // before the (FP64) block reduction
  P.g_vec = ctx->grid_for((n + 1) / 2, kBlock, 4);
  const int g_all = ctx->grid_for(n, kBlock, 8);
  const int gmax = g_all > P.g_tile ? g_all : P.g_tile;
  auto layout = [&](Arena& ar) {
    P.a.err = ar.take<int>(64);
    P.a.cnt = ar.take<unsigned>(64);
    P.a.red = take_red(ar, gmax, 4);
    P.a.S = ar.take<BcgState>(1);
    P.a.r = ar.take<double>(n);
    P.a.rh = ar.take<double>(n);
    P.a.p = ar.take<double>(n);
    P.a.v = ar.take<double>(n);
    P.a.s = ar.take<double>(n);
    P.a.t = ar.take<double>(n);
    P.wbuf = P.wmode == 0 ? ar.take<double>(n) : nullptr;
  };
  Arena sizing;
  layout(sizing);
  gsk_status s = ctx->reserve(sizing.off);
  if (s != GSK_OK) return s;
  Arena ar{(char*)ctx->ws, ctx->ws_bytes, 0};
  layout(ar);
  P.a.n = n;
  P.a.nnz = A->nnz;
  P.a.rowptr = A->rowptr;
  P.a.colidx = A->colidx;
  P.a.val = (const double*)A->val;
  P.a.b = (const double*)b;
  P.a.x = (double*)x;
  P.a.w = P.wmode == 0 ? P.wbuf : (P.wmode == 2 ? opts.weights : nullptr);
  P.a.in_graph = 0;
  P.a.h_while = P.a.h_if = 0;
  BcgState& hs = P.host_state;
  std::memset(&hs, 0, sizeof(hs));
  hs.tol = tol;
  hs.brk = 1e-16 * DBL_EPSILON;
  hs.maxit = opts.maxit;
  hs.refresh_left = opts.refresh;
  hs.w_identity = P.wmode == 1 ? 1 : 0;
  return GSK_OK;
}

// Clears the counters/flags region and uploads the initial state.
static gsk_status bcg_upload(gsk_ctx* ctx, BcgPlan& P, cudaStream_t st) {
  const char* end = (const char*)(P.a.red.counters + (P.a.red.maxgrid + kGroup - 1) / kGroup + 1);
  GSK_CK(cudaMemsetAsync(ctx->ws, 0, end - (const char*)ctx->ws, st));
  GSK_CK(cudaMemcpyAsync(P.a.S, &P.host_state, sizeof(BcgState), cudaMemcpyHostToDevice, st));
  return GSK_OK;
}

static gsk_status bcg_readback(gsk_ctx* ctx, BcgPlan& P, cudaStream_t st, BcgState& out, int& bits) {
  char* hp = (char*)ctx->host_pinned;
  GSK_CK(cudaMemcpyAsync(hp, P.a.S, sizeof(BcgState), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaMemcpyAsync(hp + 512, P.a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  std::memcpy(&out, hp, sizeof(out));
  std::memcpy(&bits, hp + 512, sizeof(int));
  return GSK_OK;
}

gsk_status bcg_profile(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, double tol, const gsk_opts& opts,
                       int max_iters, LaunchTimer& T, gsk_info* info) {
  BcgPlan P;
  gsk_status s = bcg_prepare(ctx, A, b, x, tol, opts, P);
  if (s != GSK_OK) return s;
  if (A->n == 0) return GSK_OK;
  if ((s = bcg_upload(ctx, P, T.st)) != GSK_OK) return s;
  auto timed = [&](int k, int step) -> gsk_status {
    return T.time(k, step, [&](cudaStream_t st) { bcg_launch(ctx, P, k, st); });
  };
  if (P.wmode == 0) {
    if ((s = timed(kKWeights, -1)) != GSK_OK) return s;
    if ((s = timed(kKUnitCheck, -1)) != GSK_OK) return s;
  }
  if ((s = timed(kKBcgInit, -1)) != GSK_OK) return s;
  BcgState st;
  int bits = 0;
  if ((s = bcg_readback(ctx, P, T.st, st, bits)) != GSK_OK) return s;
  for (int it = 0; it < max_iters && st.active && !bits; ++it) {
    for (int k : {kKBcgK1, kKBcgK2a, kKBcgK2b, kKBcgK3})
      if ((s = timed(k, it)) != GSK_OK) return s;
    if ((s = bcg_readback(ctx, P, T.st, st, bits)) != GSK_OK) return s;
    if (st.check || st.stop) {
      if ((s = timed(kKBcgKt, it)) != GSK_OK) return s;
      if ((s = timed(kKBcgKr, it)) != GSK_OK) return s;
    } else {
      if ((s = timed(kKBcgK4, it)) != GSK_OK) return s;
    }
    if ((s = bcg_readback(ctx, P, T.st, st, bits)) != GSK_OK) return s;
  }
  if (info) *info = gsk_info{st.iters, 0, st.refreshes, 0, st.conv, st.mu_true, st.mu_rec, 0.f};
  return err_bits_status(ctx, bits);
}

}  // namespace gsk

using namespace gsk;

extern "C" gsk_status bicgstab_solve(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, double tol,
                                     const gsk_opts* opts_in, gsk_info* info, void* stream) {
  if (!ctx) return GSK_ERR_ARG;
  gsk_status s = check_csr(ctx, A);
  if (s != GSK_OK) return s;
  gsk_opts opts;
  if (opts_in) opts = *opts_in;
  else gsk_opts_default(&opts);
  if (opts.precision == GSK_PREC_MIXED) return bicgstab_solve_mixed(ctx, A, b, x, tol, &opts, info, stream);
  cudaStream_t st = (cudaStream_t)stream;
  BcgPlan P;
  if ((s = bcg_prepare(ctx, A, b, x, tol, opts, P)) != GSK_OK) return s;
  if (A->n == 0) {
    if (info) *info = gsk_info{0, 0, 0, 0, GSK_CONVERGED, 0.0, 0.0, 0.f};
    return GSK_OK;
  }
  std::vector<uint64_t> key = {1, (uint64_t)A->n, (uint64_t)A->nnz, (uint64_t)A->rowptr, (uint64_t)A->colidx,
                               (uint64_t)A->val, (uint64_t)b, (uint64_t)x, (uint64_t)P.wmode,
                               (uint64_t)P.a.w, (uint64_t)ctx->ws};
  GraphEntry* ge = ctx->find_graph(key);
  if (!ge) {
    cudaGraphExec_t ex = nullptr;
    if ((s = bcg_record(ctx, P, &ex)) != GSK_OK) return s;
    ge = ctx->add_graph(key, ex);
  }
  GSK_CK(cudaEventRecord(ctx->ev0, st));
  if ((s = bcg_upload(ctx, P, st)) != GSK_OK) return s;
  GSK_CK(cudaGraphLaunch(ge->exec, st));
  GSK_CK(cudaEventRecord(ctx->ev1, st));
  if (!info) return GSK_OK;
  BcgState out;
  int bits = 0;
  if ((s = bcg_readback(ctx, P, st, out, bits)) != GSK_OK) return s;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  *info = gsk_info{out.iters, 0, out.refreshes, 0, out.conv, out.mu_true, out.mu_rec, ms};
  return err_bits_status(ctx, bits);
}
