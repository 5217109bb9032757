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
//               kr  finish, or refresh r = rh = p = t      (Sec. 2.2 / 4)
// The chain is recorded once into a CUDA graph: a WHILE node repeats the
// iteration and an IF/ELSE node picks k4 or kt+kr, both driven by values the
// kernels set on the device, so a solve is one graph launch.
//
// The breakdown tolerance is 1e-16 * DBL_EPSILON relative to the vector
// norms (Sec. 2.2).  The stopping metric is ||W(b - Ax)|| / ||W(b - Ax0)||
// with W the GS(2) scales of A (Sec. 2.2); when W is the identity to within
// 4 ulp (an already GS(2)-scaled system) the weight loads are skipped.
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
};

#define BCG_TILE_LOOP(a) \
  for (int tile = blockIdx.x * kWarpsPerBlock + warp_id(), ntiles_ = ((a).n + 31) / 32; tile < ntiles_; \
       tile += gridDim.x * kWarpsPerBlock)
#define BCG_ROW_LOOP(a) for (int i = blockIdx.x * kBlock + threadIdx.x; i < (a).n; i += gridDim.x * kBlock)

__device__ __forceinline__ double wgt(const double* w, bool wid, int i) { return wid ? 1.0 : __ldg(w + i); }

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_init(BcgArgs<T> a) {
  __shared__ TileStage<T, kStageCap> stage[kWarpsPerBlock];
  __shared__ double sm[4 * kWarpsPerBlock], blk[2], tot[2];
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
    S->stop = 0;
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
    cudaGraphSetConditional(a.h_while, active);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k1(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop) return;
  __shared__ TileStage<T, kStageCap> stage[kWarpsPerBlock];
  __shared__ double sm[4 * kWarpsPerBlock], blk[2], tot[2];
  double acc[2] = {0.0, 0.0};
  BCG_TILE_LOOP(a) {
    const int i = tile * 32 + lane_id();
    const T v = csr_tile_row<T, T, kStageCap>(a.rowptr, a.colidx, a.val, a.p, a.n, a.nnz, tile * 32,
                                                stage[warp_id()], a.err);
    if (i < a.n) {
      a.v[i] = v;
      acc[0] = fma((double)a.rh[i], (double)v, acc[0]);
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
  __shared__ double sm[4 * kWarpsPerBlock], blk[1], tot[1];
  const double alpha = S->alpha;
  const bool wid = S->w_identity;
  double acc[1] = {0.0};
  BCG_ROW_LOOP(a) {
    const T s = (T)fma(-alpha, (double)a.v[i], (double)a.r[i]);
    a.s[i] = s;
    const double ws = wgt(a.w, wid, i) * (double)s;
    acc[0] = fma(ws, ws, acc[0]);
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
  __shared__ double sm[4 * kWarpsPerBlock], blk[2], tot[2];
  double acc[2] = {0.0, 0.0};
  BCG_TILE_LOOP(a) {
    const int i = tile * 32 + lane_id();
    const T t = csr_tile_row<T, T, kStageCap>(a.rowptr, a.colidx, a.val, a.s, a.n, a.nnz, tile * 32,
                                                stage[warp_id()], a.err);
    if (i < a.n) {
      a.t[i] = t;
      acc[0] = fma((double)t, (double)a.s[i], acc[0]);
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
__global__ void __launch_bounds__(kBlock) bcg_k3(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.h_if, 1u);
    return;
  }
  const double alpha = S->alpha;
  if (S->halfexit) {
    BCG_ROW_LOOP(a) a.x[i] = (T)fma(alpha, (double)a.p[i], (double)a.x[i]);
    if (grid_last(a.cnt) && threadIdx.x == 0) {
      S->iters += 1;
      S->mu_rec = S->mu_s;
      S->check = 1;
      cudaGraphSetConditional(a.h_if, 1u);
    }
    return;
  }
  __shared__ double sm[4 * kWarpsPerBlock], blk[3], tot[3];
  const double omega = S->omega;
  const bool wid = S->w_identity;
  double acc[3] = {0.0, 0.0, 0.0};
  BCG_ROW_LOOP(a) {
    const double s = (double)a.s[i];
    a.x[i] = (T)((double)a.x[i] + fma(alpha, (double)a.p[i], omega * s));
    const T r = (T)fma(-omega, (double)a.t[i], s);
    a.r[i] = r;
    const double rd = (double)r, wr = wgt(a.w, wid, i) * rd;
    acc[0] = fma((double)a.rh[i], rd, acc[0]);
    acc[1] = fma(wr, wr, acc[1]);
    acc[2] = fma(rd, rd, acc[2]);
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
      const double rho1 = tot[0], rn = sqrt(tot[2]);
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
    cudaGraphSetConditional(a.h_if, (unsigned)(check | stop));
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k4(BcgArgs<T> a) {
  const BcgState* S = a.S;
  const double beta = S->beta, omega = S->omega;
  BCG_ROW_LOOP(a) {
    const double pv = fma(-omega, (double)a.v[i], (double)a.p[i]);
    a.p[i] = (T)fma(beta, pv, (double)a.r[i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.h_while, 1u);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_kt(BcgArgs<T> a) {
  __shared__ TileStage<T, kStageCap> stage[kWarpsPerBlock];
  __shared__ double sm[4 * kWarpsPerBlock], blk[2], tot[2];
  BcgState* S = a.S;
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
  const bool met = S->mu_true < S->tol;
  const bool refresh = !stop && check && !met && S->refresh_left > 0 && *(volatile int*)a.err == 0;
  if (refresh) {
    BCG_ROW_LOOP(a) {
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
    cudaGraphSetConditional(a.h_while, (unsigned)active);
  }
}

// ------------------------------------------------------------------ host

struct BcgPlan {
  int g_tile, g_vec;
  BcgArgs<double> a;
  double* wbuf;  // weights computed by the solver (or nullptr)
  int* wid_out;
};

static gsk_status bcg_record(gsk_ctx* ctx, BcgPlan& P, int wmode, cudaGraphExec_t* exec_out) {
  cudaStream_t cs = ctx->capture;
  cudaGraph_t top = nullptr;
  GSK_CK(cudaGraphCreate(&top, 0));
  struct Guard {
    cudaGraph_t g;
    ~Guard() { if (g) cudaGraphDestroy(g); }
  } guard{top};
  BcgArgs<double>& a = P.a;
  GSK_CK(cudaGraphConditionalHandleCreate(&a.h_while, top, 1u, cudaGraphCondAssignDefault));

  Capture c0;
  GSK_CK(c0.begin(cs, top));
  if (wmode == 0) {  // GS(2) metric: w = 1/||a_i||_2, then test for the identity
    launch_gs_norm(ctx, a.n, a.nnz, a.rowptr, a.val, 2.0, P.wbuf, a.err, cs);
    launch_unit_check(ctx, a.n, P.wbuf, a.red, P.wid_out, cs);
  }
  bcg_init<double><<<P.g_tile, kBlock, 0, cs>>>(a);
  GSK_CK(c0.end());

  cudaGraphNode_t wnode;
  cudaGraph_t wbody;
  GSK_CK(add_conditional(top, c0.tail, a.h_while, cudaGraphCondTypeWhile, 1, &wnode, &wbody));
  GSK_CK(cudaGraphConditionalHandleCreate(&a.h_if, wbody, 0u, 0));

  Capture c1;
  GSK_CK(c1.begin(cs, wbody));
  bcg_k1<double><<<P.g_tile, kBlock, 0, cs>>>(a);
  bcg_k2a<double><<<P.g_vec, kBlock, 0, cs>>>(a);
  bcg_k2b<double><<<P.g_tile, kBlock, 0, cs>>>(a);
  bcg_k3<double><<<P.g_vec, kBlock, 0, cs>>>(a);
  GSK_CK(c1.end());

  cudaGraphNode_t inode;
  cudaGraph_t ib[2];
  GSK_CK(add_conditional(wbody, c1.tail, a.h_if, cudaGraphCondTypeIf, 2, &inode, ib));
  Capture c2;
  GSK_CK(c2.begin(cs, ib[0]));
  bcg_kt<double><<<P.g_tile, kBlock, 0, cs>>>(a);
  bcg_kr<double><<<P.g_vec, kBlock, 0, cs>>>(a);
  GSK_CK(c2.end());
  Capture c3;
  GSK_CK(c3.begin(cs, ib[1]));
  bcg_k4<double><<<P.g_vec, kBlock, 0, cs>>>(a);
  GSK_CK(c3.end());

  GSK_CK(cudaGraphInstantiate(exec_out, top, 0));
  return GSK_OK;
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
  if (A->dtype != GSK_F64) return ctx->fail(GSK_ERR_ARG, "the FP64 solver needs an FP64 matrix");
  if (!(tol >= 0.0) || opts.maxit < 0 || opts.refresh < 0) return ctx->fail(GSK_ERR_ARG, "bad tol/maxit/refresh");
  if (A->n > 0 && (!b || !x)) return ctx->fail(GSK_ERR_ARG, "NULL b or x");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = A->n;
  if (n == 0) {
    if (info) *info = gsk_info{0, 0, 0, 0, GSK_CONVERGED, 0.0, 0.0, 0.f};
    return GSK_OK;
  }
  const int wmode = opts.weights ? 2 : (opts.metric == GSK_METRIC_PLAIN ? 1 : 0);

  BcgPlan P;
  P.g_tile = ctx->grid_for((n + 31) / 32, kWarpsPerBlock, 8);
  P.g_vec = ctx->grid_for(n, kBlock, 8);
  const int gmax = P.g_tile > P.g_vec ? P.g_tile : P.g_vec;
  // workspace layout (first pass sizes it, second pass assigns pointers)
  auto layout = [&](Arena& ar) {
    P.a.err = ar.take<int>(64);
    P.a.S = ar.take<BcgState>(1);
    P.a.cnt = ar.take<unsigned>(64);
    P.wid_out = ar.take<int>(64);
    P.a.red = take_red(ar, gmax, 4);
    P.a.r = ar.take<double>(n);
    P.a.rh = ar.take<double>(n);
    P.a.p = ar.take<double>(n);
    P.a.v = ar.take<double>(n);
    P.a.s = ar.take<double>(n);
    P.a.t = ar.take<double>(n);
    P.wbuf = wmode == 0 ? ar.take<double>(n) : nullptr;
  };
  Arena sizing;
  layout(sizing);
  if ((s = ctx->reserve(sizing.off)) != GSK_OK) return s;
  Arena ar{(char*)ctx->ws, ctx->ws_bytes, 0};
  layout(ar);
  P.a.n = n;
  P.a.nnz = A->nnz;
  P.a.rowptr = A->rowptr;
  P.a.colidx = A->colidx;
  P.a.val = (const double*)A->val;
  P.a.b = (const double*)b;
  P.a.x = (double*)x;
  P.a.w = wmode == 0 ? P.wbuf : (wmode == 2 ? opts.weights : nullptr);
  if (wmode == 0) P.wid_out = &P.a.S->w_identity;

  std::vector<uint64_t> key = {1, (uint64_t)n, (uint64_t)A->nnz, (uint64_t)A->rowptr, (uint64_t)A->colidx,
                               (uint64_t)A->val, (uint64_t)b, (uint64_t)x, (uint64_t)wmode,
                               (uint64_t)P.a.w, (uint64_t)ctx->ws};
  GraphEntry* ge = ctx->find_graph(key);
  if (!ge) {
    cudaGraphExec_t ex = nullptr;
    if ((s = bcg_record(ctx, P, wmode, &ex)) != GSK_OK) return s;
    ge = ctx->add_graph(key, ex);
  }

  BcgState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.tol = tol;
  hs.brk = 1e-16 * DBL_EPSILON;
  hs.maxit = opts.maxit;
  hs.refresh_left = opts.refresh;
  hs.w_identity = wmode == 1 ? 1 : 0;
  GSK_CK(cudaEventRecord(ctx->ev0, st));
  // error word, counters and reduction scratch sit at the start of the
  // workspace; other solves lay the workspace out differently, so clear them
  GSK_CK(cudaMemsetAsync(ctx->ws, 0, (char*)(P.a.red.counters + (P.a.red.maxgrid + kGroup - 1) / kGroup + 1) -
                                         (char*)ctx->ws, st));
  GSK_CK(cudaMemcpyAsync(P.a.S, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  GSK_CK(cudaGraphLaunch(ge->exec, st));
  GSK_CK(cudaEventRecord(ctx->ev1, st));
  if (!info) return GSK_OK;
  char* hp = (char*)ctx->host_pinned;
  GSK_CK(cudaMemcpyAsync(hp, P.a.S, sizeof(BcgState), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaMemcpyAsync(hp + 512, P.a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  BcgState out;
  std::memcpy(&out, hp, sizeof(out));
  int bits;
  std::memcpy(&bits, hp + 512, sizeof(int));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  *info = gsk_info{out.iters, 0, out.refreshes, 0, out.conv, out.mu_true, out.mu_rec, ms};
  return err_bits_status(ctx, bits);
}
