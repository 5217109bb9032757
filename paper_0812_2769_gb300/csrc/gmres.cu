// Restarted GMRES(m) with classical Gram-Schmidt applied twice (Sec. 2),
// with the Arnoldi process, the Givens rotations, the Hessenberg
// least-squares solve and every stopping decision on the device.
//
// Basis storage: V is column-major (leading dimension ldv) and column k holds
// an unnormalised vector; the Arnoldi vector is v_k = sig[k] * V[:, k].  The
// scale is folded into the next product instead of a separate normalisation
// pass over V.
//
// One Arnoldi step j (k = j + 1 basis vectors) is four kernels:
//   ga  w = A v_j -> V[:, j+1];  ||w||                           (SpMV)
//   gd  h1 = V_k^T w                                             (CGS pass 1, multi-dot)
//   gb  w -= V_k h1;             h2 = V_k^T w                    (CGS pass 2)
//   gc  w -= V_k h2;             ||w||  -> column j of H = h1 + h2,
//       h_{j+1,j} = ||w||, earlier rotations applied, new rotation, g update,
//       convergence / breakdown tests                           (device scalar work)
// A cycle ends in
//   gy  back substitution H y = g (one block)
//   gx  x += V_k y
//   gr  r = b - A x -> V[:, 0]; true metric; restart or stop
// The steps form an inner WHILE node and the cycles an outer WHILE node of a
// CUDA graph, so a whole solve is one graph launch.
//
// Stopping (Sec. 2.2): a cycle ends when |g_{j+1}| < tau * ||r0|| (the
// least-squares residual relative to the initial residual), at numerical
// breakdown h_{j+1,j} <= 1e-14 ||A v_j||, after m steps, or at maxit.  The
// true metric ||W(b - Ax)|| / ||W(b - Ax0)|| (W = GS(2) scales of A) decides
// convergence; if the estimate met tau but the metric did not, tau is
// tightened by tol / metric before the restart.
#include <cfloat>

#include "graph.hpp"
#include "internal.hpp"

namespace gsk {

struct GmState {
  double rho0, mu0, tau, tol, est, mu_true, aw_norm;
  int m, maxit, iters, restarts, conv, j, kcols, stop, est_hit, w_identity, cont;
};

template <typename T>
struct GmArgs {
  int n, nnz, m;
  long long ldv;
  const int* rowptr;
  const int* colidx;
  const T* val;
  const T* b;
  T* x;
  T* V;
  double *H, *g, *cs, *sn, *y, *h1, *h2, *sig;
  const double* w;
  GmState* S;
  GridRed red;
  unsigned* cnt;
  int* err;
  cudaGraphConditionalHandle h_outer, h_inner;
  int in_graph;
};

template <typename T>
__device__ __forceinline__ void gm_set_cond(const GmArgs<T>& a, cudaGraphConditionalHandle h, unsigned v) {
  if (a.in_graph) cudaGraphSetConditional(h, v);
}

#define GM_TILE_LOOP(a) \
  for (int tile = blockIdx.x * kWarpsPerBlock + warp_id(), ntiles_ = ((a).n + 31) / 32; tile < ntiles_; \
       tile += gridDim.x * kWarpsPerBlock)
#define GM_ROW_LOOP(a) for (int i = blockIdx.x * kBlock + threadIdx.x; i < (a).n; i += gridDim.x * kBlock)

__device__ __forceinline__ double gm_wgt(const double* w, bool wid, int i) { return wid ? 1.0 : __ldg(w + i); }

// Block sum of NV register accumulators (only the first nv are needed), in
// chunks of 16 rows of a [16][kBlock] shared table.
template <int NV>
__device__ __forceinline__ void block_sum_chunked(const double (&v)[NV], int nv, double* table, double* res) {
#pragma unroll
  for (int c0 = 0; c0 < NV; c0 += 16) {
    if (c0 < nv) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (c0 + q < NV) table[q * kBlock + threadIdx.x] = v[c0 + q];
      block_sum_table<kBlock>(table, min(16, nv - c0), res + c0);
    }
  }
}

template <typename T>
union GmSmem {
  TileStage<T, kStageCap> stage[kWarpsPerBlock];
  double table[16 * kBlock];
};

// r = b - A x into V[:, 0]; the true metric; start (init) or restart a cycle.
template <typename T, bool INIT>
__global__ void __launch_bounds__(kBlock) gm_residual(GmArgs<T> a) {
  __shared__ GmSmem<T> sm;
  __shared__ double blk[2], tot[2];
  GmState* S = a.S;
  const bool wid = S->w_identity;
  double acc[2] = {0.0, 0.0};
  GM_TILE_LOOP(a) {
    const int i = tile * 32 + lane_id();
    const T ax = csr_tile_row<T, T, kStageCap>(a.rowptr, a.colidx, a.val, a.x, a.n, a.nnz, tile * 32,
                                                 sm.stage[warp_id()], a.err);
    if (i < a.n) {
      const T r = a.b[i] - ax;
      a.V[i] = r;
      const double wr = gm_wgt(a.w, wid, i) * (double)r;
      acc[0] = fma(wr, wr, acc[0]);
      acc[1] = fma((double)r, (double)r, acc[1]);
    }
  }
  block_sum_chunked<2>(acc, 2, sm.table, blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    const int e = *(volatile int*)a.err;
    const double rn = sqrt(tot[1]);
    int stop = 0;
    if (INIT) {
      const double mu0 = sqrt(tot[0]);
      S->mu0 = mu0;
      S->rho0 = rn;
      S->iters = 0;
      S->restarts = 0;
      S->tau = S->tol;
      S->conv = GSK_MAXIT;
      S->mu_true = 1.0;
      S->est = 1.0;
      if (e) {
        stop = 1;
      } else if (!isfinite(mu0)) {
        atomicOr(a.err, kErrNonFinite);
        stop = 1;
      } else if (mu0 == 0.0) {
        S->conv = GSK_CONVERGED;
        S->mu_true = 0.0;
        S->est = 0.0;
        stop = 1;
      } else if (S->maxit <= 0) {
        stop = 1;
      }
    } else {
      const double mu = sqrt(tot[0]) / S->mu0;
      S->mu_true = mu;
      if (e) {
        stop = 1;
      } else if (mu < S->tol) {
        S->conv = GSK_CONVERGED;
        stop = 1;
      } else if (S->iters >= S->maxit || S->kcols == 0) {
        S->conv = GSK_MAXIT;
        stop = 1;
      } else {
        if (S->est_hit) S->tau = S->tau * (S->tol / mu);
        S->restarts += 1;
      }
    }
    if (!stop) {
      a.sig[0] = 1.0 / rn;
      a.g[0] = rn;
      for (int q = 1; q <= a.m; ++q) a.g[q] = 0.0;
      S->j = 0;
      S->est_hit = 0;
      S->kcols = 0;
    }
    S->stop = stop;
    S->cont = !stop;
    gm_set_cond(a, a.h_outer, (unsigned)!stop);
    gm_set_cond(a, a.h_inner, (unsigned)!stop);
  }
}

// Arnoldi step, product: w = A v_j stored in V[:, j+1]; ||w||^2 (the
// reference for the breakdown test).
template <typename T>
__global__ void __launch_bounds__(kBlock) gm_ga(GmArgs<T> a) {
  __shared__ GmSmem<T> sm;
  __shared__ double res[1], tot[1];
  const GmState* S = a.S;
  const int j = S->j;
  const T* vj = a.V + (long long)j * a.ldv;
  T* __restrict__ wout = a.V + (long long)(j + 1) * a.ldv;
  const double sj = a.sig[j];
  double ww[1] = {0.0};
  GM_TILE_LOOP(a) {
    const int i = tile * 32 + lane_id();
    const T av = csr_tile_row<T, T, kStageCap>(a.rowptr, a.colidx, a.val, vj, a.n, a.nnz, tile * 32,
                                                 sm.stage[warp_id()], a.err);
    if (i < a.n) {
      const T w = (T)(sj * (double)av);
      wout[i] = w;
      ww[0] = fma((double)w, (double)w, ww[0]);
    }
  }
  block_sum_chunked<1>(ww, 1, sm.table, res);
  if (grid_sum(res, 1, a.red, tot) && threadIdx.x == 0) a.S->aw_norm = sqrt(tot[0]);
}

// CGS pass 1: h1 = sig .* (V_k^T w).
template <typename T, int KP>
__global__ void __launch_bounds__(kBlock) gm_gd(GmArgs<T> a) {
  __shared__ double table[16 * kBlock], res[KP], tot[KP];
  const GmState* S = a.S;
  const int j = S->j, k = j + 1;
  const T* __restrict__ wv = a.V + (long long)(j + 1) * a.ldv;
  double acc[KP];
#pragma unroll
  for (int c = 0; c < KP; ++c) acc[c] = 0.0;
  GM_ROW_LOOP(a) {
    const double w = (double)wv[i];
#pragma unroll
    for (int c0 = 0; c0 < KP; c0 += 4)
      if (c0 < k) {
#pragma unroll
        for (int c = c0; c < c0 + 4; ++c)
          if (c < k) acc[c] = fma((double)a.V[(long long)c * a.ldv + i], w, acc[c]);
      }
  }
  block_sum_chunked<KP>(acc, k, table, res);
  if (grid_sum(res, k, a.red, tot)) {
    for (int c = threadIdx.x; c < k; c += kBlock) a.h1[c] = a.sig[c] * tot[c];
  }
}

// CGS pass 2: w -= V_k (sig .* h1); h2 = sig .* (V_k^T w).
template <typename T, int KP>
__global__ void __launch_bounds__(kBlock) gm_gb(GmArgs<T> a) {
  __shared__ double coef[KP], table[16 * kBlock], res[KP], tot[KP];
  const GmState* S = a.S;
  const int j = S->j, k = j + 1;
  T* wv = a.V + (long long)(j + 1) * a.ldv;
  for (int c = threadIdx.x; c < k; c += kBlock) coef[c] = a.sig[c] * a.h1[c];
  __syncthreads();
  double acc[KP];
#pragma unroll
  for (int c = 0; c < KP; ++c) acc[c] = 0.0;
  GM_ROW_LOOP(a) {
    double w = (double)wv[i];
#pragma unroll
    for (int c0 = 0; c0 < KP; c0 += 4)
      if (c0 < k) {
#pragma unroll
        for (int c = c0; c < c0 + 4; ++c)
          if (c < k) w = fma(-(double)a.V[(long long)c * a.ldv + i], coef[c], w);
      }
    const T wt = (T)w;
    wv[i] = wt;
#pragma unroll
    for (int c0 = 0; c0 < KP; c0 += 4)
      if (c0 < k) {
#pragma unroll
        for (int c = c0; c < c0 + 4; ++c)
          if (c < k) acc[c] = fma((double)a.V[(long long)c * a.ldv + i], (double)wt, acc[c]);
      }
  }
  block_sum_chunked<KP>(acc, k, table, res);
  if (grid_sum(res, k, a.red, tot)) {
    for (int c = threadIdx.x; c < k; c += kBlock) a.h2[c] = a.sig[c] * tot[c];
  }
}

// CGS pass 3: w -= V_k (sig .* h2); ||w||; then the Hessenberg column, the
// Givens rotations and the cycle's stopping tests (one thread).
template <typename T, int KP>
__global__ void __launch_bounds__(kBlock) gm_gc(GmArgs<T> a) {
  __shared__ double coef[KP], table[16 * kBlock], res[1], tot[1];
  GmState* S = a.S;
  const int j = S->j, k = j + 1;
  T* wv = a.V + (long long)(j + 1) * a.ldv;
  for (int c = threadIdx.x; c < k; c += kBlock) coef[c] = a.sig[c] * a.h2[c];
  __syncthreads();
  double acc[1] = {0.0};
  GM_ROW_LOOP(a) {
    double w = (double)wv[i];
#pragma unroll
    for (int c0 = 0; c0 < KP; c0 += 4)
      if (c0 < k) {
#pragma unroll
        for (int c = c0; c < c0 + 4; ++c)
          if (c < k) w = fma(-(double)a.V[(long long)c * a.ldv + i], coef[c], w);
      }
    const T wt = (T)w;
    wv[i] = wt;
    acc[0] = fma((double)wt, (double)wt, acc[0]);
  }
  block_sum_chunked<1>(acc, 1, table, res);
  if (grid_sum(res, 1, a.red, tot) && threadIdx.x == 0) {
    const int ld = a.m + 1;
    double* hcol = a.H + (long long)j * ld;
    for (int c = 0; c <= j; ++c) hcol[c] = a.h1[c] + a.h2[c];
    const double hnext = sqrt(tot[0]);
    S->iters += 1;
    for (int q = 0; q < j; ++q) {
      const double t0 = a.cs[q] * hcol[q] + a.sn[q] * hcol[q + 1];
      const double t1 = -a.sn[q] * hcol[q] + a.cs[q] * hcol[q + 1];
      hcol[q] = t0;
      hcol[q + 1] = t1;
    }
    const double rho = hypot(hcol[j], hnext);
    double c_, s_;
    if (rho == 0.0) {
      c_ = 1.0;
      s_ = 0.0;
    } else {
      c_ = hcol[j] / rho;
      s_ = hnext / rho;
    }
    a.cs[j] = c_;
    a.sn[j] = s_;
    hcol[j] = rho;
    hcol[j + 1] = 0.0;
    const double gj = a.g[j];
    a.g[j + 1] = -s_ * gj;
    a.g[j] = c_ * gj;
    const double est = fabs(a.g[j + 1]) / S->rho0;
    S->est = est;
    S->kcols = k;
    int cont = 1;
    if (est < S->tau) {
      S->est_hit = 1;
      cont = 0;
    } else if (hnext <= 1e-14 * S->aw_norm) {
      cont = 0;
    } else if (k >= a.m || S->iters >= S->maxit || *(volatile int*)a.err) {
      cont = 0;
    }
    if (cont) {
      a.sig[j + 1] = 1.0 / hnext;
      S->j = j + 1;
    }
    S->cont = cont;
    gm_set_cond(a, a.h_inner, (unsigned)cont);
  }
}

// Back substitution H(0:k, 0:k) y = g(0:k), row by row as in the definition.
template <typename T>
__global__ void gm_gy(GmArgs<T> a) {
  if (threadIdx.x != 0) return;
  const int k = a.S->kcols, ld = a.m + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = a.g[i];
    for (int q = i + 1; q < k; ++q) s -= a.H[(long long)q * ld + i] * a.y[q];
    a.y[i] = s / a.H[(long long)i * ld + i];
  }
}

// x += V_k (sig .* y).
template <typename T, int KP>
__global__ void __launch_bounds__(kBlock) gm_gx(GmArgs<T> a) {
  __shared__ double coef[KP];
  const int k = a.S->kcols;
  for (int c = threadIdx.x; c < k; c += kBlock) coef[c] = a.sig[c] * a.y[c];
  __syncthreads();
  GM_ROW_LOOP(a) {
    double x = (double)a.x[i];
#pragma unroll
    for (int c0 = 0; c0 < KP; c0 += 4)
      if (c0 < k) {
#pragma unroll
        for (int c = c0; c < c0 + 4; ++c)
          if (c < k) x = fma((double)a.V[(long long)c * a.ldv + i], coef[c], x);
      }
    a.x[i] = (T)x;
  }
}

// ------------------------------------------------------------------ host

struct GmPlan {
  int g_tile, g_vec, wmode, KP;
  GmArgs<double> a;
  double* wbuf;
  GmState host_state;
};

template <int KP>
static void gm_launch_kp(gsk_ctx* ctx, GmPlan& P, int k, cudaStream_t s) {
  GmArgs<double>& a = P.a;
  switch (k) {
    case kKWeights: launch_gs_norm(ctx, a.n, a.nnz, a.rowptr, a.val, 2.0, P.wbuf, a.err, s); break;
    case kKUnitCheck: launch_unit_check(ctx, a.n, P.wbuf, a.red, &a.S->w_identity, s); break;
    case kKGmInit: gm_residual<double, true><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKGmGa: gm_ga<double><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKGmGd: gm_gd<double, KP><<<P.g_vec, kBlock, 0, s>>>(a); break;
    case kKGmGb: gm_gb<double, KP><<<P.g_vec, kBlock, 0, s>>>(a); break;
    case kKGmGc: gm_gc<double, KP><<<P.g_vec, kBlock, 0, s>>>(a); break;
    case kKGmGy: gm_gy<double><<<1, 32, 0, s>>>(a); break;
    case kKGmGx: gm_gx<double, KP><<<P.g_vec, kBlock, 0, s>>>(a); break;
    case kKGmGr: gm_residual<double, false><<<P.g_tile, kBlock, 0, s>>>(a); break;
  }
}

static void gm_launch(gsk_ctx* ctx, GmPlan& P, int k, cudaStream_t s) {
  if (P.KP == 16) gm_launch_kp<16>(ctx, P, k, s);
  else if (P.KP == 32) gm_launch_kp<32>(ctx, P, k, s);
  else gm_launch_kp<64>(ctx, P, k, s);
}

static gsk_status gm_record(gsk_ctx* ctx, GmPlan& P, cudaGraphExec_t* exec_out) {
  cudaStream_t cs = ctx->capture;
  cudaGraph_t top = nullptr;
  GSK_CK(cudaGraphCreate(&top, 0));
  struct Guard {
    cudaGraph_t g;
    ~Guard() { if (g) cudaGraphDestroy(g); }
  } guard{top};
  GmArgs<double>& a = P.a;
  a.in_graph = 1;
  GSK_CK(cudaGraphConditionalHandleCreate(&a.h_outer, top, 1u, cudaGraphCondAssignDefault));
  // top: [weights] -> init -> WHILE_outer{ WHILE_inner{ga, gb, gc} -> gy -> gx -> gr }
  // The init kernel sets the inner handle, which is created against the
  // outer body; so the outer node is added first (no dependencies yet), the
  // init chain is recorded, and the edge init -> outer is added afterwards.
  cudaGraphNode_t onode;
  cudaGraph_t obody;
  GSK_CK(add_conditional(top, {}, a.h_outer, cudaGraphCondTypeWhile, 1, &onode, &obody));
  GSK_CK(cudaGraphConditionalHandleCreate(&a.h_inner, obody, 1u, 0));
  Capture c0;
  GSK_CK(c0.begin(cs, top));
  if (P.wmode == 0) {
    gm_launch(ctx, P, kKWeights, cs);
    gm_launch(ctx, P, kKUnitCheck, cs);
  }
  gm_launch(ctx, P, kKGmInit, cs);
  GSK_CK(c0.end());
  {
    std::vector<cudaGraphNode_t> to(c0.tail.size(), onode);
    GSK_CK(cudaGraphAddDependencies(top, c0.tail.data(), to.data(), nullptr, c0.tail.size()));
  }
  cudaGraphNode_t inode;
  cudaGraph_t ibody;
  GSK_CK(add_conditional(obody, {}, a.h_inner, cudaGraphCondTypeWhile, 1, &inode, &ibody));
  Capture c1;
  GSK_CK(c1.begin(cs, ibody));
  for (int k : {kKGmGa, kKGmGd, kKGmGb, kKGmGc}) gm_launch(ctx, P, k, cs);
  GSK_CK(c1.end());
  Capture c2;
  GSK_CK(c2.begin(cs, obody, {inode}));
  for (int k : {kKGmGy, kKGmGx, kKGmGr}) gm_launch(ctx, P, k, cs);
  GSK_CK(c2.end());
  GSK_CK(cudaGraphInstantiate(exec_out, top, 0));
  return GSK_OK;
}

static gsk_status gm_prepare(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                             const gsk_opts& opts, GmPlan& P) {
  if (A->dtype != GSK_F64) return ctx->fail(GSK_ERR_ARG, "the FP64 solver needs an FP64 matrix");
  if (!(tol >= 0.0) || opts.maxit < 0) return ctx->fail(GSK_ERR_ARG, "bad tol/maxit");
  if (A->n > 0 && (!b || !x)) return ctx->fail(GSK_ERR_ARG, "NULL b or x");
  const int n = A->n;
  P.wmode = opts.weights ? 2 : (opts.metric == GSK_METRIC_PLAIN ? 1 : 0);
  P.KP = m <= 16 ? 16 : (m <= 32 ? 32 : 64);
  // tile (SpMV) kernels carry no per-column accumulators: full occupancy
  P.g_tile = ctx->grid_for((n + 31) / 32, kWarpsPerBlock, 8);
  P.g_vec = ctx->grid_for(n, kBlock, P.KP <= 16 ? 4 : 2);
  const int gmax = P.g_tile > P.g_vec ? P.g_tile : P.g_vec;
  const long long ldv = ((long long)n + 63) / 64 * 64;
  GmArgs<double>& a = P.a;
  std::memset(&a, 0, sizeof(a));
  auto layout = [&](Arena& ar) {
    a.err = ar.take<int>(64);
    a.cnt = ar.take<unsigned>(64);
    a.red = take_red(ar, gmax, m + 2);
    a.S = ar.take<GmState>(1);
    a.H = ar.take<double>((size_t)(m + 1) * m);
    a.g = ar.take<double>(m + 1);
    a.cs = ar.take<double>(m);
    a.sn = ar.take<double>(m);
    a.y = ar.take<double>(m);
    a.h1 = ar.take<double>(m + 1);
    a.h2 = ar.take<double>(m + 1);
    a.sig = ar.take<double>(m + 1);
    a.V = ar.take<double>((size_t)ldv * (m + 1));
    P.wbuf = P.wmode == 0 ? ar.take<double>(n) : nullptr;
  };
  Arena sizing;
  layout(sizing);
  gsk_status s = ctx->reserve(sizing.off);
  if (s != GSK_OK) return s;
  Arena ar{(char*)ctx->ws, ctx->ws_bytes, 0};
  layout(ar);
  a.n = n;
  a.nnz = A->nnz;
  a.m = m;
  a.ldv = ldv;
  a.rowptr = A->rowptr;
  a.colidx = A->colidx;
  a.val = (const double*)A->val;
  a.b = (const double*)b;
  a.x = (double*)x;
  a.w = P.wmode == 0 ? P.wbuf : (P.wmode == 2 ? opts.weights : nullptr);
  a.in_graph = 0;
  GmState& hs = P.host_state;
  std::memset(&hs, 0, sizeof(hs));
  hs.tol = tol;
  hs.m = m;
  hs.maxit = opts.maxit;
  hs.w_identity = P.wmode == 1 ? 1 : 0;
  return GSK_OK;
}

static gsk_status gm_upload(gsk_ctx* ctx, GmPlan& P, cudaStream_t st) {
  const char* end = (const char*)(P.a.red.counters + (P.a.red.maxgrid + kGroup - 1) / kGroup + 1);
  GSK_CK(cudaMemsetAsync(ctx->ws, 0, end - (const char*)ctx->ws, st));
  GSK_CK(cudaMemcpyAsync(P.a.S, &P.host_state, sizeof(GmState), cudaMemcpyHostToDevice, st));
  return GSK_OK;
}

static gsk_status gm_readback(gsk_ctx* ctx, GmPlan& P, cudaStream_t st, GmState& out, int& bits) {
  char* hp = (char*)ctx->host_pinned;
  GSK_CK(cudaMemcpyAsync(hp, P.a.S, sizeof(GmState), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaMemcpyAsync(hp + 512, P.a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  std::memcpy(&out, hp, sizeof(out));
  std::memcpy(&bits, hp + 512, sizeof(int));
  return GSK_OK;
}

gsk_status gm_profile(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                      const gsk_opts& opts, int max_iters, LaunchTimer& T, gsk_info* info) {
  GmPlan P;
  gsk_status s = gm_prepare(ctx, A, b, x, m, tol, opts, P);
  if (s != GSK_OK) return s;
  if (A->n == 0) return GSK_OK;
  if ((s = gm_upload(ctx, P, T.st)) != GSK_OK) return s;
  auto timed = [&](int k, int step) -> gsk_status {
    return T.time(k, step, [&](cudaStream_t st) { gm_launch(ctx, P, k, st); });
  };
  if (P.wmode == 0) {
    if ((s = timed(kKWeights, -1)) != GSK_OK) return s;
    if ((s = timed(kKUnitCheck, -1)) != GSK_OK) return s;
  }
  if ((s = timed(kKGmInit, -1)) != GSK_OK) return s;
  GmState st;
  int bits = 0;
  if ((s = gm_readback(ctx, P, T.st, st, bits)) != GSK_OK) return s;
  while (!st.stop && !bits && st.iters < max_iters) {
    do {
      const int j = st.j;
      for (int k : {kKGmGa, kKGmGd, kKGmGb, kKGmGc})
        if ((s = timed(k, j)) != GSK_OK) return s;
      if ((s = gm_readback(ctx, P, T.st, st, bits)) != GSK_OK) return s;
    } while (st.cont && !bits && st.iters < max_iters);
    for (int k : {kKGmGy, kKGmGx, kKGmGr})
      if ((s = timed(k, -1)) != GSK_OK) return s;
    if ((s = gm_readback(ctx, P, T.st, st, bits)) != GSK_OK) return s;
  }
  if (info) *info = gsk_info{st.iters, st.restarts, 0, 0, st.conv, st.mu_true, st.est, 0.f};
  return err_bits_status(ctx, bits);
}

}  // namespace gsk

using namespace gsk;

extern "C" gsk_status gmres_solve(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                                  const gsk_opts* opts_in, gsk_info* info, void* stream) {
  if (!ctx) return GSK_ERR_ARG;
  gsk_status s = check_csr(ctx, A);
  if (s != GSK_OK) return s;
  gsk_opts opts;
  if (opts_in) opts = *opts_in;
  else gsk_opts_default(&opts);
  if (m < 1 || m > kMaxM) return ctx->fail(GSK_ERR_ARG, "m must be in 1..64");
  if (opts.precision == GSK_PREC_MIXED) return gmres_solve_mixed(ctx, A, b, x, m, tol, &opts, info, stream);
  cudaStream_t st = (cudaStream_t)stream;
  GmPlan P;
  if ((s = gm_prepare(ctx, A, b, x, m, tol, opts, P)) != GSK_OK) return s;
  if (A->n == 0) {
    if (info) *info = gsk_info{0, 0, 0, 0, GSK_CONVERGED, 0.0, 0.0, 0.f};
    return GSK_OK;
  }
  std::vector<uint64_t> key = {0, (uint64_t)A->n, (uint64_t)A->nnz, (uint64_t)m, (uint64_t)A->rowptr,
                               (uint64_t)A->colidx, (uint64_t)A->val, (uint64_t)b, (uint64_t)x, (uint64_t)P.wmode,
                               (uint64_t)P.a.w, (uint64_t)ctx->ws};
  GraphEntry* ge = ctx->find_graph(key);
  if (!ge) {
    cudaGraphExec_t ex = nullptr;
    if ((s = gm_record(ctx, P, &ex)) != GSK_OK) return s;
    ge = ctx->add_graph(key, ex);
  }
  GSK_CK(cudaEventRecord(ctx->ev0, st));
  if ((s = gm_upload(ctx, P, st)) != GSK_OK) return s;
  GSK_CK(cudaGraphLaunch(ge->exec, st));
  GSK_CK(cudaEventRecord(ctx->ev1, st));
  if (!info) return GSK_OK;
  GmState out;
  int bits = 0;
  if ((s = gm_readback(ctx, P, st, out, bits)) != GSK_OK) return s;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  *info = gsk_info{out.iters, out.restarts, 0, 0, out.conv, out.mu_true, out.est, ms};
  return err_bits_status(ctx, bits);
}
