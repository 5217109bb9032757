// Restarted GMRES(m) with classical Gram-Schmidt applied twice (Sec. 2),
// with the Arnoldi process, the Givens rotations, the Hessenberg
// least-squares solve and every stopping decision on the device.
//
// Basis storage: V is column-major (leading dimension ldv) and column k holds
// an unnormalised vector; the Arnoldi vector is v_k = sig[k] * V[:, k].  The
// scale is folded into the next product instead of a separate normalisation
// pass over V.
//
// One Arnoldi step j (k = j + 1 basis vectors) is three kernels:
//   ga  w = A v_j -> V[:, j+1];  h1 = V_k^T w;  ||w||            (SpMV + multi-dot)
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
  int m, maxit, iters, restarts, conv, j, kcols, stop, est_hit, w_identity;
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
};

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
    cudaGraphSetConditional(a.h_outer, (unsigned)!stop);
    cudaGraphSetConditional(a.h_inner, (unsigned)!stop);
  }
}

// Arnoldi pass 1: w = A v_j stored in V[:, j+1]; h1 = V_k^T w; ||w||^2.
template <typename T, int KP>
__global__ void __launch_bounds__(kBlock) gm_ga(GmArgs<T> a) {
  __shared__ GmSmem<T> sm;
  __shared__ double res[KP + 1], tot[KP + 1];
  const GmState* S = a.S;
  const int j = S->j, k = j + 1;
  const T* vj = a.V + (long long)j * a.ldv;
  T* wout = a.V + (long long)(j + 1) * a.ldv;
  const double sj = a.sig[j];
  double acc[KP], ww[1] = {0.0};
#pragma unroll
  for (int c = 0; c < KP; ++c) acc[c] = 0.0;
  GM_TILE_LOOP(a) {
    const int i = tile * 32 + lane_id();
    const T av = csr_tile_row<T, T, kStageCap>(a.rowptr, a.colidx, a.val, vj, a.n, a.nnz, tile * 32,
                                                 sm.stage[warp_id()], a.err);
    if (i < a.n) {
      const T w = (T)(sj * (double)av);
      wout[i] = w;
#pragma unroll
      for (int c = 0; c < KP; ++c)
        if (c < k) acc[c] = fma((double)a.V[(long long)c * a.ldv + i], (double)w, acc[c]);
      ww[0] = fma((double)w, (double)w, ww[0]);
    }
  }
  // [h1_0 .. h1_{k-1}, ||w||^2] side by side for one grid reduction
  block_sum_chunked<KP>(acc, k, sm.table, res);
  block_sum_chunked<1>(ww, 1, sm.table, res + k);
  if (grid_sum(res, k + 1, a.red, tot)) {
    for (int c = threadIdx.x; c < k; c += kBlock) a.h1[c] = a.sig[c] * tot[c];
    if (threadIdx.x == 0) a.S->aw_norm = sqrt(tot[k]);
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
    for (int c = 0; c < KP; ++c)
      if (c < k) w = fma(-(double)a.V[(long long)c * a.ldv + i], coef[c], w);
    const T wt = (T)w;
    wv[i] = wt;
#pragma unroll
    for (int c = 0; c < KP; ++c)
      if (c < k) acc[c] = fma((double)a.V[(long long)c * a.ldv + i], (double)wt, acc[c]);
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
    for (int c = 0; c < KP; ++c)
      if (c < k) w = fma(-(double)a.V[(long long)c * a.ldv + i], coef[c], w);
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
    cudaGraphSetConditional(a.h_inner, (unsigned)cont);
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
    for (int c = 0; c < KP; ++c)
      if (c < k) x = fma((double)a.V[(long long)c * a.ldv + i], coef[c], x);
    a.x[i] = (T)x;
  }
}

// ------------------------------------------------------------------ host

template <int KP>
static gsk_status gm_record(gsk_ctx* ctx, GmArgs<double>& a, int g_tile, int g_vec, int wmode, double* wbuf,
                            int* wid_out, cudaGraphExec_t* exec_out) {
  cudaStream_t cs = ctx->capture;
  cudaGraph_t top = nullptr;
  GSK_CK(cudaGraphCreate(&top, 0));
  struct Guard {
    cudaGraph_t g;
    ~Guard() { if (g) cudaGraphDestroy(g); }
  } guard{top};
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
  if (wmode == 0) {
    launch_gs_norm(ctx, a.n, a.nnz, a.rowptr, a.val, 2.0, wbuf, a.err, cs);
    launch_unit_check(ctx, a.n, wbuf, a.red, wid_out, cs);
  }
  gm_residual<double, true><<<g_tile, kBlock, 0, cs>>>(a);
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
  gm_ga<double, KP><<<g_tile, kBlock, 0, cs>>>(a);
  gm_gb<double, KP><<<g_vec, kBlock, 0, cs>>>(a);
  gm_gc<double, KP><<<g_vec, kBlock, 0, cs>>>(a);
  GSK_CK(c1.end());
  Capture c2;
  GSK_CK(c2.begin(cs, obody, {inode}));
  gm_gy<double><<<1, 32, 0, cs>>>(a);
  gm_gx<double, KP><<<g_vec, kBlock, 0, cs>>>(a);
  gm_residual<double, false><<<g_tile, kBlock, 0, cs>>>(a);
  GSK_CK(c2.end());
  GSK_CK(cudaGraphInstantiate(exec_out, top, 0));
  return GSK_OK;
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
  if (A->dtype != GSK_F64) return ctx->fail(GSK_ERR_ARG, "the FP64 solver needs an FP64 matrix");
  if (!(tol >= 0.0) || opts.maxit < 0) return ctx->fail(GSK_ERR_ARG, "bad tol/maxit");
  if (A->n > 0 && (!b || !x)) return ctx->fail(GSK_ERR_ARG, "NULL b or x");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = A->n;
  if (n == 0) {
    if (info) *info = gsk_info{0, 0, 0, 0, GSK_CONVERGED, 0.0, 0.0, 0.f};
    return GSK_OK;
  }
  const int wmode = opts.weights ? 2 : (opts.metric == GSK_METRIC_PLAIN ? 1 : 0);
  const int KP = m <= 16 ? 16 : (m <= 32 ? 32 : 64);
  const int g_tile = ctx->grid_for((n + 31) / 32, kWarpsPerBlock, KP <= 16 ? 4 : 2);
  const int g_vec = ctx->grid_for(n, kBlock, KP <= 16 ? 4 : 2);
  const int gmax = g_tile > g_vec ? g_tile : g_vec;
  const long long ldv = ((long long)n + 63) / 64 * 64;

  GmArgs<double> a;
  std::memset(&a, 0, sizeof(a));
  double* wbuf = nullptr;
  int* wid_out = nullptr;
  auto layout = [&](Arena& ar) {
    a.err = ar.take<int>(64);
    a.S = ar.take<GmState>(1);
    a.cnt = ar.take<unsigned>(64);
    a.red = take_red(ar, gmax, m + 2);
    a.H = ar.take<double>((size_t)(m + 1) * m);
    a.g = ar.take<double>(m + 1);
    a.cs = ar.take<double>(m);
    a.sn = ar.take<double>(m);
    a.y = ar.take<double>(m);
    a.h1 = ar.take<double>(m + 1);
    a.h2 = ar.take<double>(m + 1);
    a.sig = ar.take<double>(m + 1);
    a.V = ar.take<double>((size_t)ldv * (m + 1));
    wbuf = wmode == 0 ? ar.take<double>(n) : nullptr;
  };
  Arena sizing;
  layout(sizing);
  if ((s = ctx->reserve(sizing.off)) != GSK_OK) return s;
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
  a.w = wmode == 0 ? wbuf : (wmode == 2 ? opts.weights : nullptr);
  wid_out = &a.S->w_identity;

  std::vector<uint64_t> key = {0, (uint64_t)n, (uint64_t)A->nnz, (uint64_t)m, (uint64_t)A->rowptr,
                               (uint64_t)A->colidx, (uint64_t)A->val, (uint64_t)b, (uint64_t)x, (uint64_t)wmode,
                               (uint64_t)a.w, (uint64_t)ctx->ws};
  GraphEntry* ge = ctx->find_graph(key);
  if (!ge) {
    cudaGraphExec_t ex = nullptr;
    if (KP == 16) s = gm_record<16>(ctx, a, g_tile, g_vec, wmode, wbuf, wid_out, &ex);
    else if (KP == 32) s = gm_record<32>(ctx, a, g_tile, g_vec, wmode, wbuf, wid_out, &ex);
    else s = gm_record<64>(ctx, a, g_tile, g_vec, wmode, wbuf, wid_out, &ex);
    if (s != GSK_OK) return s;
    ge = ctx->add_graph(key, ex);
  }

  GmState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.tol = tol;
  hs.m = m;
  hs.maxit = opts.maxit;
  hs.w_identity = wmode == 1 ? 1 : 0;
  GSK_CK(cudaEventRecord(ctx->ev0, st));
  // error word, counters and reduction scratch sit at the start of the
  // workspace; other solves lay the workspace out differently, so clear them
  GSK_CK(cudaMemsetAsync(ctx->ws, 0, (char*)(a.red.counters + (a.red.maxgrid + kGroup - 1) / kGroup + 1) -
                                         (char*)ctx->ws, st));
  GSK_CK(cudaMemcpyAsync(a.S, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  GSK_CK(cudaGraphLaunch(ge->exec, st));
  GSK_CK(cudaEventRecord(ctx->ev1, st));
  if (!info) return GSK_OK;
  char* hp = (char*)ctx->host_pinned;
  GSK_CK(cudaMemcpyAsync(hp, a.S, sizeof(GmState), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaMemcpyAsync(hp + 512, a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  GmState out;
  std::memcpy(&out, hp, sizeof(out));
  int bits;
  std::memcpy(&bits, hp + 512, sizeof(int));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  *info = gsk_info{out.iters, out.restarts, 0, 0, out.conv, out.mu_true, out.est, ms};
  return err_bits_status(ctx, bits);
}
