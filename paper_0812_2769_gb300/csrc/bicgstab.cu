// Bi-CGSTAB host driver: graph recording, workspace layout, the C ABI entry
// point and the stream-mode profiler.  The kernels are in bicgstab_kernels.cuh.
#include "bicgstab_kernels.cuh"
#include "graph.hpp"
#include "ilu.cuh"

namespace gsk {

// ------------------------------------------------------------------ host

// Bi-CGSTAB iterations per pass of the graph's loop body.
constexpr int kBcgUnroll = 4;

// launches that apply the right preconditioner M (ILU(0)): p^ = M^-1 p before
// the product A p^, s^ = M^-1 s before A s^
constexpr int kBcgIluP = 1000, kBcgIluS = 1001;

struct BcgPlan {
  int g_tile, g_k2a, g_k3, g_k4, wmode;
  BcgArgs<double> a;
  double* wbuf;  // weights computed by the solver (or nullptr)
  const gsk_ilu0* pre = nullptr;
  double *ph = nullptr, *sh = nullptr;  // M^-1 p, M^-1 s
  BcgState host_state;
};

static void bcg_launch(gsk_ctx* ctx, BcgPlan& P, int k, cudaStream_t s) {
  BcgArgs<double>& a = P.a;
  switch (k) {
    case kKWeights: launch_gs_norm(ctx, a.n, a.nnz, a.rowptr, a.val, 2.0, P.wbuf, a.err, s); break;
    case kKUnitCheck: launch_unit_check(ctx, a.n, P.wbuf, a.red, &a.S->w_identity, s); break;
    case kKBcgInit: bcg_init<double><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKBcgK1: bcg_k1<double><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKBcgK2a: bcg_k2a<double><<<P.g_k2a, kBlock, 0, s>>>(a); break;
    case kKBcgK2b: bcg_k2b<double><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKBcgK3:
      if (P.pre) bcg_k3<double, true><<<P.g_k3, kBlock, 0, s>>>(a);
      else bcg_k3<double, false><<<P.g_k3, kBlock, 0, s>>>(a);
      break;
    case kBcgIluP:
    case kBcgIluS: {
      IluGate g = {};
      g.base = k == kBcgIluP ? a.p : a.s;
      g.skip0 = &a.S->stop;
      g.skip1 = &a.S->check;
      g.skip2 = k == kBcgIluS ? &a.S->halfexit : nullptr;
      ilu_launch_apply(ctx, P.pre, g, k == kBcgIluP ? P.ph : P.sh, s);
      break;
    }
    case kKBcgK4: bcg_k4<double><<<P.g_k4, kBlock, 0, s>>>(a); break;
    case kKBcgKt: bcg_kt<double><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kKBcgKr: bcg_kr<double><<<P.g_k4, kBlock, 0, s>>>(a); break;
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

  // loop body: kBcgUnroll iterations (k1, k2a, k2b, k3, k4) in a row, then the
  // true-residual check and finish (kt, kr), which return at entry unless an
  // iteration set check or stop; no conditional node inside the body
  Capture c1;
  GSK_CK(c1.begin(cs, wbody));
  for (int u = 0; u < kBcgUnroll; ++u) {
    if (P.pre) bcg_launch(ctx, P, kBcgIluP, cs);
    bcg_launch(ctx, P, kKBcgK1, cs);
    bcg_launch(ctx, P, kKBcgK2a, cs);
    if (P.pre) bcg_launch(ctx, P, kBcgIluS, cs);
    for (int k : {kKBcgK2b, kKBcgK3, kKBcgK4}) bcg_launch(ctx, P, k, cs);
  }
  bcg_launch(ctx, P, kKBcgKt, cs);
  bcg_launch(ctx, P, kKBcgKr, cs);
  GSK_CK(c1.end());

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
  P.pre = opts.precond;
  if (P.pre && (P.pre->n != n || P.pre->device != ctx->device))
    return ctx->fail(GSK_ERR_ARG, "the preconditioner belongs to another matrix or device");
  P.wmode = opts.weights ? 2 : (opts.metric == GSK_METRIC_PLAIN ? 1 : 0);
  P.g_tile = ctx->spmv_grid(n);
  // vector kernels (two FP64 rows per thread): as many blocks as fit, so
  // that enough loads are in flight to cover the HBM latency
  P.g_k2a = ctx->occ_grid((const void*)bcg_k2a<double>, (n + 1) / 2, kBlock);
  P.g_k3 = ctx->occ_grid((const void*)bcg_k3<double>, (n + 1) / 2, kBlock);
  P.g_k4 = ctx->occ_grid((const void*)bcg_k4<double>, (n + 1) / 2, kBlock);
  int gmax = ctx->grid_for(n, kBlock, 8);  // unit check
  for (int g : {P.g_tile, P.g_k2a, P.g_k3, P.g_k4}) gmax = g > gmax ? g : gmax;
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
    P.ph = P.pre ? ar.take<double>(n) : nullptr;
    P.sh = P.pre ? ar.take<double>(n) : nullptr;
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
  P.a.p_in = P.pre ? P.ph : P.a.p;
  P.a.s_in = P.pre ? P.sh : P.a.s;
  P.a.in_graph = 0;
  P.a.h_while = 0;
  P.a.vec_ok = ((uintptr_t)x % 16 == 0) && (P.a.w == nullptr || (uintptr_t)P.a.w % 16 == 0);
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
  const char* end = (const char*)(P.a.red.counters + 1);
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
  {
    // small systems: the whole solve on one thread-block cluster
    bool used = false;
    s = bcg_cluster_solve(ctx, A, b, x, tol, opts, info, st, &used);
    if (used) return s;
  }
  BcgPlan P;
  if ((s = bcg_prepare(ctx, A, b, x, tol, opts, P)) != GSK_OK) return s;
  if (A->n == 0) {
    if (info) *info = gsk_info{0, 0, 0, 0, GSK_CONVERGED, 0.0, 0.0, 0.f};
    return GSK_OK;
  }
  std::vector<uint64_t> key = {1, (uint64_t)A->n, (uint64_t)A->nnz, (uint64_t)A->rowptr, (uint64_t)A->colidx,
                               (uint64_t)A->val, (uint64_t)b, (uint64_t)x, (uint64_t)P.wmode,
                               (uint64_t)P.a.w, (uint64_t)ctx->ws, (uint64_t)(P.pre ? P.pre->serial : 0)};
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
  if (P.pre && (s = ilu_read_err(ctx, P.pre, st)) != GSK_OK) return s;
  return err_bits_status(ctx, bits);
}
