// GMRES(m) host driver: graph recording, workspace layout, the C ABI entry
// point and the stream-mode profiler.  The kernels are in gmres_kernels.cuh.
#include "gmres_kernels.cuh"
#include "graph.hpp"

namespace gsk {

// ------------------------------------------------------------------ host

struct GmPlan {
  int g_tile, g_gd, g_gb, g_gc, g_gx, wmode, KP;
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
    case kKGmGd: gm_gd<double, KP><<<P.g_gd, kBlock, 0, s>>>(a); break;
    case kKGmGb: gm_gb<double, KP><<<P.g_gb, kBlock, 0, s>>>(a); break;
    case kKGmGc: gm_gc<double, KP><<<P.g_gc, kBlock, 0, s>>>(a); break;
    case kKGmGy: gm_gy<double><<<1, 32, 0, s>>>(a); break;
    case kKGmGx: gm_gx<double, KP><<<P.g_gx, kBlock, 0, s>>>(a); break;
    case kKGmGr: gm_residual<double, false><<<P.g_tile, kBlock, 0, s>>>(a); break;
  }
}

// Grids of the basis kernels (CGS passes: two FP64 rows per thread; x
// update: one): as many blocks as fit at each kernel's occupancy.
template <int KP>
static void gm_grids_kp(gsk_ctx* ctx, GmPlan& P, int n) {
  P.g_gd = ctx->occ_grid((const void*)gm_gd<double, KP>, (n + 1) / 2, kBlock);
  P.g_gb = ctx->occ_grid((const void*)gm_gb<double, KP>, (n + 1) / 2, kBlock);
  P.g_gc = ctx->occ_grid((const void*)gm_gc<double, KP>, (n + 1) / 2, kBlock);
  P.g_gx = ctx->occ_grid((const void*)gm_gx<double, KP>, n, kBlock);
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
  P.g_tile = ctx->spmv_grid(n);
  if (P.KP == 16) gm_grids_kp<16>(ctx, P, n);
  else if (P.KP == 32) gm_grids_kp<32>(ctx, P, n);
  else gm_grids_kp<64>(ctx, P, n);
  int gmax = ctx->grid_for(n, kBlock, 8);  // unit check
  for (int g : {P.g_tile, P.g_gd, P.g_gb, P.g_gc}) gmax = g > gmax ? g : gmax;
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
  hs.hbrk = 1e-14;
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
