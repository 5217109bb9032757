// GMRES(m) host driver: graph recording, workspace layout, the C ABI entry
// point and the stream-mode profiler.  The kernels are in gmres_kernels.cuh.
#include "gmres_kernels.cuh"
#include "graph.hpp"
#include "ilu.cuh"

#include <cmath>

namespace gsk {

// ------------------------------------------------------------------ host

// launches of the right-preconditioned cycle (ILU(0)): z = M^-1 v_j before
// the product of step j; z = M^-1 u and x += z after the cycle's update u
constexpr int kGmIluV = 1000, kGmIluU = 1001, kGmXadd = 1002;

struct GmPlan {
  const gsk_ilu0* pre = nullptr;
  double *zbuf = nullptr, *ubuf = nullptr;
  double* xzero = nullptr;  // Arnoldi mode: x0 = 0, so that r0 = v0
  int g_tile, g_gx, wmode, KP, nclass;
  int g_gd[kGmClasses], g_gb[kGmClasses], g_gc[kGmClasses];
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
    case kKGmGy: gm_gy<double><<<1, kBlock, 0, s>>>(a); break;
    case kKGmGx: gm_gx<double, KP><<<P.g_gx, kBlock, 0, s>>>(a); break;
    case kKGmGr: gm_residual<double, false><<<P.g_tile, kBlock, 0, s>>>(a); break;
    case kGmIluV: {
      IluGate g = {};
      g.base = a.V;
      g.col = &a.S->j;
      g.stride = a.ldv;
      g.run_if = a.unrolled ? &a.S->cont : nullptr;
      ilu_launch_apply(ctx, P.pre, g, P.zbuf, s);
      break;
    }
    case kGmIluU: {
      IluGate g = {};
      g.base = P.ubuf;
      ilu_launch_apply(ctx, P.pre, g, P.zbuf, s);
      break;
    }
    case kGmXadd: gm_xadd<double><<<P.g_gx, kBlock, 0, s>>>(a); break;
  }
}

// CGS passes of class c (KP = kGmClassKP[c] columns at most).
template <int KP>
static void gm_launch_cgs_kp(GmPlan& P, int k, int c, cudaStream_t s) {
  GmArgs<double>& a = P.a;
  switch (k) {
    case kKGmGd: gm_gd<double, KP><<<P.g_gd[c], kBlock, 0, s>>>(a); break;
    case kKGmGb: gm_gb<double, KP><<<P.g_gb[c], kBlock, 0, s>>>(a); break;
    // pass 3 keeps no per-column accumulators: one instance up to 32 columns
    case kKGmGc: gm_gc<double, (KP <= 32 ? 32 : 64)><<<P.g_gc[c], kBlock, 0, s>>>(a); break;
  }
}

static void gm_launch_cgs(GmPlan& P, int k, int c, cudaStream_t s) {
  switch (c) {
    case 0: gm_launch_cgs_kp<4>(P, k, c, s); break;
    case 1: gm_launch_cgs_kp<8>(P, k, c, s); break;
    case 2: gm_launch_cgs_kp<16>(P, k, c, s); break;
    case 3: gm_launch_cgs_kp<32>(P, k, c, s); break;
    default: gm_launch_cgs_kp<64>(P, k, c, s); break;
  }
}

// Grids: CGS passes (two FP64 rows per thread) and the x update (one), as
// many blocks as fit at each kernel's occupancy.
template <int KP>
static void gm_grids_class(gsk_ctx* ctx, GmPlan& P, int c, int n) {
  const int cap = ctx->basis_per_sm;
  P.g_gd[c] = ctx->occ_grid((const void*)gm_gd<double, KP>, (n + 1) / 2, kBlock, cap);
  P.g_gb[c] = ctx->occ_grid((const void*)gm_gb<double, KP>, (n + 1) / 2, kBlock, cap);
  P.g_gc[c] = ctx->occ_grid((const void*)gm_gc<double, (KP <= 32 ? 32 : 64)>, (n + 1) / 2, kBlock, cap);
}

static void gm_grids(gsk_ctx* ctx, GmPlan& P, int n) {
  for (int c = 0; c < kGmClasses; ++c) P.g_gd[c] = P.g_gb[c] = P.g_gc[c] = 1;
  gm_grids_class<4>(ctx, P, 0, n);
  if (P.nclass > 1) gm_grids_class<8>(ctx, P, 1, n);
  if (P.nclass > 2) gm_grids_class<16>(ctx, P, 2, n);
  if (P.nclass > 3) gm_grids_class<32>(ctx, P, 3, n);
  if (P.nclass > 4) gm_grids_class<64>(ctx, P, 4, n);
  if (P.KP == 16) P.g_gx = ctx->occ_grid((const void*)gm_gx<double, 16>, (n + 1) / 2, kBlock, ctx->basis_per_sm);
  else if (P.KP == 32) P.g_gx = ctx->occ_grid((const void*)gm_gx<double, 32>, (n + 1) / 2, kBlock, ctx->basis_per_sm);
  else P.g_gx = ctx->occ_grid((const void*)gm_gx<double, 64>, (n + 1) / 2, kBlock, ctx->basis_per_sm);
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
  // top: [weights] -> init -> WHILE_outer{ step 0 -> ... -> step m-1 -> gy -> gx -> gr },
  // step j = ga -> gd, gb (class of k = j + 1) -> gc.  The cycle's steps are
  // unrolled (no inner conditional node to relaunch per step, and each step's
  // basis kernels are fixed at record time); steps after the end of a cycle
  // return at entry.
  a.unrolled = 1;
  cudaGraphNode_t onode;
  cudaGraph_t obody;
  GSK_CK(add_conditional(top, {}, a.h_outer, cudaGraphCondTypeWhile, 1, &onode, &obody));
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
  Capture c1;
  GSK_CK(c1.begin(cs, obody));
  for (int j = 0; j < a.m; ++j) {
    const int c = gm_kclass(j + 1);
    if (P.pre) gm_launch(ctx, P, kGmIluV, cs);
    gm_launch(ctx, P, kKGmGa, cs);
    for (int k : {kKGmGd, kKGmGb, kKGmGc}) gm_launch_cgs(P, k, c, cs);
  }
  for (int k : {kKGmGy, kKGmGx}) gm_launch(ctx, P, k, cs);
  if (P.pre)
    for (int k : {kGmIluU, kGmXadd}) gm_launch(ctx, P, k, cs);
  gm_launch(ctx, P, kKGmGr, cs);
  GSK_CK(c1.end());
  GSK_CK(cudaGraphInstantiate(exec_out, top, 0));
  return GSK_OK;
}

static gsk_status gm_prepare(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                             const gsk_opts& opts, GmPlan& P, bool arnoldi = false) {
  if (A->dtype != GSK_F64) return ctx->fail(GSK_ERR_ARG, "the FP64 solver needs an FP64 matrix");
  if (!(tol >= 0.0) || opts.maxit < 0) return ctx->fail(GSK_ERR_ARG, "bad tol/maxit");
  if (A->n > 0 && (!b || !x)) return ctx->fail(GSK_ERR_ARG, "NULL b or x");
  const int n = A->n;
  P.pre = opts.precond;
  if (P.pre && (P.pre->n != n || P.pre->device != ctx->device))
    return ctx->fail(GSK_ERR_ARG, "the preconditioner belongs to another matrix or device");
  P.wmode = opts.weights ? 2 : (opts.metric == GSK_METRIC_PLAIN ? 1 : 0);
  P.KP = m <= 16 ? 16 : (m <= 32 ? 32 : 64);
  // tile (SpMV) kernels carry no per-column accumulators: full occupancy
  P.g_tile = ctx->spmv_grid(n);
  P.nclass = gm_kclass(m) + 1;
  gm_grids(ctx, P, n);
  int gmax = ctx->grid_for(n, kBlock, 8);  // unit check
  if (P.g_tile > gmax) gmax = P.g_tile;
  for (int c = 0; c < P.nclass; ++c)
    for (int g : {P.g_gd[c], P.g_gb[c], P.g_gc[c]}) gmax = g > gmax ? g : gmax;
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
    P.zbuf = P.pre ? ar.take<double>(n) : nullptr;
    P.ubuf = P.pre ? ar.take<double>(n) : nullptr;
    P.xzero = arnoldi ? ar.take<double>(n) : nullptr;
    a.Hraw = arnoldi ? ar.take<double>((size_t)(m + 1) * m) : nullptr;
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
  a.x = arnoldi ? P.xzero : (double*)x;
  a.w = P.wmode == 0 ? P.wbuf : (P.wmode == 2 ? opts.weights : nullptr);
  a.in_graph = 0;
  a.vec_ok = ((uintptr_t)x % 16) == 0;
  a.zin = P.pre ? P.zbuf : nullptr;
  a.u_out = P.pre ? P.ubuf : nullptr;
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
  const char* end = (const char*)(P.a.red.counters + 1);
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
      if ((s = timed(kKGmGa, j)) != GSK_OK) return s;
      for (int k : {kKGmGd, kKGmGb, kKGmGc})
        if ((s = T.time(k, j, [&](cudaStream_t q) { gm_launch_cgs(P, k, gm_kclass(j + 1), q); })) != GSK_OK)
          return s;
      if ((s = gm_readback(ctx, P, T.st, st, bits)) != GSK_OK) return s;
    } while (st.cont && !bits && st.iters < max_iters);
    for (int k : {kKGmGy, kKGmGx, kKGmGr})
      if ((s = timed(k, k == kKGmGr ? -1 : st.kcols - 1)) != GSK_OK) return s;
    if ((s = gm_readback(ctx, P, T.st, st, bits)) != GSK_OK) return s;
  }
  if (info) *info = gsk_info{st.iters, st.restarts, 0, 0, st.conv, st.mu_true, st.est, 0.f};
  return err_bits_status(ctx, bits);
}

// The Arnoldi process alone: init (r0 = v0 - A 0 = v0) and m steps of the
// solver's basis kernels, recorded once as a plain graph (no conditional
// node: as in the solver's unrolled cycle, the steps after the cycle has
// ended return at entry) and cached per (matrix, v0, m, workspace); gm_gc
// records the unrotated Hessenberg columns.  The steps end where a GMRES
// cycle would (k = m or breakdown): tol 0 never ends it, maxit = m.
static gsk_status gm_arnoldi(gsk_ctx* ctx, const gsk_csr* A, const double* v0, int m, double* H, int* steps,
                             cudaStream_t st) {
  gsk_opts opts;
  gsk_opts_default(&opts);
  opts.metric = GSK_METRIC_PLAIN;
  opts.maxit = m;
  GmPlan P;
  gsk_status s = gm_prepare(ctx, A, v0, (void*)v0, m, 0.0, opts, P, true);
  if (s != GSK_OK) return s;
  const size_t hbytes = sizeof(double) * (size_t)(m + 1) * m;
  std::memset(H, 0, hbytes);
  *steps = 0;
  if (A->n == 0) return GSK_OK;
  P.a.in_graph = 0;  // no conditional handle in this graph
  P.a.unrolled = 1;
  std::vector<uint64_t> key = {7, (uint64_t)A->n, (uint64_t)A->nnz, (uint64_t)m, (uint64_t)A->rowptr,
                               (uint64_t)A->colidx, (uint64_t)A->val, (uint64_t)v0, (uint64_t)ctx->ws};
  GraphEntry* ge = ctx->find_graph(key);
  if (!ge) {
    cudaGraph_t gph = nullptr;
    GSK_CK(cudaGraphCreate(&gph, 0));
    struct Guard {
      cudaGraph_t g;
      ~Guard() { if (g) cudaGraphDestroy(g); }
    } guard{gph};
    cudaStream_t cs = ctx->capture;
    Capture c0;
    GSK_CK(c0.begin(cs, gph));
    gm_launch(ctx, P, kKGmInit, cs);
    for (int j = 0; j < m; ++j) {
      gm_launch(ctx, P, kKGmGa, cs);
      for (int k : {kKGmGd, kKGmGb, kKGmGc}) gm_launch_cgs(P, k, gm_kclass(j + 1), cs);
    }
    GSK_CK(c0.end());
    cudaGraphExec_t ex = nullptr;
    GSK_CK(cudaGraphInstantiate(&ex, gph, 0));
    ge = ctx->add_graph(key, ex);
  }
  if ((s = gm_upload(ctx, P, st)) != GSK_OK) return s;
  GSK_CK(cudaMemsetAsync(P.xzero, 0, sizeof(double) * (size_t)A->n, st));
  GSK_CK(cudaMemsetAsync(P.a.Hraw, 0, hbytes, st));
  GSK_CK(cudaGraphLaunch(ge->exec, st));
  GmState S;
  int bits = 0;
  if ((s = gm_readback(ctx, P, st, S, bits)) != GSK_OK) return s;
  if ((s = err_bits_status(ctx, bits)) != GSK_OK) return s;
  if (!S.stop) *steps = S.kcols;
  GSK_CK(cudaMemcpyAsync(H, P.a.Hraw, hbytes, cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  for (size_t i = 0; i < (size_t)(m + 1) * m; ++i)
    if (!std::isfinite(H[i])) return ctx->fail(GSK_ERR_NONFINITE, "non-finite Hessenberg entry");
  return GSK_OK;
}

}  // namespace gsk

using namespace gsk;

extern "C" gsk_status gsk_arnoldi(gsk_ctx* ctx, const gsk_csr* A, const double* v0, int m, double* H, int* steps,
                                  void* stream) {
  if (!ctx) return GSK_ERR_ARG;
  gsk_status s = check_csr(ctx, A);
  if (s != GSK_OK) return s;
  if (m < 1 || m > kMaxM) return ctx->fail(GSK_ERR_ARG, "m must be in 1..64");
  if (!H || !steps || (A->n > 0 && !v0)) return ctx->fail(GSK_ERR_ARG, "NULL v0, H or steps");
  return gm_arnoldi(ctx, A, v0, m, H, steps, (cudaStream_t)stream);
}

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
  {
    // small systems: the whole solve on one thread-block cluster
    bool used = false;
    s = gm_cluster_solve(ctx, A, b, x, m, tol, opts, info, st, &used);
    if (used) return s;
  }
  GmPlan P;
  if ((s = gm_prepare(ctx, A, b, x, m, tol, opts, P)) != GSK_OK) return s;
  if (A->n == 0) {
    if (info) *info = gsk_info{0, 0, 0, 0, GSK_CONVERGED, 0.0, 0.0, 0.f};
    return GSK_OK;
  }
  std::vector<uint64_t> key = {0, (uint64_t)A->n, (uint64_t)A->nnz, (uint64_t)m, (uint64_t)A->rowptr,
                               (uint64_t)A->colidx, (uint64_t)A->val, (uint64_t)b, (uint64_t)x, (uint64_t)P.wmode,
                               (uint64_t)P.a.w, (uint64_t)ctx->ws, (uint64_t)(P.pre ? P.pre->serial : 0)};
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
  if (P.pre && (s = ilu_read_err(ctx, P.pre, st)) != GSK_OK) return s;
  return err_bits_status(ctx, bits);
}
