// Context management and the thin C ABI entry points that are not solvers.
#include <cmath>
#include <cstdlib>

#include "internal.hpp"

gsk_status gsk_ctx::reserve(size_t bytes) {
  if (bytes <= ws_bytes) return GSK_OK;
  clear_graphs();
  if (ws) {
    cudaError_t e = cudaFree(ws);
    ws = nullptr;
    ws_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
  }
  size_t want = bytes + bytes / 8 + (1u << 20);
  cudaError_t e = cudaMalloc(&ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ws = nullptr;
    return fail(GSK_ERR_OOM, "workspace allocation of " + std::to_string(want) + " bytes failed");
  }
  // reduction counters and flags must start at zero
  e = cudaMemset(ws, 0, want);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(workspace)");
  ws_bytes = want;
  return GSK_OK;
}

void gsk_ctx::clear_graphs() {
  for (auto& g : graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  graphs.clear();
}

gsk::GraphEntry* gsk_ctx::find_graph(const std::vector<uint64_t>& key) {
  for (auto& g : graphs)
    if (g.key == key) {
      g.last_use = ++clock;
      return &g;
    }
  return nullptr;
}

gsk::GraphEntry* gsk_ctx::add_graph(const std::vector<uint64_t>& key, cudaGraphExec_t exec) {
  constexpr size_t kMaxGraphs = 16;
  if (graphs.size() >= kMaxGraphs) {
    size_t victim = 0;
    for (size_t i = 1; i < graphs.size(); ++i)
      if (graphs[i].last_use < graphs[victim].last_use) victim = i;
    cudaGraphExecDestroy(graphs[victim].exec);
    graphs.erase(graphs.begin() + victim);
  }
  graphs.push_back(gsk::GraphEntry{key, exec, ++clock});
  return &graphs.back();
}

extern "C" {

const char* gsk_version(void) { return "gsk 0.1 (sm_103a)"; }

gsk_status gsk_ctx_create(gsk_ctx** out, int device) {
  if (!out) return GSK_ERR_ARG;
  *out = nullptr;
  gsk_ctx* ctx = new (std::nothrow) gsk_ctx();
  if (!ctx) return GSK_ERR_OOM;
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (const char* v = std::getenv("GSK_SPMV_BLOCKS_PER_SM")) {
    const int k = std::atoi(v);
    if (k >= 1 && k <= 5) ctx->spmv_per_sm = k;
  }
  if (const char* v = std::getenv("GSK_BASIS_BLOCKS_PER_SM")) {
    const int k = std::atoi(v);
    if (k >= 1 && k <= 32) ctx->basis_per_sm = k;
  }
  if (const char* v = std::getenv("GSK_SMALL_N")) {
    const int k = std::atoi(v);
    if (k >= 0) ctx->small_n = k;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->host_pinned, 1 << 16);
  if (e != cudaSuccess) {
    gsk_ctx_destroy(ctx);
    return GSK_ERR_CUDA;
  }
  *out = ctx;
  return GSK_OK;
}

gsk_status gsk_ctx_destroy(gsk_ctx* ctx) {
  if (!ctx) return GSK_OK;
  cudaSetDevice(ctx->device);
  ctx->clear_graphs();
  if (ctx->aux) gsk_ctx_destroy(ctx->aux);
  cudaSetDevice(ctx->device);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  delete ctx;
  return GSK_OK;
}

const char* gsk_last_error(gsk_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

void gsk_opts_default(gsk_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->maxit = 10000;
  o->refresh = 3;
  o->precision = GSK_PREC_F64;
  o->metric = GSK_METRIC_GS2;
  o->weights = nullptr;
  o->inner_tol = 1e-5;
  o->inner_maxit = 0;
  o->max_refinements = 0;
}

gsk_status gs_scale(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* d_out, void* stream) {
  if (!ctx) return GSK_ERR_ARG;
  gsk_status s = gsk::check_csr(ctx, A);
  if (s != GSK_OK) return s;
  if (!(p >= 1.0)) return ctx->fail(GSK_ERR_ARG, "p must be >= 1 or INFINITY");
  if (A->n == 0) return GSK_OK;
  return gsk::run_gs_scale(ctx, A, b, p, d_out, (cudaStream_t)stream);
}

gsk_status gsk_profile_gs_scale(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* d_out, void* stream,
                                float* kernel_ms) {
  if (!ctx) return GSK_ERR_ARG;
  if (!kernel_ms) return ctx->fail(GSK_ERR_ARG, "NULL kernel_ms");
  *kernel_ms = 0.0f;
  gsk_status s = gsk::check_csr(ctx, A);
  if (s != GSK_OK) return s;
  if (!(p >= 1.0)) return ctx->fail(GSK_ERR_ARG, "p must be >= 1 or INFINITY");
  if (A->n == 0) return GSK_OK;
  return gsk::run_gs_scale(ctx, A, b, p, d_out, (cudaStream_t)stream, kernel_ms);
}

gsk_status gs_scale_sym(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* s_out, double* w_out, void* stream) {
  if (!ctx) return GSK_ERR_ARG;
  gsk_status s = gsk::check_csr(ctx, A);
  if (s != GSK_OK) return s;
  if (!(p >= 1.0)) return ctx->fail(GSK_ERR_ARG, "p must be >= 1 or INFINITY");
  if (A->n > 0 && (!A->colidx || !s_out)) return ctx->fail(GSK_ERR_ARG, "NULL colidx or s_out");
  if (A->n == 0) return GSK_OK;
  return gsk::run_gs_scale_sym(ctx, A, b, p, s_out, w_out, (cudaStream_t)stream);
}

gsk_status gsk_diag_mul(gsk_ctx* ctx, int n, const double* s, void* x, gsk_dtype dtype, void* stream) {
  if (!ctx) return GSK_ERR_ARG;
  if (n < 0 || (n > 0 && (!s || !x)) || (dtype != GSK_F64 && dtype != GSK_F32))
    return ctx->fail(GSK_ERR_ARG, "bad n, s, x or dtype");
  if (n == 0) return GSK_OK;
  return gsk::launch_diag_mul(ctx, n, s, x, dtype, (cudaStream_t)stream);
}

gsk_status gsk_spmv(gsk_ctx* ctx, const gsk_csr* A, const void* x, void* y, void* stream) {
  if (!ctx) return GSK_ERR_ARG;
  gsk_status s = gsk::check_csr(ctx, A);
  if (s != GSK_OK) return s;
  if (A->n > 0 && (!x || !y)) return ctx->fail(GSK_ERR_ARG, "NULL x or y");
  if ((s = ctx->reserve(256)) != GSK_OK) return s;
  // the structure error word lives at the start of the workspace; it is
  // read back by gsk_spmv_check (tests) and reset here
  int* err = (int*)ctx->ws;
  cudaStream_t st = (cudaStream_t)stream;
  GSK_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  return gsk::launch_spmv(ctx, A, x, y, err, st);
}

const char* gsk_kernel_name(int k) {
  static const char* names[gsk::kKCount] = {
      "gs_norm(w)", "unit_check", "bcg_init", "bcg_k1_spmv_dot", "bcg_k2a_s_update", "bcg_k2b_spmv_dot",
      "bcg_k3_xr_update", "bcg_k4_p_update", "bcg_kt_true_residual", "bcg_kr_finish", "gm_init_residual",
      "gm_ga_spmv", "gm_gb_cgs_pass2", "gm_gc_cgs_pass3_givens", "gm_gy_backsolve", "gm_gx_x_update",
      "gm_gr_restart_residual", "gm_gd_cgs_pass1"};
  return (k >= 0 && k < gsk::kKCount) ? names[k] : "";
}

gsk_status gsk_profile_solve(gsk_ctx* ctx, int solver, const gsk_csr* A, const void* b, void* x, int m,
                             double tol, const gsk_opts* opts_in, int max_iters, gsk_launch_record* recs, int cap,
                             int* nrec, gsk_info* info, void* stream) {
  if (!ctx) return GSK_ERR_ARG;
  gsk_status s = gsk::check_csr(ctx, A);
  if (s != GSK_OK) return s;
  if (!recs || cap < 0 || max_iters < 0) return ctx->fail(GSK_ERR_ARG, "bad record buffer or max_iters");
  gsk_opts opts;
  if (opts_in) opts = *opts_in;
  else gsk_opts_default(&opts);
  if (opts.precision != GSK_PREC_F64) return ctx->fail(GSK_ERR_ARG, "profiling runs the FP64 solvers");
  if (opts.precond) return ctx->fail(GSK_ERR_ARG, "profiling runs the solvers without a preconditioner");
  gsk::LaunchTimer T;
  T.ctx = ctx;
  T.st = (cudaStream_t)stream;
  if (solver == 0) {
    if (m < 1 || m > gsk::kMaxM) return ctx->fail(GSK_ERR_ARG, "m must be in 1..64");
    s = gsk::gm_profile(ctx, A, b, x, m, tol, opts, max_iters, T, info);
  } else if (solver == 1) {
    s = gsk::bcg_profile(ctx, A, b, x, tol, opts, max_iters, T, info);
  } else {
    return ctx->fail(GSK_ERR_ARG, "solver must be 0 (GMRES) or 1 (Bi-CGSTAB)");
  }
  gsk_status s2 = T.finish(recs, cap, nrec);
  return s != GSK_OK ? s : s2;
}

gsk_status gsk_workspace_bytes(int n, int nnz, int solver, int m, int precision, size_t* bytes) {
  if (!bytes || n < 0 || nnz < 0) return GSK_ERR_ARG;
  const size_t nn = (size_t)n;
  size_t vec = precision == GSK_PREC_MIXED ? 4 : 8;
  size_t b = 1u << 20;  // states, counters, reduction scratch
  if (solver == 0) {
    if (m < 1 || m > gsk::kMaxM) return GSK_ERR_ARG;
    b += vec * nn * (size_t)(m + 2) + 8 * nn;  // basis, weights
  } else {
    b += vec * nn * 6 + 8 * nn;
  }
  if (precision == GSK_PREC_MIXED) b += 8 * nn * 2 + 4 * (size_t)nnz;  // FP64 residual/correction + FP32 values
  *bytes = b;
  return GSK_OK;
}

}  // extern "C"
