// Host-side internals of libgsk: the context, its workspace arena, launch
// geometry and the cache of instantiated CUDA graphs.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "gsk.h"
#include "device_common.cuh"

namespace gsk {

constexpr int kBlock = 256;           // threads per block for every kernel
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr int kStageCap = 256;        // nonzeros staged per 32-row tile (7-point: 224)
constexpr int kMaxRedValues = 72;     // values per grid-reduction site (GMRES: m+2)
constexpr int kMaxM = 64;             // largest GMRES restart length of the graph path

// One instantiated graph plus the key it was built for.
struct GraphEntry {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

// Bump allocator over the context's device workspace.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

}  // namespace gsk

struct gsk_ctx {
  int device = 0;
  int num_sms = 0;
  // blocks per SM of the SpMV-family kernels (GSK_SPMV_BLOCKS_PER_SM, 1..5)
  int spmv_per_sm = 5;
  // cap on blocks per SM of the GMRES basis kernels (GSK_BASIS_BLOCKS_PER_SM):
  // more resident blocks hide less latency than they cost, as the second CGS
  // pass re-reads the basis rows of the first from L1 (measured best: 3)
  int basis_per_sm = 3;
  // Bi-CGSTAB and GMRES on one thread-block cluster for systems of at most
  // small_n rows that fit the cluster's shared memory (GSK_SMALL_N
  // overrides; 0 disables); cluster_max_n: the most rows the Bi-CGSTAB
  // cluster kernel holds on this device (-1: not yet queried)
  int small_n = 32768;
  int cluster_max_n = -1;
  int cluster_smem = 0;  // shared memory per CTA of the cluster kernel
  std::string last_error;
  // device workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // pinned host staging for small read-backs
  void* host_pinned = nullptr;
  cudaStream_t capture = nullptr;  // private stream used only for graph capture
  // the batched solvers' grid-wide lane: a child context (its own workspace
  // and graphs) and stream, so that systems routed out of a batch run beside
  // its persistent launch; created on first use
  gsk_ctx* aux = nullptr;
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<gsk::GraphEntry> graphs;
  uint64_t clock = 0;

  gsk_status fail(gsk_status st, const std::string& what) {
    last_error = what;
    return st;
  }
  gsk_status cuda_fail(cudaError_t e, const char* what) {
    last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return GSK_ERR_CUDA;
  }
  // Make the workspace at least `bytes` large.  Growing invalidates every
  // cached graph (their kernel arguments point into the old workspace).
  gsk_status reserve(size_t bytes);
  void clear_graphs();
  gsk::GraphEntry* find_graph(const std::vector<uint64_t>& key);
  gsk::GraphEntry* add_graph(const std::vector<uint64_t>& key, cudaGraphExec_t exec);
  // Grid of the SpMV-family kernels: one 256-row chunk per block trip, at
  // most spmv_per_sm blocks per SM (each holds a 45 KB shared-memory ring).
  int spmv_grid(int n) const { return grid_for(((long long)n + 255) / 256, 1, spmv_per_sm); }
  // Grid of a grid-stride kernel: every block that fits on the device at once
  // (the kernel's occupancy at kBlock threads, cached per kernel), fewer when
  // there is less work.
  std::unordered_map<const void*, int> occ_cache;
  int occ_grid(const void* kernel, long long work_items, int per_block, int cap_per_sm = 0) {
    auto it = occ_cache.find(kernel);
    int per_sm;
    if (it != occ_cache.end()) {
      per_sm = it->second;
    } else {
      per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      occ_cache[kernel] = per_sm;
    }
    if (cap_per_sm > 0 && per_sm > cap_per_sm) per_sm = cap_per_sm;
    return grid_for(work_items, per_block, per_sm);
  }
  int grid_for(long long work_items, int per_block, int per_sm = 8) const {
    long long g = (work_items + per_block - 1) / per_block;
    long long cap = (long long)num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
  }
};

#define GSK_CK(call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call); \
  } while (0)

namespace gsk {

// Reduction scratch for one site sized for `nv` values and `grid` blocks.
inline GridRed take_red(Arena& a, int grid, int nv) {
  GridRed r;
  r.partials = a.take<double>((size_t)nv * grid);
  r.counters = a.take<unsigned>(1);
  r.maxgrid = grid;
  return r;
}

// Validates the host-visible parts of a CSR descriptor.
inline gsk_status check_csr(gsk_ctx* ctx, const gsk_csr* A) {
  if (!A) return ctx->fail(GSK_ERR_ARG, "A is NULL");
  if (A->n < 0 || A->nnz < 0) return ctx->fail(GSK_ERR_ARG, "negative n or nnz");
  if (A->n > 0 && (!A->rowptr || (A->nnz > 0 && (!A->colidx || !A->val))))
    return ctx->fail(GSK_ERR_ARG, "NULL rowptr/colidx/val");
  if (A->dtype != GSK_F64 && A->dtype != GSK_F32) return ctx->fail(GSK_ERR_ARG, "unknown dtype");
  return GSK_OK;
}

// Status of the input checks done by the kernels (bits of kErr*).
inline gsk_status err_bits_status(gsk_ctx* ctx, int bits) {
  if (bits & kErrTimeout) return ctx->fail(GSK_ERR_TIMEOUT, "a bounded wait for a TMA copy gave up");
  if (bits & kErrIndex) return ctx->fail(GSK_ERR_ARG, "malformed CSR structure (rowptr extent or column index out of range)");
  if (bits & kErrNonFinite) return ctx->fail(GSK_ERR_NONFINITE, "NaN or Inf in the matrix or right-hand side");
  if (bits & kErrZeroRow) return ctx->fail(GSK_ERR_ZERO_ROW, "a row of the matrix is all zeros");
  return GSK_OK;
}

// Kernel identifiers used by the stream-mode profiler (gsk_profile_solve).
enum KernelId : int {
  kKWeights = 0, kKUnitCheck, kKBcgInit, kKBcgK1, kKBcgK2a, kKBcgK2b, kKBcgK3, kKBcgK4, kKBcgKt, kKBcgKr,
  kKGmInit, kKGmGa, kKGmGb, kKGmGc, kKGmGy, kKGmGx, kKGmGr, kKGmGd, kKCount
};

// Times kernel launches in stream mode with a CUDA event pair around each.
struct LaunchTimer {
  gsk_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> evs;
  std::vector<std::pair<int, int>> ids;

  template <class F>
  gsk_status time(int kernel, int step, F&& launch) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      launch(st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e0) evs.push_back(e0);
    if (e1) evs.push_back(e1);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "timed launch");
    ids.push_back({kernel, step});
    return GSK_OK;
  }
  // After the stream is synchronised: writes up to cap records.
  gsk_status finish(gsk_launch_record* recs, int cap, int* nrec) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaStreamSynchronize");
    int n = 0;
    for (size_t i = 0; i < ids.size() && n < cap; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, evs[2 * i], evs[2 * i + 1]);
      recs[n++] = gsk_launch_record{ids[i].first, ids[i].second, ms};
    }
    if (nrec) *nrec = n;
    return GSK_OK;
  }
  ~LaunchTimer() {
    for (auto ev : evs) cudaEventDestroy(ev);
  }
};

gsk_status bcg_cluster_solve(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, double tol,
                             const gsk_opts& opts, gsk_info* info, cudaStream_t st, bool* used);
// GMRES(m) on one thread-block cluster for small systems (cluster_gmres.cu);
// *used = false when the system is not taken.  gm_cluster_rows: the most
// rows it takes for restart length m.
gsk_status gm_cluster_solve(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                            const gsk_opts& opts, gsk_info* info, cudaStream_t st, bool* used);
int gm_cluster_rows(gsk_ctx* ctx, int m);
gsk_status bcg_profile(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, double tol, const gsk_opts& opts,
                       int max_iters, LaunchTimer& T, gsk_info* info);
gsk_status gm_profile(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                      const gsk_opts& opts, int max_iters, LaunchTimer& T, gsk_info* info);

// launchers implemented in the .cu files (capture-safe: no synchronisation)
gsk_status launch_spmv(gsk_ctx* ctx, const gsk_csr* A, const void* x, void* y, int* err, cudaStream_t st);
void launch_gs_norm(gsk_ctx* ctx, int n, int nnz, const int* rowptr, const double* val, double p, double* d,
                    int* err, cudaStream_t st);
void launch_unit_check(gsk_ctx* ctx, int n, const double* w, const GridRed& red, int* out, cudaStream_t st);
// kernel_ms (host, optional): device time of the GS(p) kernel alone, from a
// CUDA event pair around its launch.
gsk_status run_gs_scale(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* d_out, cudaStream_t st,
                        float* kernel_ms = nullptr);
gsk_status run_gs_scale_sym(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* s_out, double* w_out,
                            cudaStream_t st);
gsk_status launch_diag_mul(gsk_ctx* ctx, int n, const double* s, void* x, gsk_dtype dtype, cudaStream_t st);

}  // namespace gsk

// mixed-precision drivers (FP32 inner Krylov, FP64 refinement)
gsk_status gmres_solve_mixed(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                             const gsk_opts* opts, gsk_info* info, void* stream);
gsk_status bicgstab_solve_mixed(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, double tol,
                                const gsk_opts* opts, gsk_info* info, void* stream);

namespace gsk {

}  // namespace gsk
