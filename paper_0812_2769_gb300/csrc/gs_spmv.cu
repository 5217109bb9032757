// Geometric scaling GS(p) (Sec. 1; Sec. 2, Eq. (2)) and the CSR product
// y = A x used by every Krylov step.
//
// GS(p) is one pass over the matrix (gs_rows_kernel<SCALE = true>): a warp
// copies the nonzeros of 32 consecutive rows into shared memory with
// coalesced loads, each lane forms d_i = 1/||a_i||_p of its own row in one
// sweep (row_inv_norm) and multiplies the row by it in place there, and the
// warp writes the tile back with coalesced stores: the values are read once
// and written once.  A row that is all zero or holds a non-finite entry (or
// whose b_i is not finite), and every row of a tile whose row pointers are
// out of range, is left as it is and the error is reported.
// The same kernel without the scaling (SCALE = false) gives the scales alone:
// the solvers' stopping-metric weights W = 1/||a_i||_2 and the first pass of
// the two-pass forms (the allocation-free entry point and the two-sided
// scaling), which scale only after every row has been checked.
#include <mutex>

#include "internal.hpp"
#include "spmv_tma.cuh"

namespace gsk {


struct TileExt {
  int row, rs, re, e0, e1;
  bool ok, tile_ok;
};

// Extents of the tile r0..r0+31 and of this lane's row, with bounds checks.
__device__ __forceinline__ TileExt tile_extents(const int* __restrict__ rowptr, int n, int nnz, int r0,
                                                int* err) {
  TileExt t;
  t.row = r0 + lane_id();
  const int last = min(31, n - 1 - r0);
  t.rs = t.re = 0;
  if (t.row < n) {
    t.rs = __ldg(rowptr + t.row);
    t.re = __ldg(rowptr + t.row + 1);
  }
  t.e0 = __shfl_sync(kFull, t.rs, 0);
  t.e1 = __shfl_sync(kFull, t.re, last);
  t.tile_ok = (t.e0 >= 0) && (t.e1 <= nnz) && (t.e1 >= t.e0);
  t.ok = t.tile_ok && ((t.row >= n) || (t.rs >= t.e0 && t.re >= t.rs && t.re <= t.e1));
  if (!t.ok) atomicOr(err, kErrIndex);
  return t;
}

__device__ __forceinline__ bool finite_bits(double v) { return finite_pattern(dbits(v)); }

// One warp per 32-row tile, tiles strided over the grid; PM is the kind of
// norm (p = 1, 2, inf or general).  d (optional)
// receives d_i = 1/||a_i||_p, or 0 for a row in error.  With SCALE, row i of
// A and b_i are multiplied by d_i in place (rows in error are left as they
// are).  Tiles whose nonzeros exceed the staging capacity (very long rows)
// are read straight from global memory.
template <typename T, bool SCALE, int PM>
__global__ void __launch_bounds__(kBlock, 8) gs_rows_kernel(int n, int nnz, const int* __restrict__ rowptr,
                                                         T* __restrict__ val, T* __restrict__ b, double p,
                                                         double* __restrict__ d, int* err) {
  __shared__ T stage[kWarpsPerBlock][kStageCap];
  T* st = stage[warp_id()];
  const long long ntiles = ((long long)n + 31) / 32;
  for (long long tile = (long long)blockIdx.x * kWarpsPerBlock + warp_id(); tile < ntiles;
       tile += (long long)gridDim.x * kWarpsPerBlock) {
    const TileExt t = tile_extents(rowptr, n, nnz, (int)(tile * 32), err);
    if (!t.tile_ok) continue;  // recorded; the tile's rows are not touched
    const int cnt = t.e1 - t.e0;
    const bool staged = cnt <= kStageCap;
    if (staged) {
#pragma unroll 4
      for (int k = lane_id(); k < cnt; k += 32) st[k] = val[t.e0 + k];
      __syncwarp();
    }
    double di = 0.0;
    bool scale = false;
    if (t.ok && t.row < n) {
      const T* rv = staged ? st + (t.rs - t.e0) : val + t.rs;
      di = row_inv_norm_pm<PM>(rv, t.re - t.rs, p, err);
      scale = dbits(di) != 0ull;  // 0 marks a row in error
      if (b && !finite_bits((double)b[t.row])) {
        atomicOr(err, kErrNonFinite);
        scale = false;
      }
      if (d) d[t.row] = scale ? di : 0.0;
    }
    if (SCALE) {
      if (staged) {
        if (scale)
          for (int k = t.rs - t.e0; k < t.re - t.e0; ++k) st[k] = (T)((double)st[k] * di);
        __syncwarp();
        if (__any_sync(kFull, scale)) {
#pragma unroll 4
          for (int k = lane_id(); k < cnt; k += 32) val[t.e0 + k] = st[k];
        }
      } else if (scale) {
        for (int k = t.rs; k < t.re; ++k) val[k] = (T)((double)val[k] * di);
      }
      if (scale && b) b[t.row] = (T)((double)b[t.row] * di);
    }
    if (staged) __syncwarp();  // the stage is reused by the warp's next tile
  }
}

// Second pass of the two-pass form: row i of A and b_i multiplied by d_i,
// only if the first pass recorded no error (A and b are then left as they
// were).  The same multiplications as gs_rows_kernel<SCALE = true>.
template <typename T>
__global__ void __launch_bounds__(kBlock) gs_apply_kernel(int n, int nnz, const int* __restrict__ rowptr,
                                                          T* __restrict__ val, T* __restrict__ b,
                                                          const double* __restrict__ d, int* err) {
  if (*(volatile int*)err != 0) return;  // errors found by the first pass: leave A and b as they are
  __shared__ T stage[kWarpsPerBlock][kStageCap];
  T* st = stage[warp_id()];
  const long long ntiles = ((long long)n + 31) / 32;
  for (long long tile = (long long)blockIdx.x * kWarpsPerBlock + warp_id(); tile < ntiles;
       tile += (long long)gridDim.x * kWarpsPerBlock) {
    const TileExt t = tile_extents(rowptr, n, nnz, (int)(tile * 32), err);
    const int cnt = t.e1 - t.e0;
    const double di = t.row < n ? d[t.row] : 0.0;
    if (cnt <= kStageCap) {
      for (int k = lane_id(); k < cnt; k += 32) st[k] = val[t.e0 + k];
      __syncwarp();
      if (t.row < n)
        for (int k = t.rs - t.e0; k < t.re - t.e0; ++k) st[k] = (T)((double)st[k] * di);
      __syncwarp();
      for (int k = lane_id(); k < cnt; k += 32) val[t.e0 + k] = st[k];
      __syncwarp();
    } else if (t.row < n) {
      for (int k = t.rs; k < t.re; ++k) val[k] = (T)((double)val[k] * di);
    }
    if (b && t.row < n) b[t.row] = (T)((double)b[t.row] * di);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) spmv_kernel(int n, int nnz, const int* __restrict__ rowptr,
                                                      const int* __restrict__ colidx, const T* __restrict__ val,
                                                      const T* __restrict__ x, T* __restrict__ y, int* err) {
  __shared__ PipeSmem<T> pipe;
  spmv_rows_tma(rowptr, colidx, val, x, n, nnz, pipe, err, [&](int i, T v) { y[i] = v; });
}

// Counts entries of w outside [1 - 4 eps, 1 + 4 eps] (integer compares on
// the bit patterns of positive doubles) and stores 1 in *out when there are
// none: the stopping-test weights are then the identity and are not loaded.
__global__ void __launch_bounds__(kBlock) unit_check_kernel(int n, const double* __restrict__ w, GridRed red,
                                                            int* out) {
  __shared__ double sm[kBlock], blk[1], tot[1];
  const long long lo = __double_as_longlong(1.0 - 4.0 * 2.220446049250313e-16);
  const long long hi = __double_as_longlong(1.0 + 4.0 * 2.220446049250313e-16);
  int cnt = 0;
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
    const long long bits = __double_as_longlong(__ldg(w + i));
    cnt += (bits < lo || bits > hi) ? 1 : 0;
  }
  double acc[1] = {(double)cnt};
  block_sum<1, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 1, red, tot) && threadIdx.x == 0) *out = tot[0] == 0.0 ? 1 : 0;
}

// Grid of the GS kernels: one warp per 32-row tile, every block that fits.
static int gs_grid(gsk_ctx* ctx, const void* kernel, int n) {
  return ctx->occ_grid(kernel, ((long long)n + 31) / 32, kWarpsPerBlock);
}

// Launches gs_rows_kernel<T, SCALE, PM> with PM taken from p; grid = 0 sizes
// the grid from the kernel's occupancy (needs ctx), else the given grid.
template <typename T, bool SCALE>
static void launch_gs_rows(gsk_ctx* ctx, int grid, int n, int nnz, const int* rowptr, T* val, T* b, double p,
                           double* d, int* err, cudaStream_t st) {
  auto go = [&](auto kernel) {
    const int g = grid > 0 ? grid : gs_grid(ctx, (const void*)kernel, n);
    kernel<<<g, kBlock, 0, st>>>(n, nnz, rowptr, val, b, p, d, err);
  };
  switch (pmode_of(p)) {
    case kP1: go(gs_rows_kernel<T, SCALE, kP1>); break;
    case kP2: go(gs_rows_kernel<T, SCALE, kP2>); break;
    case kPInf: go(gs_rows_kernel<T, SCALE, kPInf>); break;
    default: go(gs_rows_kernel<T, SCALE, kPGen>); break;
  }
}

void launch_gs_norm(gsk_ctx* ctx, int n, int nnz, const int* rowptr, const double* val, double p, double* d,
                    int* err, cudaStream_t st) {
  launch_gs_rows<double, false>(ctx, 0, n, nnz, rowptr, const_cast<double*>(val), nullptr, p, d, err, st);
}

void launch_unit_check(gsk_ctx* ctx, int n, const double* w, const GridRed& red, int* out, cudaStream_t st) {
  int grid = ctx->grid_for(n, kBlock, 8);
  if (grid > red.maxgrid) grid = red.maxgrid;
  unit_check_kernel<<<grid, kBlock, 0, st>>>(n, w, red, out);
}

gsk_status launch_spmv(gsk_ctx* ctx, const gsk_csr* A, const void* x, void* y, int* err, cudaStream_t st) {
  if (A->n == 0) return GSK_OK;
  const int grid = ctx->spmv_grid(A->n);
  if (A->dtype == GSK_F64)
    spmv_kernel<double><<<grid, kBlock, 0, st>>>(A->n, A->nnz, A->rowptr, A->colidx, (const double*)A->val,
                                                  (const double*)x, (double*)y, err);
  else
    spmv_kernel<float><<<grid, kBlock, 0, st>>>(A->n, A->nnz, A->rowptr, A->colidx, (const float*)A->val,
                                                 (const float*)x, (float*)y, err);
  GSK_CK(cudaGetLastError());
  return GSK_OK;
}

gsk_status run_gs_scale(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* d_out, cudaStream_t st,
                        float* kernel_ms) {
  const int n = A->n;
  Arena a;
  a.take<int>(64);  // error word
  gsk_status s = ctx->reserve(a.off);
  if (s != GSK_OK) return s;
  int* err = (int*)ctx->ws;
  GSK_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (kernel_ms) {
    GSK_CK(cudaEventCreate(&ev[0]));
    GSK_CK(cudaEventCreate(&ev[1]));
    GSK_CK(cudaEventRecord(ev[0], st));
  }
  if (A->dtype == GSK_F64)
    launch_gs_rows<double, true>(ctx, 0, n, A->nnz, A->rowptr, (double*)A->val, (double*)b, p, d_out, err, st);
  else
    launch_gs_rows<float, true>(ctx, 0, n, A->nnz, A->rowptr, (float*)A->val, (float*)b, p, d_out, err, st);
  GSK_CK(cudaGetLastError());
  if (kernel_ms) GSK_CK(cudaEventRecord(ev[1], st));
  int* hbits = (int*)ctx->host_pinned;
  GSK_CK(cudaMemcpyAsync(hbits, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  if (kernel_ms) {
    GSK_CK(cudaEventElapsedTime(kernel_ms, ev[0], ev[1]));
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
  }
  return err_bits_status(ctx, *hbits);
}

// ------------------------------------------------ two-sided D^(1/2) scaling
//
// The variant the paper also tried (Sec. 2): with D = diag(1/||a_i||_p),
// solve D^(1/2) A D^(1/2) y = D^(1/2) b and recover x = D^(1/2) y.  gs_norm
// gives d_i = 1/||a_i||_p (and the GS(2) scales when the metric weights are
// wanted), sym_check validates the column indices, and sym_apply scales
// a_ij by s_i s_j only if no error was recorded, so that A and b are left
// untouched on error.

// Column indices must lie in [0, n): the column scale s_j is gathered.
__global__ void __launch_bounds__(kBlock) sym_check_kernel(int nnz, int n, const int* __restrict__ colidx, int* err) {
  for (int k = blockIdx.x * kBlock + threadIdx.x; k < nnz; k += gridDim.x * kBlock)
    if ((unsigned)__ldg(colidx + k) >= (unsigned)n) atomicOr(err, kErrIndex);
}

// s_i = sqrt(d_i); w_i = d2_i / s_i (d2 = d for p = 2, else the GS(2) scales
// already stored in w).
__global__ void __launch_bounds__(kBlock) sym_prep_kernel(int n, const double* __restrict__ d, double* __restrict__ s,
                                                          double* w, int w_is_d) {
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
    const double si = sqrt(d[i]);
    s[i] = si;
    if (w) w[i] = (w_is_d ? d[i] : w[i]) / si;
  }
}

// a_ij <- a_ij s_i s_j, b_i <- b_i s_i; one row per thread.
template <typename T>
__global__ void __launch_bounds__(kBlock) sym_apply_kernel(int n, const int* __restrict__ rowptr,
                                                           const int* __restrict__ colidx, T* __restrict__ val,
                                                           T* __restrict__ b, const double* __restrict__ s,
                                                           const int* err) {
  if (*(volatile const int*)err != 0) return;  // leave A and b as they are
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
    const double si = s[i];
    for (int k = __ldg(rowptr + i); k < __ldg(rowptr + i + 1); ++k)
      val[k] = (T)((double)val[k] * si * __ldg(s + __ldg(colidx + k)));
    if (b) b[i] = (T)((double)b[i] * si);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) diag_mul_kernel(int n, const double* __restrict__ s, T* __restrict__ x) {
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) x[i] = (T)((double)x[i] * s[i]);
}

gsk_status run_gs_scale_sym(gsk_ctx* ctx, gsk_csr* A, void* b, double p, double* s_out, double* w_out,
                            cudaStream_t st) {
  const int pmode = pmode_of(p);
  const int n = A->n;
  Arena a;
  a.take<int>(64);
  a.take<double>(n);
  gsk_status s = ctx->reserve(a.off);
  if (s != GSK_OK) return s;
  a = Arena{(char*)ctx->ws, ctx->ws_bytes, 0};
  int* err = a.take<int>(64);
  double* d = a.take<double>(n);
  GSK_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  const int gt = ctx->grid_for(((long long)n + 31) / 32, kWarpsPerBlock, 8);
  const int gr = ctx->grid_for(n, kBlock, 8);
  const int gn = ctx->grid_for(A->nnz, kBlock, 8);
  const bool w_is_d = pmode == kP2;
  if (A->dtype == GSK_F64) {
    launch_gs_rows<double, false>(ctx, gt, n, A->nnz, A->rowptr, (double*)A->val, (double*)b, p, d, err, st);
    if (w_out && !w_is_d)
      launch_gs_rows<double, false>(ctx, gt, n, A->nnz, A->rowptr, (double*)A->val, nullptr, 2.0, w_out, err, st);
  } else {
    launch_gs_rows<float, false>(ctx, gt, n, A->nnz, A->rowptr, (float*)A->val, (float*)b, p, d, err, st);
    if (w_out && !w_is_d)
      launch_gs_rows<float, false>(ctx, gt, n, A->nnz, A->rowptr, (float*)A->val, nullptr, 2.0, w_out, err, st);
  }
  if (A->nnz > 0) sym_check_kernel<<<gn, kBlock, 0, st>>>(A->nnz, n, A->colidx, err);
  sym_prep_kernel<<<gr, kBlock, 0, st>>>(n, d, s_out, w_out, w_is_d ? 1 : 0);
  if (A->dtype == GSK_F64)
    sym_apply_kernel<double><<<gr, kBlock, 0, st>>>(n, A->rowptr, A->colidx, (double*)A->val, (double*)b, s_out,
                                                     err);
  else
    sym_apply_kernel<float><<<gr, kBlock, 0, st>>>(n, A->rowptr, A->colidx, (float*)A->val, (float*)b, s_out, err);
  GSK_CK(cudaGetLastError());
  int* hbits = (int*)ctx->host_pinned;
  GSK_CK(cudaMemcpyAsync(hbits, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  return err_bits_status(ctx, *hbits);
}

gsk_status launch_diag_mul(gsk_ctx* ctx, int n, const double* s, void* x, gsk_dtype dtype, cudaStream_t st) {
  const int g = ctx->grid_for(n, kBlock, 8);
  if (dtype == GSK_F64) diag_mul_kernel<double><<<g, kBlock, 0, st>>>(n, s, (double*)x);
  else diag_mul_kernel<float><<<g, kBlock, 0, st>>>(n, s, (float*)x);
  GSK_CK(cudaGetLastError());
  return GSK_OK;
}

}  // namespace gsk

// --------------------------------------------------- allocation-free GS(p)
//
// gs_scale_static: GS(p) for callers that must not allocate device memory
// (and so cannot create a gsk_ctx, whose workspace is allocated).  It runs
// the two-pass form -- every row's scale and check first, the scaling only if
// no row failed -- with the per-row arithmetic of gs_scale, so on valid input
// the two give bit-identical results.  Its scratch -- the error word and,
// when the caller passes no d_out, the per-row scales -- lives in the
// file-scope array below, which every device that loads the library holds
// until the process exits.
namespace gsk {
namespace {
constexpr int kStaticMaxRows = 1 << 20;  // rows whose scales fit in the array
constexpr size_t kStaticHeader = 256;    // error word (padded)
constexpr size_t kStaticBytes = kStaticHeader + sizeof(double) * (size_t)kStaticMaxRows;  // 8 MiB + 256 B
constexpr int kStaticMaxDevices = 64;

struct StaticDevice {
  void* scratch;  // device address of g_gs_static_scratch on this device
  int sms;
  bool ready;
};
StaticDevice g_static_dev[kStaticMaxDevices];
std::mutex g_static_mu;
}  // namespace

static __device__ __align__(256) unsigned char g_gs_static_scratch[kStaticBytes];

// Once per device, with that device current: look up the array's device
// address (host code cannot use the symbol itself) and the SM count.
static gsk_status static_setup(int dev, StaticDevice** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticDevice& d = g_static_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gs_static_scratch) != cudaSuccess || p == nullptr) return GSK_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return GSK_ERR_CUDA;
    d.scratch = p;
    d.sms = sms;
    d.ready = true;
  }
  *out = &d;
  return GSK_OK;
}

}  // namespace gsk

extern "C" gsk_status gs_scale_static(gsk_csr* A, void* b, double p, double* d_out, void* stream) {
  using namespace gsk;
  if (!A || A->n < 0 || A->nnz < 0) return GSK_ERR_ARG;
  if (A->n > 0 && (!A->rowptr || (A->nnz > 0 && !A->val))) return GSK_ERR_ARG;
  if (A->dtype != GSK_F64 && A->dtype != GSK_F32) return GSK_ERR_ARG;
  if (!(p >= 1.0)) return GSK_ERR_ARG;
  if (!d_out && A->n > kStaticMaxRows) return GSK_ERR_ARG;  // the scales would not fit
  if (A->n == 0) return GSK_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GSK_ERR_CUDA;
  if (dev < 0 || dev >= kStaticMaxDevices) return GSK_ERR_ARG;
  StaticDevice* sd = nullptr;
  gsk_status s = static_setup(dev, &sd);
  if (s != GSK_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = (int*)sd->scratch;
  double* d = d_out ? d_out : (double*)((char*)sd->scratch + kStaticHeader);
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return GSK_ERR_CUDA;  // left set by the last call
  const long long g = (((long long)A->n + 31) / 32 + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int grid = (int)(g < (long long)sd->sms * 8 ? (g < 1 ? 1 : g) : (long long)sd->sms * 8);
  const int n = A->n;
  if (A->dtype == GSK_F64) {
    launch_gs_rows<double, false>(nullptr, grid, n, A->nnz, A->rowptr, (double*)A->val, (double*)b, p, d, err, st);
    gs_apply_kernel<double><<<grid, kBlock, 0, st>>>(n, A->nnz, A->rowptr, (double*)A->val, (double*)b, d, err);
  } else {
    launch_gs_rows<float, false>(nullptr, grid, n, A->nnz, A->rowptr, (float*)A->val, (float*)b, p, d, err, st);
    gs_apply_kernel<float><<<grid, kBlock, 0, st>>>(n, A->nnz, A->rowptr, (float*)A->val, (float*)b, d, err);
  }
  if (cudaGetLastError() != cudaSuccess) return GSK_ERR_CUDA;
  int bits = 0;
  if (cudaMemcpyAsync(&bits, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return GSK_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GSK_ERR_CUDA;
  if (bits & kErrIndex) return GSK_ERR_ARG;
  if (bits & kErrNonFinite) return GSK_ERR_NONFINITE;
  if (bits & kErrZeroRow) return GSK_ERR_ZERO_ROW;
  return GSK_OK;
}

