// ILU(0) preconditioner (Sec. 2: the paper's ILUT with drop tolerance 0 and
// fill-in 1 acted as ILU(0)): level schedule on the host, factorisation and
// triangular solves on the device.  See ilu.cuh for the kernel design.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ilu.cuh"

namespace gsk {

// Factor rows level by level: for row i and each k < i in its pattern,
// l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for j > k in both rows (the two
// column lists are sorted, so one merge finds the common j).
__global__ void __launch_bounds__(kIluBlock) ilu_factor_kernel(IluArgs a, double* lu) {
  const int nthreads = gridDim.x * kIluBlock;
  const int tid = blockIdx.x * kIluBlock + threadIdx.x;
  for (int lev = 0; lev < a.nlevL; ++lev) {
    const int l0 = a.lptrL[lev], cnt = a.lptrL[lev + 1] - l0;
    for (int t = tid; t < cnt; t += nthreads) {
      const int i = a.orderL[l0 + t];
      const int rs = a.rowptr[i], re = a.rowptr[i + 1], di = a.dpos[i];
      for (int kk = rs; kk < di; ++kk) {
        const int k = a.colidx[kk];
        const int dk = a.dpos[k], ke = a.rowptr[k + 1];
        const double ukk = __ldcg(lu + dk);
        if (ukk == 0.0 || !isfinite(ukk)) {
          atomicOr(a.err, kErrZeroRow);
          continue;
        }
        const double lik = lu[kk] / ukk;
        lu[kk] = lik;
        // merge row i's entries after kk with row k's entries after its diagonal
        int q = dk + 1;
        for (int jj = kk + 1; jj < re; ++jj) {
          const int j = a.colidx[jj];
          while (q < ke && a.colidx[q] < j) ++q;
          if (q < ke && a.colidx[q] == j) lu[jj] = fma(-lik, __ldcg(lu + q), lu[jj]);
        }
      }
      const double uii = lu[di];
      if (uii == 0.0 || !isfinite(uii)) atomicOr(a.err, kErrZeroRow);
    }
    if (lev + 1 < a.nlevL) ilu_barrier(a.bar, (unsigned)lev, a.err);
  }
}

// A row of a sweep with its index data loaded ahead of the level: the row,
// the range [k0, k1) of its entries in the sweep's triangle, the first
// kIluPre of those (column, factor entry) and, backward, the pivot.  None of
// it depends on z, so a thread loads the next level's row while it works on
// the current one and waits at the barrier; after the barrier only the loads
// of z remain on the level's critical path (a level's cost was its chain of
// dependent loads: level pointer, row, columns, z).
constexpr int kIluPre = 4;
struct IluRow {
  int i, k0, k1, cnt;  // cnt: rows in the level
  int col[kIluPre];
  double val[kIluPre];
  double pivot;
};

__device__ __forceinline__ IluRow ilu_fetch(const IluArgs& a, bool upper, int lev, int tid) {
  IluRow w;
  w.i = -1;
  w.k0 = w.k1 = w.cnt = 0;
  w.pivot = 1.0;
  const int* lptr = upper ? a.lptrU : a.lptrL;
  if (lev >= (upper ? a.nlevU : a.nlevL)) return w;
  const int l0 = lptr[lev];
  w.cnt = lptr[lev + 1] - l0;
  if (tid >= w.cnt) return w;
  const int i = (upper ? a.orderU : a.orderL)[l0 + tid];
  const int di = a.dpos[i];
  w.i = i;
  w.k0 = upper ? di + 1 : a.rowptr[i];
  w.k1 = upper ? a.rowptr[i + 1] : di;
  if (upper) w.pivot = a.lu[di];
#pragma unroll
  for (int q = 0; q < kIluPre; ++q) {
    const int k = w.k0 + q;
    w.col[q] = k < w.k1 ? a.colidx[k] : 0;
    w.val[q] = k < w.k1 ? a.lu[k] : 0.0;
  }
  return w;
}

// Forward: y_i = r_i - sum_{k<i} l_ik y_k; backward: z_i = (y_i - sum_{j>i}
// u_ij z_j) / u_ii; the entries in ascending column order either way.
__device__ __forceinline__ void ilu_row(const IluArgs& a, bool upper, const IluRow& w, const double* r, double* z) {
  double s = upper ? __ldcg(z + w.i) : r[w.i];
  const int np = min(w.k1 - w.k0, kIluPre);
#pragma unroll
  for (int q = 0; q < kIluPre; ++q)
    if (q < np) s = fma(-w.val[q], __ldcg(z + w.col[q]), s);
  for (int k = w.k0 + kIluPre; k < w.k1; ++k) s = fma(-a.lu[k], __ldcg(z + a.colidx[k]), s);
  z[w.i] = upper ? s / w.pivot : s;
}

__global__ void __launch_bounds__(kIluBlock) ilu_solve_kernel(IluArgs a) {
  if (ilu_gate_closed(a.gate)) return;  // the same decision in every block
  const double* r = a.gate.base + (a.gate.col ? (long long)(*a.gate.col) * a.gate.stride : 0ll);
  double* z = a.z;
  const int nthreads = gridDim.x * kIluBlock;
  const int tid = blockIdx.x * kIluBlock + threadIdx.x;
  unsigned nb = 0;
  // levels wider than the grid: the rows after a thread's first one are
  // fetched when they are processed
  auto rest = [&](bool upper, int lev, int cnt) {
    for (int t = tid + nthreads; t < cnt; t += nthreads) ilu_row(a, upper, ilu_fetch(a, upper, lev, t), r, z);
  };
  IluRow cur = ilu_fetch(a, false, 0, tid);
  for (int lev = 0; lev < a.nlevL; ++lev) {
    const IluRow nxt = lev + 1 < a.nlevL ? ilu_fetch(a, false, lev + 1, tid) : ilu_fetch(a, true, 0, tid);
    if (cur.i >= 0) ilu_row(a, false, cur, r, z);
    rest(false, lev, cur.cnt);
    ilu_barrier(a.bar, nb++, a.err);
    cur = nxt;
  }
  for (int lev = 0; lev < a.nlevU; ++lev) {
    const IluRow nxt = ilu_fetch(a, true, lev + 1, tid);
    if (cur.i >= 0) ilu_row(a, true, cur, r, z);
    rest(true, lev, cur.cnt);
    if (lev + 1 < a.nlevU) ilu_barrier(a.bar, nb++, a.err);
    cur = nxt;
  }
}

IluArgs ilu_args(const gsk_ilu0* h, const IluGate& gate, double* z) {
  IluArgs a;
  a.n = h->n;
  a.rowptr = h->rowptr;
  a.colidx = h->colidx;
  a.lu = h->lu;
  a.dpos = h->dpos;
  a.orderL = h->orderL;
  a.lptrL = h->lptrL;
  a.orderU = h->orderU;
  a.lptrU = h->lptrU;
  a.nlevL = h->nlevL;
  a.nlevU = h->nlevU;
  a.bar = h->bar;
  a.err = h->err;
  a.gate = gate;
  a.z = z;
  return a;
}

// One application on `st` (capturable): clear the barrier counter, then the
// cooperative sweep kernel.
gsk_status ilu_launch_apply(gsk_ctx* ctx, const gsk_ilu0* h, const IluGate& gate, double* z, cudaStream_t st) {
  IluArgs a = ilu_args(h, gate, z);
  GSK_CK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st));
  void* params[] = {&a};
  GSK_CK(cudaLaunchCooperativeKernel((const void*)ilu_solve_kernel, dim3(h->grid), dim3(kIluBlock), params, 0, st));
  return GSK_OK;
}

gsk_status ilu_read_err(gsk_ctx* ctx, const gsk_ilu0* h, cudaStream_t st) {
  int* hb = (int*)ctx->host_pinned;
  GSK_CK(cudaMemcpyAsync(hb, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  return err_bits_status(ctx, *hb);
}

}  // namespace gsk

using namespace gsk;

extern "C" gsk_status gsk_ilu0_create(gsk_ctx* ctx, const gsk_csr* A, gsk_ilu0** out, void* stream) {
  if (!ctx || !out) return GSK_ERR_ARG;
  *out = nullptr;
  gsk_status s = check_csr(ctx, A);
  if (s != GSK_OK) return s;
  if (A->dtype != GSK_F64) return ctx->fail(GSK_ERR_ARG, "ILU(0) needs an FP64 matrix");
  if (A->n == 0 || !A->colidx) return ctx->fail(GSK_ERR_ARG, "empty matrix or NULL colidx");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = A->n, nnz = A->nnz;
  // structure to the host; diagonal positions, checks and the level sets
  std::vector<int> rp(n + 1), ci(nnz);
  GSK_CK(cudaMemcpyAsync(rp.data(), A->rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, st));
  if (nnz) GSK_CK(cudaMemcpyAsync(ci.data(), A->colidx, sizeof(int) * nnz, cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  std::vector<int> dpos(n), levL(n, 0), levU(n, 0);
  int nlevL = 0, nlevU = 0;
  for (int i = 0; i < n; ++i) {
    if (rp[i] < 0 || rp[i + 1] < rp[i] || rp[i + 1] > nnz) return ctx->fail(GSK_ERR_ARG, "malformed rowptr");
    int d = -1, lv = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = ci[k];
      if (j < 0 || j >= n) return ctx->fail(GSK_ERR_ARG, "column index out of range");
      if (k > rp[i] && j <= ci[k - 1]) return ctx->fail(GSK_ERR_ARG, "columns must be sorted within a row");
      if (j == i) d = k;
      if (j < i && levL[j] + 1 > lv) lv = levL[j] + 1;
    }
    if (d < 0) return ctx->fail(GSK_ERR_ARG, "a row has no diagonal entry");
    dpos[i] = d;
    levL[i] = lv;
    if (lv + 1 > nlevL) nlevL = lv + 1;
  }
  for (int i = n - 1; i >= 0; --i) {
    int lv = 0;
    for (int k = dpos[i] + 1; k < rp[i + 1]; ++k)
      if (levU[ci[k]] + 1 > lv) lv = levU[ci[k]] + 1;
    levU[i] = lv;
    if (lv + 1 > nlevU) nlevU = lv + 1;
  }
  auto order_by = [&](const std::vector<int>& lev, int nlev, std::vector<int>& order, std::vector<int>& ptr) {
    ptr.assign(nlev + 1, 0);
    for (int i = 0; i < n; ++i) ptr[lev[i] + 1]++;
    for (int l = 0; l < nlev; ++l) ptr[l + 1] += ptr[l];
    order.assign(n, 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int i = 0; i < n; ++i) order[fill[lev[i]]++] = i;
  };
  std::vector<int> orderL, lptrL, orderU, lptrU;
  order_by(levL, nlevL, orderL, lptrL);
  order_by(levU, nlevU, orderU, lptrU);

  gsk_ilu0* h = new (std::nothrow) gsk_ilu0();
  if (!h) return ctx->fail(GSK_ERR_OOM, "host allocation failed");
  static std::atomic<unsigned long long> next_serial{1};
  h->serial = next_serial.fetch_add(1);
  h->device = ctx->device;
  h->n = n;
  h->nnz = nnz;
  h->rowptr = A->rowptr;
  h->colidx = A->colidx;
  h->nlevL = nlevL;
  h->nlevU = nlevU;
  Arena sz;
  sz.take<unsigned>(64);
  sz.take<int>(64);
  sz.take<double>(nnz);
  sz.take<int>(n);
  sz.take<int>(n);
  sz.take<int>(nlevL + 1);
  sz.take<int>(n);
  sz.take<int>(nlevU + 1);
  if (cudaMalloc(&h->mem, sz.off) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return ctx->fail(GSK_ERR_OOM, "cudaMalloc of the ILU(0) factors failed");
  }
  Arena ar{(char*)h->mem, sz.off, 0};
  h->bar = ar.take<unsigned>(64);
  h->err = ar.take<int>(64);
  h->lu = ar.take<double>(nnz);
  h->dpos = ar.take<int>(n);
  h->orderL = ar.take<int>(n);
  h->lptrL = ar.take<int>(nlevL + 1);
  h->orderU = ar.take<int>(n);
  h->lptrU = ar.take<int>(nlevU + 1);
  auto fail = [&](cudaError_t e, const char* what) {
    gsk_status r = ctx->cuda_fail(e, what);
    cudaFree(h->mem);
    delete h;
    return r;
  };
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  up(h->dpos, dpos.data(), sizeof(int) * n);
  up(h->orderL, orderL.data(), sizeof(int) * n);
  up(h->lptrL, lptrL.data(), sizeof(int) * (nlevL + 1));
  up(h->orderU, orderU.data(), sizeof(int) * n);
  up(h->lptrU, lptrU.data(), sizeof(int) * (nlevU + 1));
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(h->lu, A->val, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return fail(e, "ILU(0) upload");
  // cooperative grid: co-resident blocks, at most one per SM (a cheap barrier)
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)ilu_factor_kernel, kIluBlock, 0);
  int per_sm2 = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, (const void*)ilu_solve_kernel, kIluBlock, 0);
  if (e != cudaSuccess || per_sm < 1 || per_sm2 < 1) return fail(e == cudaSuccess ? cudaErrorInvalidValue : e, "occupancy");
  h->grid = ctx->num_sms;
  IluGate none = {};
  IluArgs a = ilu_args(h, none, nullptr);
  double* lu = h->lu;
  void* params[] = {&a, &lu};
  e = cudaLaunchCooperativeKernel((const void*)ilu_factor_kernel, dim3(h->grid), dim3(kIluBlock), params, 0, st);
  if (e != cudaSuccess) return fail(e, "ILU(0) factorisation launch");
  gsk_status rs = ilu_read_err(ctx, h, st);
  if (rs != GSK_OK) {
    cudaFree(h->mem);
    delete h;
    return rs;
  }
  *out = h;
  return GSK_OK;
}

extern "C" gsk_status gsk_ilu0_destroy(gsk_ilu0* h) {
  if (!h) return GSK_OK;
  cudaSetDevice(h->device);
  cudaFree(h->mem);
  delete h;
  return GSK_OK;
}

extern "C" gsk_status gsk_ilu0_apply(gsk_ctx* ctx, const gsk_ilu0* h, const double* r, double* z, void* stream) {
  if (!ctx || !h || !r || !z || r == z) return ctx ? ctx->fail(GSK_ERR_ARG, "bad ILU(0) apply arguments") : GSK_ERR_ARG;
  IluGate g = {};
  g.base = r;
  return ilu_launch_apply(ctx, h, g, z, (cudaStream_t)stream);
}
