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

__global__ void __launch_bounds__(kIluBlock) ilu_solve_kernel(IluArgs a) {
  if (ilu_gate_closed(a.gate)) return;  // the same decision in every block
  const double* r = a.gate.base + (a.gate.col ? (long long)(*a.gate.col) * a.gate.stride : 0ll);
  double* z = a.z;
  const int nthreads = gridDim.x * kIluBlock;
  const int tid = blockIdx.x * kIluBlock + threadIdx.x;
  unsigned nb = 0;
  // forward: y_i = r_i - sum_{k<i} l_ik y_k
  for (int lev = 0; lev < a.nlevL; ++lev) {
    const int l0 = a.lptrL[lev], cnt = a.lptrL[lev + 1] - l0;
    for (int t = tid; t < cnt; t += nthreads) {
      const int i = a.orderL[l0 + t];
      double s = r[i];
      for (int k = a.rowptr[i]; k < a.dpos[i]; ++k) s = fma(-a.lu[k], __ldcg(z + a.colidx[k]), s);
      z[i] = s;
    }
    ilu_barrier(a.bar, nb++, a.err);
  }
  // backward: z_i = (y_i - sum_{j>i} u_ij z_j) / u_ii
  for (int lev = 0; lev < a.nlevU; ++lev) {
    const int l0 = a.lptrU[lev], cnt = a.lptrU[lev + 1] - l0;
    for (int t = tid; t < cnt; t += nthreads) {
      const int i = a.orderU[l0 + t];
      const int di = a.dpos[i];
      double s = __ldcg(z + i);
      for (int k = di + 1; k < a.rowptr[i + 1]; ++k) s = fma(-a.lu[k], __ldcg(z + a.colidx[k]), s);
      z[i] = s / a.lu[di];
    }
    if (lev + 1 < a.nlevU) ilu_barrier(a.bar, nb++, a.err);
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
