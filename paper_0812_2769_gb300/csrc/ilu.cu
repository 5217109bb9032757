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

// A level-ordered row of the one-CTA sweep, loaded ahead (every address
// follows from its position p alone).
struct IluPRow {
  int i, k0, k1;
  int col[kIluPack];
  double val[kIluPack];
  double piv;
};

__device__ __forceinline__ IluPRow ilu_pfetch(const IluPackedSweep& P, int p, bool upper) {
  IluPRow w;
  w.i = P.row[p];
  w.k0 = P.k0[p];
  w.k1 = P.k1[p];
#pragma unroll
  for (int q = 0; q < kIluPack; ++q) {
    w.col[q] = P.col[kIluPack * p + q];
    w.val[q] = P.val[kIluPack * p + q];
  }
  w.piv = upper ? P.piv[p] : 1.0;
  return w;
}

// The row of ilu_row with z in shared memory: the same FMAs in the same order.
__device__ __forceinline__ void ilu_prow(const IluArgs& a, bool upper, const IluPRow& w, double* zs) {
  double s = zs[w.i];
  const int np = min(w.k1 - w.k0, kIluPack);
#pragma unroll
  for (int q = 0; q < kIluPack; ++q)
    if (q < np) s = fma(-w.val[q], zs[w.col[q]], s);
  for (int k = w.k0 + kIluPack; k < w.k1; ++k) s = fma(-a.lu[k], zs[a.colidx[k]], s);
  zs[w.i] = upper ? s / w.piv : s;
}

__global__ void __launch_bounds__(kIluSBlock) ilu_solve_smem(IluArgs a, IluPackedSweep L, IluPackedSweep U) {
  if (ilu_gate_closed(a.gate)) return;
  extern __shared__ double zs[];  // [n] z, then the level pointers of both sweeps
  int* lp = reinterpret_cast<int*>(zs + a.n);
  const double* r = a.gate.base + (a.gate.col ? (long long)(*a.gate.col) * a.gate.stride : 0ll);
  const int t = threadIdx.x;
  for (int i = t; i < a.n; i += kIluSBlock) zs[i] = r[i];
  for (int q = t; q <= a.nlevL; q += kIluSBlock) lp[q] = a.lptrL[q];
  for (int q = t; q <= a.nlevU; q += kIluSBlock) lp[a.nlevL + 1 + q] = a.lptrU[q];
  __syncthreads();
  for (int sw = 0; sw < 2; ++sw) {
    const bool upper = sw == 1;
    const IluPackedSweep& P = upper ? U : L;
    const int* lev = upper ? lp + a.nlevL + 1 : lp;
    const int nlev = upper ? a.nlevU : a.nlevL;
    bool have = lev[0] + t < lev[1];
    IluPRow cur = have ? ilu_pfetch(P, lev[0] + t, upper) : IluPRow{};
    for (int l = 0; l < nlev; ++l) {
      const bool have_next = l + 1 < nlev && lev[l + 1] + t < lev[l + 2];
      const IluPRow nxt = have_next ? ilu_pfetch(P, lev[l + 1] + t, upper) : IluPRow{};
      if (have) ilu_prow(a, upper, cur, zs);
      for (int p = lev[l] + t + kIluSBlock; p < lev[l + 1]; p += kIluSBlock)
        ilu_prow(a, upper, ilu_pfetch(P, p, upper), zs);
      __syncthreads();
      cur = nxt;
      have = have_next;
    }
  }
  for (int i = t; i < a.n; i += kIluSBlock) a.z[i] = zs[i];
}

// dst[t] = lu[src[t]] (0 where src[t] < 0): the packed factor entries, taken
// once after the factorisation.
__global__ void ilu_gather_kernel(int count, const int* src, const double* lu, double* dst) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x)
    dst[t] = src[t] >= 0 ? lu[src[t]] : 0.0;
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
  if (h->smem_bytes > 0) {
    const IluPackedSweep L = {h->prowL, h->pk0L, h->pk1L, h->pcolL, h->pvalL, nullptr};
    const IluPackedSweep U = {h->prowU, h->pk0U, h->pk1U, h->pcolU, h->pvalU, h->ppiv};
    ilu_solve_smem<<<1, kIluSBlock, h->smem_bytes, st>>>(a, L, U);
    GSK_CK(cudaGetLastError());
    return GSK_OK;
  }
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

// The one-CTA sweep's data, when z and the level pointers of both sweeps fit
// in one CTA's shared memory (GSK_ILU_SWEEP=grid keeps the grid sweep): the
// rows in level order, their triangle's entry range, the first kIluPack
// columns and (gathered from the factors just computed) entries, the pivots.
// Any failure here leaves the handle on the grid sweep.
static void ilu_pack_small(gsk_ctx* ctx, gsk_ilu0* h, const std::vector<int>& rp, const std::vector<int>& ci,
                           const std::vector<int>& dpos, const std::vector<int>& orderL,
                           const std::vector<int>& orderU, cudaStream_t st) {
  const int n = h->n;
  const char* sweep = std::getenv("GSK_ILU_SWEEP");
  if (sweep && std::strcmp(sweep, "grid") == 0) return;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const size_t sbytes = sizeof(double) * (size_t)n + sizeof(int) * (size_t)(h->nlevL + 1 + h->nlevU + 1);
  if (sbytes + 1024 > (size_t)optin) return;
  std::vector<int> row[2], k0[2], k1[2], col[2], src[2], psrc(n);
  for (int sw = 0; sw < 2; ++sw) {
    const std::vector<int>& order = sw ? orderU : orderL;
    row[sw].resize(n);
    k0[sw].resize(n);
    k1[sw].resize(n);
    col[sw].assign((size_t)kIluPack * n, 0);
    src[sw].assign((size_t)kIluPack * n, -1);
    for (int p = 0; p < n; ++p) {
      const int i = order[p];
      const int a0 = sw ? dpos[i] + 1 : rp[i], a1 = sw ? rp[i + 1] : dpos[i];
      row[sw][p] = i;
      k0[sw][p] = a0;
      k1[sw][p] = a1;
      for (int q = 0; q < kIluPack && a0 + q < a1; ++q) {
        col[sw][(size_t)kIluPack * p + q] = ci[a0 + q];
        src[sw][(size_t)kIluPack * p + q] = a0 + q;
      }
      if (sw) psrc[p] = dpos[i];
    }
  }
  Arena sz;
  for (int sw = 0; sw < 2; ++sw) {
    sz.take<int>(n);
    sz.take<int>(n);
    sz.take<int>(n);
    sz.take<int>((size_t)kIluPack * n);
    sz.take<int>((size_t)kIluPack * n);
    sz.take<double>((size_t)kIluPack * n);
  }
  sz.take<int>(n);
  sz.take<double>(n);
  void* mem = nullptr;
  if (cudaMalloc(&mem, sz.off) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  Arena ar{(char*)mem, sz.off, 0};
  int *prow[2], *pk0[2], *pk1[2], *pcol[2], *psr[2];
  double* pval[2];
  for (int sw = 0; sw < 2; ++sw) {
    prow[sw] = ar.take<int>(n);
    pk0[sw] = ar.take<int>(n);
    pk1[sw] = ar.take<int>(n);
    pcol[sw] = ar.take<int>((size_t)kIluPack * n);
    psr[sw] = ar.take<int>((size_t)kIluPack * n);
    pval[sw] = ar.take<double>((size_t)kIluPack * n);
  }
  int* ppsrc = ar.take<int>(n);
  double* ppiv = ar.take<double>(n);
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* s, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, s, bytes, cudaMemcpyHostToDevice, st);
  };
  for (int sw = 0; sw < 2; ++sw) {
    up(prow[sw], row[sw].data(), sizeof(int) * n);
    up(pk0[sw], k0[sw].data(), sizeof(int) * n);
    up(pk1[sw], k1[sw].data(), sizeof(int) * n);
    up(pcol[sw], col[sw].data(), sizeof(int) * kIluPack * (size_t)n);
    up(psr[sw], src[sw].data(), sizeof(int) * kIluPack * (size_t)n);
  }
  up(ppsrc, psrc.data(), sizeof(int) * n);
  const int gg = ctx->grid_for((long long)kIluPack * n, 256, 8);
  if (e == cudaSuccess) {
    for (int sw = 0; sw < 2; ++sw) ilu_gather_kernel<<<gg, 256, 0, st>>>(kIluPack * n, psr[sw], h->lu, pval[sw]);
    ilu_gather_kernel<<<gg, 256, 0, st>>>(n, ppsrc, h->lu, ppiv);
    e = cudaGetLastError();
  }
  // the attribute belongs to the kernel, not the handle: allow the device's
  // maximum once, so that every handle's launch fits whatever its size
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)ilu_solve_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(mem);
    return;
  }
  h->pmem = mem;
  h->prowL = prow[0];
  h->pk0L = pk0[0];
  h->pk1L = pk1[0];
  h->pcolL = pcol[0];
  h->psrcL = psr[0];
  h->pvalL = pval[0];
  h->prowU = prow[1];
  h->pk0U = pk0[1];
  h->pk1U = pk1[1];
  h->pcolU = pcol[1];
  h->psrcU = psr[1];
  h->pvalU = pval[1];
  h->ppsrc = ppsrc;
  h->ppiv = ppiv;
  h->smem_bytes = (int)sbytes;
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
  ilu_pack_small(ctx, h, rp, ci, dpos, orderL, orderU, st);
  *out = h;
  return GSK_OK;
}

extern "C" gsk_status gsk_ilu0_info(const gsk_ilu0* h, int* levels_lower, int* levels_upper, int* one_block) {
  if (!h) return GSK_ERR_ARG;
  if (levels_lower) *levels_lower = h->nlevL;
  if (levels_upper) *levels_upper = h->nlevU;
  if (one_block) *one_block = h->smem_bytes > 0 ? 1 : 0;
  return GSK_OK;
}

extern "C" gsk_status gsk_ilu0_destroy(gsk_ilu0* h) {
  if (!h) return GSK_OK;
  cudaSetDevice(h->device);
  cudaFree(h->mem);
  if (h->pmem) cudaFree(h->pmem);
  delete h;
  return GSK_OK;
}

extern "C" gsk_status gsk_ilu0_apply(gsk_ctx* ctx, const gsk_ilu0* h, const double* r, double* z, void* stream) {
  if (!ctx || !h || !r || !z || r == z) return ctx ? ctx->fail(GSK_ERR_ARG, "bad ILU(0) apply arguments") : GSK_ERR_ARG;
  IluGate g = {};
  g.base = r;
  return ilu_launch_apply(ctx, h, g, z, (cudaStream_t)stream);
}
