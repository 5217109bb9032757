// Batched persistent solver: many independent sparse systems in one launch.
//
// Each thread block takes the next system from an atomic work queue (systems
// ordered largest first, so the tail of the batch is made of small ones),
// applies GS(p) to it in place (Sec. 2, Eq. (2)), solves it with Bi-CGSTAB
// (Sec. 2) using only block-level reductions, writes x and the outcome, and
// takes the next system.  There is no grid-wide synchronisation and no
// waiting on other blocks.  A system's arithmetic depends only on the system
// and the block size, so its result is bit-identical alone and in any batch.
//
// GMRES(m) (FP64, batch_gmres) runs the same way, one block per system, with
// the basis in the block's slot memory.
// The block size (128, 256 or 512 threads) is a template parameter chosen
// per call (gsk_opts.batch_block, picked by the autotuner).
//
// Two precisions (template MIXED):
//   FP64   Bi-CGSTAB as bicgstab_solve: recursive residual, true-residual
//          confirmation and up to `refresh` restarts, breakdown tests.
//   mixed  FP64 refinement around FP32 Bi-CGSTAB solves of (W2 A)_32 d =
//          W2 r / ||W2 r|| to a relative tolerance inner_tol (W2 = GS(2)
//          scales of the scaled matrix), x += ||W2 r|| d, as mixed.cu.  A
//          system on which one refinement step gains less than 10x in the FP64
//          metric (FP32 too coarse for its conditioning) is finished in FP64
//          from its current x.
// Per-block scratch vectors live in global memory (L2-resident while the
// block works on its system).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <numeric>

#include "internal.hpp"

namespace gsk {

// mixed precision: FP32 iterations per refinement step when inner_maxit is 0
// (short inner solves let the FP64 refinement and the escalation test act
// early on systems whose conditioning is too much for FP32)
constexpr int kBatchInnerMaxit = 40;

struct BatchSys {
  int n, nnz;
  const int* rowptr;
  const int* colidx;
  double* val;
  double* b;
  double* x;
  double p;  // GS(p) applied first; NaN = none
};

struct BatchOut {
  int iters, restarts, refreshes, refinements, conv, status;
  double relres_true, relres_rec;
};

struct BatchParams {
  const BatchSys* sys;
  const int* order;
  const int* mvec;  // GMRES: restart length per system
  int nsys;
  unsigned* queue;
  BatchOut* out;
  char* scratch;
  long long slot_bytes;
  double tol, inner_tol, brk;
  int maxit, refresh, inner_maxit, metric_plain;
};

template <int NV, int BS>
__device__ __forceinline__ void bsum(const double (&v)[NV], double* sm, double* res) {
  block_sum_tree<NV, BS>(v, sm, res);
}

// y = A x for one system, thread per row; bad indices flag *err.
template <int BS, typename T>
__device__ __forceinline__ void block_spmv(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                           const T* __restrict__ val, const T* __restrict__ x, T* __restrict__ y,
                                           int* err) {
  using Acc = typename AccOf<T>::type;
  for (int i = threadIdx.x; i < n; i += BS) {
    const int rs = rowptr[i], re = rowptr[i + 1];
    Acc sum = Acc(0);
    for (int k = rs; k < re; ++k) {
      const int c = colidx[k];
      if ((unsigned)c < (unsigned)n) sum = fma((Acc)val[k], (Acc)x[c], sum);
      else *err = 1;
    }
    y[i] = (T)sum;
  }
}

// Bi-CGSTAB on one system, block-local.  x holds the initial guess on entry.
// confirm: FP64 mode (true residual check and refresh); otherwise an inner
// solve stopped by the recursive residual relative to ||rhs||.
// restart_on_breakdown (used only when a mixed-precision system is finished
// in FP64): a breakdown restarts from the true residual while refreshes are
// left, instead of ending the solve.
template <int BS, typename T>
__device__ void block_bicgstab(int n, const int* rowptr, const int* colidx, const T* val, const T* rhs, T* x,
                               T* r, T* rh, T* p, T* v, T* s, T* t, const double* w, double tol, int maxit,
                               int refresh, bool confirm, double brk, double* sm, int* err, BatchOut& o,
                               bool restart_on_breakdown = false) {
  using Acc = typename AccOf<T>::type;
  __shared__ double res[4];
  const bool wid = (w == nullptr);
  // r = rhs - A x
  block_spmv<BS>(n, rowptr, colidx, val, x, t, err);
  __syncthreads();
  double acc2[2] = {0.0, 0.0};
  {
    Acc a0 = 0, a1 = 0;
    for (int i = threadIdx.x; i < n; i += BS) {
      const T ri = (T)((Acc)rhs[i] - (Acc)t[i]);
      r[i] = ri;
      rh[i] = ri;
      p[i] = ri;
      const Acc wr = (Acc)(wid ? 1.0 : w[i]) * (Acc)ri;
      a0 = fma(wr, wr, a0);
      a1 = fma((Acc)ri, (Acc)ri, a1);
    }
    acc2[0] = a0;
    acc2[1] = a1;
  }
  bsum<2, BS>(acc2, sm, res);
  const double mu0 = sqrt(res[0]);
  double rho = res[1], rhn = sqrt(res[1]);
  o.iters = 0;
  o.refreshes = 0;
  o.relres_rec = 1.0;
  o.relres_true = 1.0;
  o.conv = GSK_MAXIT;
  if (!(mu0 > 0.0)) {
    if (mu0 == 0.0) {
      o.conv = GSK_CONVERGED;
      o.relres_true = o.relres_rec = 0.0;
    }
    return;
  }
  int refresh_left = refresh;
  bool broke = false;
#define BCG_BREAKDOWN                                  \
  {                                                    \
    if (restart_on_breakdown && refresh_left > 0) {    \
      broke = true;                                    \
      check_true = true;                               \
      break;                                           \
    }                                                  \
    o.conv = GSK_BREAKDOWN;                            \
    goto done;                                         \
  }
  for (;;) {
    bool check_true = false;
    broke = false;
    while (!check_true) {
      if (o.iters >= maxit) {
        o.conv = GSK_MAXIT;
        goto done;
      }
      block_spmv<BS>(n, rowptr, colidx, val, p, v, err);
      __syncthreads();
      {
        Acc a0 = 0, a1 = 0;
        for (int i = threadIdx.x; i < n; i += BS) {
          a0 = fma((Acc)rh[i], (Acc)v[i], a0);
          a1 = fma((Acc)v[i], (Acc)v[i], a1);
        }
        double ad[2] = {(double)a0, (double)a1};
        bsum<2, BS>(ad, sm, res);
      }
      const double sigma = res[0], vn = sqrt(res[1]);
      if (!(fabs(sigma) > brk * rhn * vn)) BCG_BREAKDOWN
      const double alpha = rho / sigma;
      {
        Acc a0 = 0;
        for (int i = threadIdx.x; i < n; i += BS) {
          const T si = (T)fma(-(Acc)alpha, (Acc)v[i], (Acc)r[i]);
          s[i] = si;
          const Acc ws = (Acc)(wid ? 1.0 : w[i]) * (Acc)si;
          a0 = fma(ws, ws, a0);
        }
        double ad[1] = {(double)a0};
        bsum<1, BS>(ad, sm, res);
      }
      const double mus = sqrt(res[0]) / mu0;
      if (mus < tol) {
        for (int i = threadIdx.x; i < n; i += BS) x[i] = (T)fma((Acc)alpha, (Acc)p[i], (Acc)x[i]);
        o.iters += 1;
        o.relres_rec = mus;
        check_true = true;
        break;
      }
      block_spmv<BS>(n, rowptr, colidx, val, s, t, err);
      __syncthreads();
      {
        Acc a0 = 0, a1 = 0;
        for (int i = threadIdx.x; i < n; i += BS) {
          a0 = fma((Acc)t[i], (Acc)s[i], a0);
          a1 = fma((Acc)t[i], (Acc)t[i], a1);
        }
        double ad[2] = {(double)a0, (double)a1};
        bsum<2, BS>(ad, sm, res);
      }
      if (!(res[1] > 0.0)) BCG_BREAKDOWN
      const double omega = res[0] / res[1];
      {
        Acc a0 = 0, a1 = 0, a2 = 0;
        for (int i = threadIdx.x; i < n; i += BS) {
          const Acc si = (Acc)s[i];
          x[i] = (T)fma((Acc)omega, si, fma((Acc)alpha, (Acc)p[i], (Acc)x[i]));
          const T ri = (T)fma(-(Acc)omega, (Acc)t[i], si);
          r[i] = ri;
          const Acc rd = (Acc)ri, wr = (Acc)(wid ? 1.0 : w[i]) * rd;
          a0 = fma((Acc)rh[i], rd, a0);
          a1 = fma(wr, wr, a1);
          a2 = fma(rd, rd, a2);
        }
        double ad[3] = {(double)a0, (double)a1, (double)a2};
        bsum<3, BS>(ad, sm, res);
      }
      o.iters += 1;
      const double mur = sqrt(res[1]) / mu0;
      o.relres_rec = mur;
      if (mur < tol) {
        check_true = true;
        break;
      }
      if (omega == 0.0) BCG_BREAKDOWN
      const double rho1 = res[0], rn = sqrt(res[2]);
      if (!(fabs(rho1) > brk * rhn * rn)) BCG_BREAKDOWN
      const double beta = (rho1 / rho) * (alpha / omega);
      rho = rho1;
      for (int i = threadIdx.x; i < n; i += BS)
        p[i] = (T)fma((Acc)beta, fma(-(Acc)omega, (Acc)v[i], (Acc)p[i]), (Acc)r[i]);
      __syncthreads();
    }
    if (!confirm) {  // inner solve: the recursive residual decides
      o.conv = GSK_CONVERGED;
      return;
    }
    // true residual
    __syncthreads();
    block_spmv<BS>(n, rowptr, colidx, val, x, t, err);
    __syncthreads();
    {
      Acc a0 = 0, a1 = 0;
      for (int i = threadIdx.x; i < n; i += BS) {
        const T ti = (T)((Acc)rhs[i] - (Acc)t[i]);
        t[i] = ti;
        const Acc wt = (Acc)(wid ? 1.0 : w[i]) * (Acc)ti;
        a0 = fma(wt, wt, a0);
        a1 = fma((Acc)ti, (Acc)ti, a1);
      }
      double ad[2] = {(double)a0, (double)a1};
      bsum<2, BS>(ad, sm, res);
    }
    const double mu = sqrt(res[0]) / mu0;
    o.relres_true = mu;
    if (mu < tol) {
      o.conv = GSK_CONVERGED;
      return;
    }
    if (refresh_left == 0) {
      o.conv = broke ? GSK_BREAKDOWN : GSK_STAGNATED;
      return;
    }
    refresh_left -= 1;
    o.refreshes += 1;
    for (int i = threadIdx.x; i < n; i += BS) {
      r[i] = t[i];
      rh[i] = t[i];
      p[i] = t[i];
    }
    rho = res[1];
    rhn = sqrt(res[1]);
    __syncthreads();
  }
#undef BCG_BREAKDOWN
done:
  if (confirm) {  // report the true metric of the returned x
    __syncthreads();
    block_spmv<BS>(n, rowptr, colidx, val, x, t, err);
    __syncthreads();
    Acc a0 = 0;
    for (int i = threadIdx.x; i < n; i += BS) {
      const Acc wt = (Acc)(wid ? 1.0 : w[i]) * ((Acc)rhs[i] - (Acc)t[i]);
      a0 = fma(wt, wt, a0);
    }
    double ad[1] = {(double)a0};
    bsum<1, BS>(ad, sm, res);
    o.relres_true = sqrt(res[0]) / mu0;
  }
}

// GS(p) of one system in place (norms first, then the scaling only if no
// row is zero or non-finite); then the metric weights W2 = 1/||a_i||_2 of the
// scaled rows into w2 (left unused when p = 2: the rows then have unit norm).
// Returns false (and the status) on an input error.  INT_SUM: the row sums
// in the integer pipes (row_inv_norm_pm); measured on the 4,096-system batch
// it pays in the mixed-precision kernel (484 against 531 ms) and not in the
// FP64 one (572 against 455 ms), so each kernel takes its faster form.
template <int BS, bool INT_SUM>
__device__ bool block_gs(const BatchSys& S, double* d, double* w2, bool need_w2, int* status) {
  __shared__ int s_err;
  if (threadIdx.x == 0) s_err = 0;
  __syncthreads();
  const bool scale = !(S.p != S.p);
  const int pm = scale ? pmode_of(S.p) : kP2;
  for (int i = threadIdx.x; i < S.n; i += BS) {
    const int rs = S.rowptr[i], re = S.rowptr[i + 1];
    if (rs < 0 || re < rs || re > S.nnz) {
      atomicOr(&s_err, kErrIndex);
      continue;
    }
    if (scale) d[i] = row_inv_norm<INT_SUM>(S.val + rs, re - rs, pm, S.p, &s_err);
    const unsigned long long bb = (unsigned long long)__double_as_longlong(S.b[i]);
    if ((bb & 0x7ff0000000000000ull) == 0x7ff0000000000000ull) atomicOr(&s_err, kErrNonFinite);
  }
  __syncthreads();
  if (s_err) {
    *status = (s_err & kErrIndex) ? GSK_ERR_ARG : ((s_err & kErrNonFinite) ? GSK_ERR_NONFINITE : GSK_ERR_ZERO_ROW);
    return false;
  }
  for (int i = threadIdx.x; i < S.n; i += BS) {
    const int rs = S.rowptr[i], re = S.rowptr[i + 1];
    if (scale) {
      const double di = d[i];
      for (int k = rs; k < re; ++k) S.val[k] *= di;
      S.b[i] *= di;
    }
    if (need_w2) w2[i] = row_inv_norm<INT_SUM>(S.val + rs, re - rs, kP2, 2.0, &s_err);
  }
  __syncthreads();
  if (s_err) {
    *status = GSK_ERR_ZERO_ROW;
    return false;
  }
  return true;
}

// Register budget of the batched Bi-CGSTAB kernel, as the minimum number of
// resident blocks per SM given to __launch_bounds__ (0: the compiler's own
// choice).  Measured on the 4096-system batch (2D inclusions, side 16..128):
// FP64 at 256 threads is fastest with the compiler's choice (496 ms); the
// mixed kernel at 256 threads is 13% faster held to 3 blocks per SM (80
// registers; 502 ms against 577 ms at its best before), and both 128-thread
// instances gain from 6 blocks per SM.  (batch_gmres keeps the compiler's
// choice: held to 3 or 4 blocks per SM it ran 41% and 73% longer.)
template <int BS, bool MIXED>
constexpr int batch_min_blocks() {
  return BS == 128 ? 6 : (MIXED ? (BS == 256 ? 3 : 1) : 0);
}

template <int BS, bool MIXED>
__global__ void __launch_bounds__(BS, (batch_min_blocks<BS, MIXED>())) batch_bicgstab(BatchParams P) {
  __shared__ double sm[3 * BS];
  __shared__ int s_idx, s_err;
  char* slot = P.scratch + (long long)blockIdx.x * P.slot_bytes;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_idx = (int)atomicAdd(P.queue, 1u);
      s_err = 0;
    }
    __syncthreads();
    if (s_idx >= P.nsys) break;
    const int id = P.order[s_idx];
    const BatchSys S = P.sys[id];
    BatchOut o = {0, 0, 0, 0, GSK_MAXIT, GSK_OK, 1.0, 1.0};
    const int n = S.n;
    double* d = reinterpret_cast<double*>(slot);
    double* w2 = d + n;
    // after GS(2) the rows have unit norm: the metric weights are the identity
    const bool w_identity = P.metric_plain || S.p == 2.0;
    const bool ok = block_gs<BS, MIXED>(S, d, w2, !w_identity || MIXED, &o.status);
    if (ok) {
      if (!MIXED) {
        double* v = w2 + n;
        block_bicgstab<BS, double>(n, S.rowptr, S.colidx, S.val, S.b, S.x, v, v + n, v + 2 * n, v + 3 * n, v + 4 * n,
                               v + 5 * n, w_identity ? nullptr : w2, P.tol, P.maxit, P.refresh, true, P.brk, sm,
                               &s_err, o);
      } else {
        // FP64 refinement around FP32 solves of (W2 A)_32 d = W2 r / ||W2 r||;
        // a system whose refinement step gains less than 10x in the FP64 metric
        // is finished by FP64 Bi-CGSTAB from its current x (escalation)
        double* v64 = w2 + n;        // 6n doubles for the FP64 finish
        double* r64 = v64 + 6 * n;
        float* a32 = reinterpret_cast<float*>(r64 + n);
        float* f = a32 + ((S.nnz + 3) / 4) * 4;
        float *x32 = f, *r = f + n, *rh = f + 2 * n, *p = f + 3 * n, *v = f + 4 * n, *s = f + 5 * n,
              *t = f + 6 * n, *rhs = f + 7 * n;
        __shared__ double res[2];
        for (int i = threadIdx.x; i < n; i += BS)
          for (int k = S.rowptr[i]; k < S.rowptr[i + 1]; ++k) a32[k] = (float)(S.val[k] * w2[i]);
        double mu0 = -1.0, mu_prev = 1.0;
        int total = 0;
        for (int ref = 0;; ++ref) {
          __syncthreads();
          block_spmv<BS, double>(n, S.rowptr, S.colidx, S.val, S.x, r64, &s_err);
          __syncthreads();
          double a0 = 0.0, a1 = 0.0;
          for (int i = threadIdx.x; i < n; i += BS) {
            const double ri = S.b[i] - r64[i];
            r64[i] = ri;
            const double wr = (w_identity ? 1.0 : w2[i]) * ri, w2r = w2[i] * ri;
            a0 = fma(wr, wr, a0);
            a1 = fma(w2r, w2r, a1);
          }
          double ad[2] = {a0, a1};
          bsum<2, BS>(ad, sm, res);
          const double mw = sqrt(res[0]), rn = sqrt(res[1]);
          if (ref == 0) mu0 = mw;
          o.refinements = ref;
          if (!(mu0 > 0.0)) {
            o.conv = mu0 == 0.0 ? GSK_CONVERGED : GSK_MAXIT;
            o.relres_true = mu0 == 0.0 ? 0.0 : 1.0;
            break;
          }
          const double mu = mw / mu0;
          o.relres_true = mu;
          if (mu < P.tol) {
            o.conv = GSK_CONVERGED;
            break;
          }
          if (total >= P.maxit || !(mu == mu)) {
            o.conv = GSK_MAXIT;
            break;
          }
          bool escalate = ref > 0 && mu > 0.1 * mu_prev;
          if (!escalate) {
            mu_prev = mu;
            const double inv = 1.0 / rn;
            for (int i = threadIdx.x; i < n; i += BS) {
              rhs[i] = (float)(w2[i] * r64[i] * inv);
              x32[i] = 0.f;
            }
            __syncthreads();
            BatchOut oi = {0, 0, 0, 0, GSK_MAXIT, GSK_OK, 1.0, 1.0};
            block_bicgstab<BS, float>(n, S.rowptr, S.colidx, a32, rhs, x32, r, rh, p, v, s, t, nullptr, P.inner_tol,
                                  min(P.inner_maxit, P.maxit - total), 0, false, (double)FLT_EPSILON, sm, &s_err,
                                  oi);
            total += oi.iters;
            o.relres_rec = oi.relres_rec;
            __syncthreads();
            // a correction that is not finite, or an inner solve that made no
            // step, is not applied: the system goes to FP64 instead
            int bad = oi.iters == 0;
            for (int i = threadIdx.x; i < n; i += BS) bad |= !isfinite(x32[i]);
            escalate = __syncthreads_or(bad) != 0;
            if (!escalate) {
              for (int i = threadIdx.x; i < n; i += BS) S.x[i] = fma(rn, (double)x32[i], S.x[i]);
              continue;
            }
          }
          // escalate: FP64 Bi-CGSTAB on the remaining error, the tolerance
          // rescaled so that it is still relative to the first residual
          BatchOut o64 = {0, 0, 0, 0, GSK_MAXIT, GSK_OK, 1.0, 1.0};
          block_bicgstab<BS, double>(n, S.rowptr, S.colidx, S.val, S.b, S.x, v64, v64 + n, v64 + 2 * n, v64 + 3 * n,
                                 v64 + 4 * n, v64 + 5 * n, w_identity ? nullptr : w2, P.tol / mu, P.maxit - total,
                                 P.refresh > 10 ? P.refresh : 10, true, P.brk, sm, &s_err, o64, true);
          total += o64.iters;
          o.conv = o64.conv;
          o.refreshes = o64.refreshes;
          o.relres_true = o64.relres_true * mu;
          o.relres_rec = o64.relres_rec * mu;
          o.refinements = ref + 1;
          break;
        }
        o.iters = total;
      }
    }
    __syncthreads();
    if (s_err) o.status = GSK_ERR_ARG;
    if (threadIdx.x == 0) P.out[id] = o;
  }
}

// ------------------------------------------------------------ batched GMRES

// Per-block GMRES work arrays (slot memory, L2-resident while the block
// works on its system).
struct GmWork {
  double *V, *H, *g, *cs, *sn, *y, *h;
};

// h[c] = (V_c, w) for c < k: the columns in chunks of 8 register
// accumulators, one block reduction per chunk.
template <int BS>
__device__ void block_multidot(int n, int k, const double* V, const double* w, double* h, double* sm,
                               double* res) {
  for (int c0 = 0; c0 < k; c0 += 8) {
    const int nc = min(8, k - c0);
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += BS) {
      const double wi = w[i];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < nc) acc[q] = fma(V[(long long)(c0 + q) * n + i], wi, acc[q]);
    }
    bsum<8, BS>(acc, sm, res);
    if (threadIdx.x < nc) h[c0 + threadIdx.x] = res[threadIdx.x];
  }
  __syncthreads();
}

// w -= sum_c h[c] V_c for c < k.
template <int BS>
__device__ void block_subtract(int n, int k, const double* V, double* w, const double* h) {
  for (int i = threadIdx.x; i < n; i += BS) {
    double wi = w[i];
    for (int c = 0; c < k; ++c) wi = fma(-h[c], V[(long long)c * n + i], wi);
    w[i] = wi;
  }
  __syncthreads();
}

// V[:, 0] = rhs - A x; res2 = (||W r||, ||r||).
template <int BS>
__device__ void block_gm_residual(int n, const int* rowptr, const int* colidx, const double* val,
                                  const double* rhs, const double* x, const double* wgt, double* r, double* sm,
                                  double* res, int* err, double& mu_w, double& nrm) {
  block_spmv<BS, double>(n, rowptr, colidx, val, x, r, err);
  __syncthreads();
  double a0 = 0.0, a1 = 0.0;
  for (int i = threadIdx.x; i < n; i += BS) {
    const double ri = rhs[i] - r[i];
    r[i] = ri;
    const double wr = (wgt ? wgt[i] : 1.0) * ri;
    a0 = fma(wr, wr, a0);
    a1 = fma(ri, ri, a1);
  }
  double ad[2] = {a0, a1};
  bsum<2, BS>(ad, sm, res);
  mu_w = sqrt(res[0]);
  nrm = sqrt(res[1]);
}

// Restarted GMRES(m) with classical Gram-Schmidt applied twice (Sec. 2) on
// one system, block-local, with the cycle of gmres_solve: a normalised basis,
// Givens rotations of the Hessenberg columns (one thread), the cycle ending
// when |g_{j+1}| < tau ||r0||, at breakdown h_{j+1,j} <= 1e-14 ||A v_j||
// (from the CGS coefficients and h_{j+1,j}), after m steps or at maxit; the
// true metric ||W r|| / ||W r0|| decides convergence and tau is tightened by
// tol / metric when the estimate met it but the metric did not.
template <int BS>
__device__ void block_gmres(int n, const int* rowptr, const int* colidx, const double* val, const double* rhs,
                            double* x, const double* wgt, int m, double tol, int maxit, const GmWork& W,
                            double* sm, int* err, BatchOut& o) {
  __shared__ double res[8];
  __shared__ double s_scal[3];
  const int ld = m + 1;
  double mu_w, beta;
  block_gm_residual<BS>(n, rowptr, colidx, val, rhs, x, wgt, W.V, sm, res, err, mu_w, beta);
  const double mu0 = mu_w, rho0 = beta;
  o.iters = 0;
  o.restarts = 0;
  o.relres_rec = 1.0;
  o.relres_true = 1.0;
  o.conv = GSK_MAXIT;
  if (!(mu0 > 0.0)) {
    if (mu0 == 0.0) {
      o.conv = GSK_CONVERGED;
      o.relres_true = o.relres_rec = 0.0;
    }
    return;
  }
  double tau = tol;
  for (;;) {
    const double ib = 1.0 / beta;
    for (int i = threadIdx.x; i < n; i += BS) W.V[i] *= ib;
    if (threadIdx.x == 0) {
      W.g[0] = beta;
      for (int q = 1; q <= m; ++q) W.g[q] = 0.0;
    }
    __syncthreads();
    int kcols = 0;
    bool est_hit = false;
    for (int j = 0; j < m && o.iters < maxit; ++j) {
      double* w = W.V + (long long)(j + 1) * n;
      block_spmv<BS, double>(n, rowptr, colidx, val, W.V + (long long)j * n, w, err);
      __syncthreads();
      const int k = j + 1;
      double* hc = W.H + (long long)j * ld;
      block_multidot<BS>(n, k, W.V, w, W.h, sm, res);
      if (threadIdx.x < k) hc[threadIdx.x] = W.h[threadIdx.x];
      block_subtract<BS>(n, k, W.V, w, W.h);
      block_multidot<BS>(n, k, W.V, w, W.h, sm, res);
      if (threadIdx.x < k) hc[threadIdx.x] += W.h[threadIdx.x];
      block_subtract<BS>(n, k, W.V, w, W.h);
      double a0 = 0.0;
      for (int i = threadIdx.x; i < n; i += BS) a0 = fma(w[i], w[i], a0);
      double ad[1] = {a0};
      bsum<1, BS>(ad, sm, res);
      const double hnext = sqrt(res[0]);
      if (threadIdx.x == 0) {
        double aw2 = hnext * hnext;  // ||A v_j||^2 = ||h||^2 + h_{j+1,j}^2
        for (int c = 0; c <= j; ++c) aw2 = fma(hc[c], hc[c], aw2);
        for (int q = 0; q < j; ++q) {
          const double t0 = W.cs[q] * hc[q] + W.sn[q] * hc[q + 1];
          const double t1 = -W.sn[q] * hc[q] + W.cs[q] * hc[q + 1];
          hc[q] = t0;
          hc[q + 1] = t1;
        }
        const double rho = hypot(hc[j], hnext);
        const double c_ = rho == 0.0 ? 1.0 : hc[j] / rho, s_ = rho == 0.0 ? 0.0 : hnext / rho;
        W.cs[j] = c_;
        W.sn[j] = s_;
        hc[j] = rho;
        hc[j + 1] = 0.0;
        const double gj = W.g[j];
        W.g[j + 1] = -s_ * gj;
        W.g[j] = c_ * gj;
        const double est = fabs(W.g[j + 1]) / rho0;
        s_scal[0] = est;
        s_scal[1] = est < tau ? 1.0 : (hnext <= 1e-14 * sqrt(aw2) ? 2.0 : 0.0);
        s_scal[2] = hnext;
      }
      __syncthreads();
      o.iters += 1;
      kcols = k;
      o.relres_rec = s_scal[0];
      if (s_scal[1] == 1.0) {
        est_hit = true;
        break;
      }
      if (s_scal[1] == 2.0) break;
      const double ih = 1.0 / s_scal[2];
      for (int i = threadIdx.x; i < n; i += BS) w[i] *= ih;
      __syncthreads();
    }
    // H y = g by back substitution, then x += V y
    if (threadIdx.x == 0) {
      for (int i = kcols - 1; i >= 0; --i) {
        double sacc = W.g[i];
        for (int q = i + 1; q < kcols; ++q) sacc -= W.H[(long long)q * ld + i] * W.y[q];
        W.y[i] = sacc / W.H[(long long)i * ld + i];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += BS) {
      double xi = x[i];
      for (int c = 0; c < kcols; ++c) xi = fma(W.y[c], W.V[(long long)c * n + i], xi);
      x[i] = xi;
    }
    __syncthreads();
    block_gm_residual<BS>(n, rowptr, colidx, val, rhs, x, wgt, W.V, sm, res, err, mu_w, beta);
    const double mu = mu_w / mu0;
    o.relres_true = mu;
    if (mu < tol) {
      o.conv = GSK_CONVERGED;
      return;
    }
    if (o.iters >= maxit || kcols == 0 || !(beta > 0.0)) {
      o.conv = GSK_MAXIT;
      return;
    }
    if (est_hit) tau = tau * (tol / mu);
    o.restarts += 1;
  }
}

template <int BS>
__global__ void __launch_bounds__(BS) batch_gmres(BatchParams P) {
  __shared__ double sm[8 * BS];
  __shared__ int s_idx, s_err;
  char* slot = P.scratch + (long long)blockIdx.x * P.slot_bytes;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_idx = (int)atomicAdd(P.queue, 1u);
      s_err = 0;
    }
    __syncthreads();
    if (s_idx >= P.nsys) break;
    const int id = P.order[s_idx];
    const BatchSys S = P.sys[id];
    BatchOut o = {0, 0, 0, 0, GSK_MAXIT, GSK_OK, 1.0, 1.0};
    const int n = S.n, m = P.mvec[id];
    double* d = reinterpret_cast<double*>(slot);
    double* w2 = d + n;
    const bool w_identity = P.metric_plain || S.p == 2.0;
    const bool ok = block_gs<BS, false>(S, d, w2, !w_identity, &o.status);
    if (ok) {
      GmWork W;
      W.V = w2 + n;
      W.H = W.V + (long long)(m + 1) * n;
      W.g = W.H + (long long)(m + 1) * m;
      W.cs = W.g + m + 1;
      W.sn = W.cs + m;
      W.y = W.sn + m;
      W.h = W.y + m;
      block_gmres<BS>(n, S.rowptr, S.colidx, S.val, S.b, S.x, w_identity ? nullptr : w2, m, P.tol, P.maxit, W, sm,
                      &s_err, o);
    }
    __syncthreads();
    if (s_err) o.status = GSK_ERR_ARG;
    if (threadIdx.x == 0) P.out[id] = o;
  }
}

static size_t batch_gmres_slot_bytes(int nmax, int mmax) {
  // d, w2, V (m+1 columns), H, g, cs, sn, y, h
  size_t b = 8 * ((size_t)nmax * (mmax + 3) + (size_t)(mmax + 1) * mmax + 5 * (size_t)(mmax + 1));
  return (b + 255) / 256 * 256;
}

static size_t batch_slot_bytes(bool mixed, int nmax, int nnzmax) {
  // FP64: d, w2, six vectors.  Mixed: d, w2, six FP64 vectors (escalation),
  // the FP64 residual, (W2 A)_32 and eight FP32 vectors.
  size_t b = mixed ? (9 * 8 * (size_t)nmax + 4 * ((size_t)(nnzmax + 3) / 4 * 4) + 8 * 4 * (size_t)nmax)
                   : 8 * 8 * (size_t)nmax;
  return (b + 255) / 256 * 256;
}

// One persistent launch of the solver over the systems in `order`.
template <int BS>
static void batch_launch(int solver, bool mixed, int grid, const BatchParams& P, cudaStream_t st) {
  if (solver == 0) batch_gmres<BS><<<grid, BS, 0, st>>>(P);
  else if (mixed) batch_bicgstab<BS, true><<<grid, BS, 0, st>>>(P);
  else batch_bicgstab<BS, false><<<grid, BS, 0, st>>>(P);
}

template <int BS>
static int batch_blocks_per_sm(int solver, bool mixed) {
  int per_sm = 0;
  cudaError_t e;
  if (solver == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_gmres<BS>, BS, 0);
  else if (mixed) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_bicgstab<BS, true>, BS, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_bicgstab<BS, false>, BS, 0);
  if (e != cudaSuccess) cudaGetLastError();
  return (e != cudaSuccess || per_sm < 1) ? 1 : per_sm;
}

// The grid-wide lane of a batch: the context's child context and stream,
// created on first use.
static gsk_status batch_aux(gsk_ctx* ctx) {
  if (ctx->aux) return GSK_OK;
  gsk_ctx* aux = nullptr;
  gsk_status s = gsk_ctx_create(&aux, ctx->device);
  if (s != GSK_OK) return ctx->fail(s, "creating the batch's grid-wide lane failed");
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    gsk_ctx_destroy(aux);
    return ctx->cuda_fail(e, "creating the batch's grid-wide lane");
  }
  ctx->aux = aux;
  return GSK_OK;
}

// solver 0: GMRES(m[i]) (FP64), 1: Bi-CGSTAB (FP64 or mixed).  Systems with
// more than opts.batch_large_n rows go to the grid-wide solvers (gs_scale,
// then gmres_solve / bicgstab_solve with the same options), one at a time;
// the others to one persistent launch, one block each.  When a batch has
// both, the persistent launch goes first on `stream` and the grid-wide
// solves run beside it on a second stream with a child context (its own
// workspace), their kernels taking the SMs the batch's blocks leave as
// they finish; `stream` waits for both before the call returns.
static gsk_status batch_solve(gsk_ctx* ctx, int solver, int nsys, const gsk_csr* A, void* const* b, void* const* x,
                              const double* p, const int* mvec, double tol, const gsk_opts* opts_in, gsk_info* infos,
                              int32_t* status, void* stream) {
  if (!ctx) return GSK_ERR_ARG;
  if (nsys < 0 || (nsys > 0 && (!A || !b || !x))) return ctx->fail(GSK_ERR_ARG, "bad batch arrays");
  gsk_opts opts;
  if (opts_in) opts = *opts_in;
  else gsk_opts_default(&opts);
  if (!(tol >= 0.0) || opts.maxit < 0 || opts.refresh < 0 || !(opts.inner_tol > 0.0) || opts.inner_maxit < 0)
    return ctx->fail(GSK_ERR_ARG, "bad tol/maxit/refresh/inner_tol");
  if (opts.weights) return ctx->fail(GSK_ERR_ARG, "the batched solver derives its metric weights itself");
  if (opts.precond) return ctx->fail(GSK_ERR_ARG, "the batched solver takes no preconditioner");
  const int BS = opts.batch_block == 0 ? 256 : opts.batch_block;
  if (BS != 128 && BS != 256 && BS != 512) return ctx->fail(GSK_ERR_ARG, "batch_block must be 0, 128, 256 or 512");
  if (opts.batch_large_n < 0) return ctx->fail(GSK_ERR_ARG, "batch_large_n must be >= 0");
  const bool mixed = opts.precision == GSK_PREC_MIXED;
  if (solver == 0 && !mixed && !mvec) return ctx->fail(GSK_ERR_ARG, "NULL m array");
  if (nsys == 0) return GSK_OK;
  std::vector<BatchSys> hs(nsys);
  std::vector<int> small, large;
  int nmax = 0, nnzmax = 0, mmax = 1;
  for (int i = 0; i < nsys; ++i) {
    gsk_status s = check_csr(ctx, &A[i]);
    if (s != GSK_OK) return s;
    if (A[i].dtype != GSK_F64) return ctx->fail(GSK_ERR_ARG, "batched systems must be FP64");
    if (A[i].n > 0 && (!b[i] || !x[i])) return ctx->fail(GSK_ERR_ARG, "NULL b or x in the batch");
    const double pi = p ? p[i] : NAN;
    if (!(pi != pi) && !(pi >= 1.0)) return ctx->fail(GSK_ERR_ARG, "p must be >= 1, INFINITY or NaN");
    if (solver == 0 && (!mvec || mvec[i] < 1 || mvec[i] > kMaxM)) return ctx->fail(GSK_ERR_ARG, "m must be in 1..64");
    hs[i] = BatchSys{A[i].n, A[i].nnz, A[i].rowptr, A[i].colidx, (double*)A[i].val, (double*)b[i], (double*)x[i], pi};
    if (opts.batch_large_n > 0 && A[i].n > opts.batch_large_n) {
      large.push_back(i);
    } else {
      small.push_back(i);
      nmax = std::max(nmax, A[i].n);
      nnzmax = std::max(nnzmax, A[i].nnz);
      if (solver == 0) mmax = std::max(mmax, mvec[i]);
    }
  }
  if (solver == 0 && mixed && !small.empty())
    return ctx->fail(GSK_ERR_ARG, "the one-block GMRES is FP64: mixed precision only with batch_large_n routing");
  gsk_status worst = GSK_OK;
  std::string first_error;
  cudaStream_t st = (cudaStream_t)stream;
  // grid-wide lane: beside the persistent launch when there is one
  const bool beside = !large.empty() && !small.empty();
  gsk_ctx* lctx = ctx;
  cudaStream_t lst = st;
  if (beside) {
    gsk_status s = batch_aux(ctx);
    if (s != GSK_OK) return s;
    lctx = ctx->aux;
    lst = ctx->aux_stream;
    // size the lane's workspace for its largest system now: growing it later
    // would free memory, which waits for the whole device
    size_t need = 0;
    for (int i : large) {
      size_t bi = 0;
      if (gsk_workspace_bytes(A[i].n, A[i].nnz, solver == 0 ? 0 : 1, solver == 0 ? mvec[i] : 1, opts.precision,
                              &bi) == GSK_OK)
        need = std::max(need, bi);
    }
    if ((s = lctx->reserve(need)) != GSK_OK) {
      ctx->last_error = lctx->last_error;
      return s;
    }
    // the second stream starts after the work the caller queued on `stream`
    GSK_CK(cudaEventRecord(ctx->ev_fork, st));
    GSK_CK(cudaStreamWaitEvent(lst, ctx->ev_fork, 0));
  }
  BatchOut* dout = nullptr;
  if (!small.empty()) {
    const int ns = (int)small.size();
    // largest systems first
    std::stable_sort(small.begin(), small.end(), [&](int a, int c) { return hs[a].nnz > hs[c].nnz; });
    int per_sm = BS == 128 ? batch_blocks_per_sm<128>(solver, mixed)
                           : (BS == 256 ? batch_blocks_per_sm<256>(solver, mixed) : batch_blocks_per_sm<512>(solver, mixed));
    const int grid = std::max(1, std::min(ns, ctx->num_sms * per_sm));
    const size_t slot = solver == 0 ? batch_gmres_slot_bytes(nmax, mmax) : batch_slot_bytes(mixed, nmax, nnzmax);
    Arena sizing;
    sizing.take<unsigned>(64);
    sizing.take<BatchSys>(nsys);
    sizing.take<int>(ns);
    sizing.take<int>(nsys);
    sizing.take<BatchOut>(nsys);
    sizing.take<char>(slot * grid);
    gsk_status s = ctx->reserve(sizing.off);
    if (s != GSK_OK) return s;
    Arena ar{(char*)ctx->ws, ctx->ws_bytes, 0};
    unsigned* queue = ar.take<unsigned>(64);
    BatchSys* dsys = ar.take<BatchSys>(nsys);
    int* dorder = ar.take<int>(ns);
    int* dm = ar.take<int>(nsys);
    dout = ar.take<BatchOut>(nsys);
    char* scratch = ar.take<char>(slot * grid);
    GSK_CK(cudaEventRecord(ctx->ev0, st));
    GSK_CK(cudaMemsetAsync(queue, 0, sizeof(unsigned), st));
    GSK_CK(cudaMemcpyAsync(dsys, hs.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice, st));
    GSK_CK(cudaMemcpyAsync(dorder, small.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
    if (solver == 0) GSK_CK(cudaMemcpyAsync(dm, mvec, sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
    BatchParams P{dsys, dorder, solver == 0 ? dm : nullptr, ns, queue, dout, scratch, (long long)slot, tol,
                  opts.inner_tol, 1e-16 * DBL_EPSILON, opts.maxit, opts.refresh,
                  opts.inner_maxit > 0 ? opts.inner_maxit : kBatchInnerMaxit, opts.metric == GSK_METRIC_PLAIN ? 1 : 0};
    if (BS == 128) batch_launch<128>(solver, mixed, grid, P, st);
    else if (BS == 256) batch_launch<256>(solver, mixed, grid, P, st);
    else batch_launch<512>(solver, mixed, grid, P, st);
    GSK_CK(cudaGetLastError());
    GSK_CK(cudaEventRecord(ctx->ev1, st));
  }
  // large systems: the grid-wide path, one after the other (each call waits
  // for its own stream only, so the persistent launch keeps running)
  for (int i : large) {
    gsk_info inf = {};
    gsk_status si = GSK_OK;
    if (!(hs[i].p != hs[i].p)) si = gs_scale(lctx, const_cast<gsk_csr*>(&A[i]), b[i], hs[i].p, nullptr, lst);
    if (si == GSK_OK)
      si = solver == 0 ? gmres_solve(lctx, &A[i], b[i], x[i], mvec[i], tol, &opts, &inf, lst)
                       : bicgstab_solve(lctx, &A[i], b[i], x[i], tol, &opts, &inf, lst);
    if (infos) infos[i] = inf;
    if (status) status[i] = si;
    if (si != GSK_OK && worst == GSK_OK) {
      worst = si;
      first_error = lctx->last_error;
    }
  }
  if (beside) {
    GSK_CK(cudaEventRecord(ctx->ev_join, lst));
    GSK_CK(cudaStreamWaitEvent(st, ctx->ev_join, 0));
  }
  if (dout && (infos || status)) {
    std::vector<BatchOut> ho(nsys);
    GSK_CK(cudaMemcpyAsync(ho.data(), dout, sizeof(BatchOut) * nsys, cudaMemcpyDeviceToHost, st));
    GSK_CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    for (int i : small) {
      if (infos) infos[i] = gsk_info{ho[i].iters, ho[i].restarts, ho[i].refreshes, ho[i].refinements, ho[i].conv,
                                     ho[i].relres_true, ho[i].relres_rec, ms};
      if (status) status[i] = ho[i].status;
      if (ho[i].status != GSK_OK && worst == GSK_OK) worst = (gsk_status)ho[i].status;
    }
  }
  if (worst != GSK_OK)
    return ctx->fail(worst, "at least one system of the batch failed (see status[])" +
                                (first_error.empty() ? std::string() : ": " + first_error));
  return GSK_OK;
}

}  // namespace gsk

extern "C" gsk_status bicgstab_solve_batched(gsk_ctx* ctx, int nsys, const gsk_csr* A, void* const* b,
                                             void* const* x, const double* p, double tol, const gsk_opts* opts,
                                             gsk_info* infos, int32_t* status, void* stream) {
  return gsk::batch_solve(ctx, 1, nsys, A, b, x, p, nullptr, tol, opts, infos, status, stream);
}

extern "C" gsk_status gmres_solve_batched(gsk_ctx* ctx, int nsys, const gsk_csr* A, void* const* b, void* const* x,
                                          const double* p, const int* m, double tol, const gsk_opts* opts,
                                          gsk_info* infos, int32_t* status, void* stream) {
  return gsk::batch_solve(ctx, 0, nsys, A, b, x, p, m, tol, opts, infos, status, stream);
}
