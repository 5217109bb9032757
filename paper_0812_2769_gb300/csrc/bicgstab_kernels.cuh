// Bi-CGSTAB (Sec. 2; van der Vorst 1992) with every scalar and every
// stopping decision on the device.
//
// One iteration is the kernel chain
//   k1  v = A p,           sigma = <rh, v>, ||v||         -> alpha or breakdown
//   k2a s = r - alpha v
//   k2b t = A s,           ||W s||, <t, s>, <t, t>         -> half-step exit,
//                                                             omega or breakdown
// (the half-step test ||W s|| < tol is taken where s is read anyway, in k2b's
// epilogue: k2a then needs no cross-block reduction, and the product t = A s
// of the last iteration is the only work done for nothing)
//   k3  x += alpha p + omega s, r = s - omega t,
//                          <rh, r>, ||W r||, ||r||         -> beta, flags
//   then either k4  p = r + beta (p - omega v)             (keep iterating)
//   or          kt  t = b - A x, ||W t||, ||t||            (true residual)
//               kr  finish, or refresh r = rh = p = t
// The chain is recorded once into a CUDA graph: a WHILE node whose body holds
// several iterations k1..k4 in a row, then kt and kr.  Every kernel checks
// the device flags at entry: after the iteration that set check or stop the
// remaining ones return at once, and kt/kr work only when one did; kr sets
// the WHILE condition.  A solve is one graph launch.  The same kernels can
// also be driven from a host loop with a CUDA event around each launch
// (gsk_profile_solve).
//
// The breakdown tolerance is 1e-16 * DBL_EPSILON relative to the vector
// norms (Sec. 2.2).  The stopping metric is ||W(b - Ax)|| / ||W(b - Ax0)||
// with W the GS(2) scales of A (Sec. 2.2); when W is the identity to within
// 4 ulp (an already GS(2)-scaled system) the weight loads are skipped and
// ||r|| is taken from ||W r||.
#pragma once

#include <cfloat>

#include "internal.hpp"
#include "spmv_tma.cuh"

namespace gsk {

struct BcgState {
  double rho, alpha, omega, beta, rhn, mu0, mu_s, mu_rec, mu_true, tt_true, tol, brk;
  int maxit, refresh_left, iters, refreshes, conv, stop, halfexit, check, active, w_identity;
};

template <typename T>
struct BcgArgs {
  int n, nnz;
  const int* rowptr;
  const int* colidx;
  const T* val;
  const T* b;
  T* x;
  T *r, *rh, *p, *v, *s, *t;
  // the vectors multiplied by A and along which x moves: p and s, or, with a
  // right preconditioner M, M^-1 p and M^-1 s (Sec. 2)
  const T* p_in;
  const T* s_in;
  const double* w;
  BcgState* S;
  GridRed red;
  unsigned* cnt;
  int* err;
  cudaGraphConditionalHandle h_while;
  int in_graph;
  int vec_ok;  // x (and w, if any) are 16-byte aligned: 128-bit loads allowed
};

template <typename T>
__device__ __forceinline__ void set_cond(const BcgArgs<T>& a, cudaGraphConditionalHandle h, unsigned v) {
  if (a.in_graph) cudaGraphSetConditional(h, v);
}

// Vector kernels: each thread takes R = 16/sizeof(T) consecutive rows per
// trip (128-bit loads of the workspace vectors, which are 256-byte aligned);
// the last partial group, and everything when the caller's x or weights are
// not 16-byte aligned, takes the scalar path.  The row-to-thread map depends
// only on the grid.
#define BCG_VEC_LOOP(a, R)                                                                         \
  for (int i0 = (R) * (blockIdx.x * kBlock + threadIdx.x), vstride_ = (R) * gridDim.x * kBlock; \
       i0 < (a).n; i0 += vstride_)

__device__ __forceinline__ double wgt(const double* w, bool wid, int i) { return wid ? 1.0 : __ldg(w + i); }

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_init(BcgArgs<T> a) {
  __shared__ PipeSmem<T> pipe;
  __shared__ double blk[2], tot[2];
  double* sm = reinterpret_cast<double*>(&pipe);  // reduction scratch after the product
  BcgState* S = a.S;
  const bool wid = S->w_identity;
  double acc[2] = {0.0, 0.0};
  spmv_rows_tma(a.rowptr, a.colidx, a.val, a.x, a.n, a.nnz, pipe, a.err, [&](int i, T ax) {
    const T r = a.b[i] - ax;
    a.r[i] = r;
    a.rh[i] = r;
    a.p[i] = r;
    const double wr = wgt(a.w, wid, i) * (double)r;
    acc[0] = fma(wr, wr, acc[0]);
    acc[1] = fma((double)r, (double)r, acc[1]);
  });
  block_sum<2, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    const int e = *(volatile int*)a.err;
    const double mu0 = sqrt(tot[0]);
    S->iters = 0;
    S->refreshes = 0;
    S->halfexit = 0;
    S->check = 0;
    S->mu0 = mu0;
    S->rho = tot[1];
    S->rhn = sqrt(tot[1]);
    S->mu_rec = 1.0;
    S->mu_true = 1.0;
    S->conv = GSK_MAXIT;
    int active = 1;
    if (e) {
      active = 0;
    } else if (!isfinite(mu0)) {
      atomicOr(a.err, kErrNonFinite);
      active = 0;
    } else if (mu0 == 0.0) {
      S->conv = GSK_CONVERGED;
      S->mu_true = 0.0;
      S->mu_rec = 0.0;
      active = 0;
    } else if (S->maxit <= 0) {
      active = 0;
    }
    S->stop = !active;
    S->active = active;
    set_cond(a, a.h_while, active);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k1(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop || S->check) return;
  __shared__ PipeSmem<T> pipe;
  __shared__ double blk[2], tot[2], sc[3];
  // the scalars of the closing decision, loaded at entry (their round trip
  // overlaps the product) into shared memory (no registers held meanwhile)
  if (threadIdx.x == 0) {
    sc[0] = S->brk;
    sc[1] = S->rhn;
    sc[2] = S->rho;
  }
  double* sm = reinterpret_cast<double*>(&pipe);  // reduction scratch after the product
  using Acc = typename AccOf<T>::type;
  const T* __restrict__ rh = a.rh;
  T* __restrict__ vout = a.v;
  Acc acc[2] = {Acc(0), Acc(0)};
  spmv_rows_tma(a.rowptr, a.colidx, a.val, a.p_in, a.n, a.nnz, pipe, a.err, [&](int i, T v) {
    vout[i] = v;
    acc[0] = fma((Acc)rh[i], (Acc)v, acc[0]);
    acc[1] = fma((Acc)v, (Acc)v, acc[1]);
  });
  block_sum<2, kBlock>(acc, reinterpret_cast<Acc*>(sm), blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    const double sigma = tot[0], vn = sqrt(tot[1]);
    if (*(volatile int*)a.err) {
      S->stop = 1;
    } else if (!(fabs(sigma) > sc[0] * sc[1] * vn)) {
      S->conv = GSK_BREAKDOWN;
      S->stop = 1;
    } else {
      S->alpha = sc[2] / sigma;
    }
  }
}

// s = r - alpha v.
template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k2a(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop || S->check) return;
  using Acc = typename AccOf<T>::type;
  const Acc alpha = (Acc)S->alpha;
  constexpr int R = Vec16<T>::R;
  const T* __restrict__ r = a.r;
  const T* __restrict__ v = a.v;
  T* __restrict__ s = a.s;
  BCG_VEC_LOOP(a, R) {
    if (i0 + R <= a.n) {
      const Vec16<T> rv = vload(r + i0), vv = vload(v + i0);
      Vec16<T> sv;
#pragma unroll
      for (int q = 0; q < R; ++q) sv.v[q] = (T)fma(-alpha, (Acc)vv.v[q], (Acc)rv.v[q]);
      vstore(s + i0, sv);
    } else {
      for (int i = i0; i < a.n; ++i) s[i] = (T)fma(-alpha, (Acc)v[i], (Acc)r[i]);
    }
  }
}

// t = A s with <t, s>, <t, t> and ||W s||^2 in the epilogue; the weights'
// presence (WID: W = I) is a compile-time choice, so no predicated-off FP64
// multiply runs per row.
template <bool WID, typename T, typename Acc>
__device__ __forceinline__ void bcg_k2b_rows(const BcgArgs<T>& a, PipeSmem<T>& pipe, Acc (&acc)[3]) {
  const T* __restrict__ sv = a.s;
  T* __restrict__ tout = a.t;
  spmv_rows_tma(a.rowptr, a.colidx, a.val, a.s_in, a.n, a.nnz, pipe, a.err, [&](int i, T t) {
    tout[i] = t;
    const Acc si = (Acc)sv[i];
    acc[0] = fma((Acc)t, si, acc[0]);
    acc[1] = fma((Acc)t, (Acc)t, acc[1]);
    const Acc ws = WID ? si : (Acc)__ldg(a.w + i) * si;
    acc[2] = fma(ws, ws, acc[2]);
  });
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k2b(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop || S->check) return;
  __shared__ PipeSmem<T> pipe;
  __shared__ double blk[3], tot[3], sc[2];
  if (threadIdx.x == 0) {  // the closing decision's scalars, loaded at entry
    sc[0] = S->mu0;
    sc[1] = S->tol;
  }
  double* sm = reinterpret_cast<double*>(&pipe);  // reduction scratch after the product
  using Acc = typename AccOf<T>::type;
  Acc acc[3] = {Acc(0), Acc(0), Acc(0)};
  if (S->w_identity) bcg_k2b_rows<true>(a, pipe, acc);
  else bcg_k2b_rows<false>(a, pipe, acc);
  block_sum<3, kBlock>(acc, reinterpret_cast<Acc*>(sm), blk);
  if (grid_sum(blk, 3, a.red, tot) && threadIdx.x == 0) {
    const double mus = sqrt(tot[2]) / sc[0];
    S->mu_s = mus;
    if (*(volatile int*)a.err) {
      S->stop = 1;
    } else if (mus < sc[1]) {
      S->halfexit = 1;  // x += alpha p in k3; this t is not used
    } else if (!(tot[1] > 0.0)) {
      S->conv = GSK_BREAKDOWN;
      S->stop = 1;
    } else {
      S->omega = tot[0] / tot[1];
    }
  }
}

template <bool WID, bool PRE, typename T, typename Acc>
__device__ __forceinline__ void bcg_k3_row(const BcgArgs<T>& a, int i, Acc alpha, Acc omega, Acc (&acc)[3]) {
  const Acc s = (Acc)a.s[i];
  const Acc x = fma(alpha, (Acc)a.p_in[i], (Acc)a.x[i]);
  a.x[i] = (T)fma(omega, PRE ? (Acc)a.s_in[i] : s, x);
  const T r = (T)fma(-omega, (Acc)a.t[i], s);
  a.r[i] = r;
  const Acc rd = (Acc)r;
  acc[0] = fma((Acc)a.rh[i], rd, acc[0]);
  if (WID) {
    acc[1] = fma(rd, rd, acc[1]);
  } else {
    const Acc wr = (Acc)__ldg(a.w + i) * rd;
    acc[1] = fma(wr, wr, acc[1]);
    acc[2] = fma(rd, rd, acc[2]);
  }
}

// x += alpha p + omega s (p_in, s_in with a preconditioner: PRE),
// r = s - omega t, and the sums (r^, r), ||W r||^2 and (weights present)
// ||r||^2; WID as in bcg_k2b_rows.
template <bool WID, bool PRE, typename T, typename Acc>
__device__ __forceinline__ void bcg_k3_rows(const BcgArgs<T>& a, Acc alpha, Acc omega, Acc (&acc)[3]) {
  constexpr int R = Vec16<T>::R;
  BCG_VEC_LOOP(a, R) {
    if (i0 + R <= a.n && a.vec_ok) {
      const Vec16<T> sv = vload(a.s + i0), pv = vload(a.p_in + i0), xv = vload(a.x + i0), tv = vload(a.t + i0),
                     hv = vload(a.rh + i0);
      Vec16<T> shv;
      if (PRE) shv = vload(a.s_in + i0);
      Vec16<T> xo, ro;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const Acc sq = (Acc)sv.v[q];
        xo.v[q] = (T)fma(omega, PRE ? (Acc)shv.v[q] : sq, fma(alpha, (Acc)pv.v[q], (Acc)xv.v[q]));
        ro.v[q] = (T)fma(-omega, (Acc)tv.v[q], sq);
        const Acc rd = (Acc)ro.v[q];
        acc[0] = fma((Acc)hv.v[q], rd, acc[0]);
        if (WID) {
          acc[1] = fma(rd, rd, acc[1]);
        } else {
          const Acc wr = (Acc)__ldg(a.w + i0 + q) * rd;
          acc[1] = fma(wr, wr, acc[1]);
          acc[2] = fma(rd, rd, acc[2]);
        }
      }
      vstore(a.x + i0, xo);
      vstore(a.r + i0, ro);
    } else {
      for (int i = i0; i < min(i0 + R, a.n); ++i) bcg_k3_row<WID, PRE>(a, i, alpha, omega, acc);
    }
  }
}

template <typename T, bool PRE = false>
__global__ void __launch_bounds__(kBlock) bcg_k3(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (S->stop || S->check) return;
  using Acc = typename AccOf<T>::type;
  const Acc alpha = (Acc)S->alpha;
  if (S->halfexit) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < a.n; i += gridDim.x * kBlock)
      a.x[i] = (T)fma(alpha, (Acc)a.p_in[i], (Acc)a.x[i]);
    if (grid_last(a.cnt) && threadIdx.x == 0) {
      S->iters += 1;
      S->mu_rec = S->mu_s;
      S->check = 1;
    }
    return;
  }
  __shared__ double sm[3 * kBlock], blk[3], tot[3], sc[8];
  __shared__ int si[2];
  if (threadIdx.x == 0) {  // the closing decision's scalars, loaded at entry
    sc[0] = S->mu0;
    sc[1] = S->tol;
    sc[2] = S->omega;
    sc[3] = S->brk;
    sc[4] = S->rhn;
    sc[5] = S->rho;
    sc[6] = S->alpha;
    si[0] = S->iters;
    si[1] = S->maxit;
  }
  const Acc omega = (Acc)S->omega;
  const bool wid = S->w_identity;
  Acc acc[3] = {Acc(0), Acc(0), Acc(0)};
  if (wid) bcg_k3_rows<true, PRE>(a, alpha, omega, acc);
  else bcg_k3_rows<false, PRE>(a, alpha, omega, acc);
  block_sum<3, kBlock>(acc, reinterpret_cast<Acc*>(sm), blk);
  if (grid_sum(blk, 3, a.red, tot) && threadIdx.x == 0) {
    const int iters = si[0] + 1;
    S->iters = iters;
    const double mur = sqrt(tot[1]) / sc[0];
    S->mu_rec = mur;
    int check = 0, stop = 0;
    if (mur < sc[1]) {
      check = 1;
    } else if (sc[2] == 0.0) {
      S->conv = GSK_BREAKDOWN;
      stop = 1;
    } else {
      const double rho1 = tot[0], rn = sqrt(wid ? tot[1] : tot[2]);
      if (!(fabs(rho1) > sc[3] * sc[4] * rn)) {
        S->conv = GSK_BREAKDOWN;
        stop = 1;
      } else {
        S->beta = (rho1 / sc[5]) * (sc[6] / sc[2]);
        S->rho = rho1;
      }
    }
    if (!check && !stop && iters >= si[1]) {
      S->conv = GSK_MAXIT;
      stop = 1;
    }
    S->check = check;
    S->stop = stop;
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_k4(BcgArgs<T> a) {
  const BcgState* S = a.S;
  if (S->check || S->stop) return;
  using Acc = typename AccOf<T>::type;
  const Acc beta = (Acc)S->beta, omega = (Acc)S->omega;
  const T* __restrict__ r = a.r;
  const T* __restrict__ v = a.v;
  T* __restrict__ p = a.p;
  constexpr int R = Vec16<T>::R;
  BCG_VEC_LOOP(a, R) {
    if (i0 + R <= a.n) {
      const Vec16<T> pv = vload(p + i0), vv = vload(v + i0), rv = vload(r + i0);
      Vec16<T> po;
#pragma unroll
      for (int q = 0; q < R; ++q)
        po.v[q] = (T)fma(beta, fma(-omega, (Acc)vv.v[q], (Acc)pv.v[q]), (Acc)rv.v[q]);
      vstore(p + i0, po);
    } else {
      for (int i = i0; i < a.n; ++i) p[i] = (T)fma(beta, fma(-omega, (Acc)v[i], (Acc)p[i]), (Acc)r[i]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a, a.h_while, 1u);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_kt(BcgArgs<T> a) {
  BcgState* S = a.S;
  if (!(S->check || S->stop)) return;  // nothing to confirm yet
  __shared__ PipeSmem<T> pipe;
  __shared__ double blk[2], tot[2];
  double* sm = reinterpret_cast<double*>(&pipe);  // reduction scratch after the product
  const bool wid = S->w_identity;
  double acc[2] = {0.0, 0.0};
  spmv_rows_tma(a.rowptr, a.colidx, a.val, a.x, a.n, a.nnz, pipe, a.err, [&](int i, T ax) {
    const T t = a.b[i] - ax;
    a.t[i] = t;
    const double wt = wgt(a.w, wid, i) * (double)t;
    acc[0] = fma(wt, wt, acc[0]);
    acc[1] = fma((double)t, (double)t, acc[1]);
  });
  block_sum<2, kBlock>(acc, sm, blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    S->mu_true = sqrt(tot[0]) / S->mu0;
    S->tt_true = tot[1];
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) bcg_kr(BcgArgs<T> a) {
  BcgState* S = a.S;
  const int stop = S->stop, check = S->check;
  if (!(check || stop)) return;  // nothing to confirm yet
  const bool met = S->mu_true < S->tol;
  const bool refresh = !stop && check && !met && S->refresh_left > 0 && *(volatile int*)a.err == 0;
  if (refresh) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < a.n; i += gridDim.x * kBlock) {
      const T t = a.t[i];
      a.r[i] = t;
      a.rh[i] = t;
      a.p[i] = t;
    }
  }
  if (grid_last(a.cnt) && threadIdx.x == 0) {
    int active = 0;
    if (!stop && check) {
      if (met) {
        S->conv = GSK_CONVERGED;
      } else if (refresh) {
        S->refresh_left -= 1;
        S->refreshes += 1;
        S->rho = S->tt_true;
        S->rhn = sqrt(S->tt_true);
        S->check = 0;
        S->halfexit = 0;
        if (S->iters >= S->maxit) {
          S->conv = GSK_MAXIT;
        } else {
          active = 1;
        }
      } else {
        S->conv = GSK_STAGNATED;
      }
    }
    S->stop = !active;
    S->active = active;
    set_cond(a, a.h_while, (unsigned)active);
  }
}

}  // namespace gsk
