// Restarted GMRES(m) with classical Gram-Schmidt applied twice (Sec. 2),
// with the Arnoldi process, the Givens rotations, the Hessenberg
// least-squares solve and every stopping decision on the device.
//
// Basis storage: V is column-major (leading dimension ldv) and column k holds
// an unnormalised vector; the Arnoldi vector is v_k = sig[k] * V[:, k].  The
// scale is folded into the next product instead of a separate normalisation
// pass over V.
//
// One Arnoldi step j (k = j + 1 basis vectors) is four kernels:
//   ga  w = A v_j -> V[:, j+1];  ||w||                           (SpMV)
//   gd  h1 = V_k^T w                                             (CGS pass 1, multi-dot)
//   gb  w -= V_k h1;             h2 = V_k^T w                    (CGS pass 2)
//   gc  w -= V_k h2;             ||w||  -> column j of H = h1 + h2,
//       h_{j+1,j} = ||w||, earlier rotations applied, new rotation, g update,
//       convergence / breakdown tests                           (device scalar work)
// A cycle ends in
//   gy  back substitution H y = g (one block)
//   gx  x += V_k y
//   gr  r = b - A x -> V[:, 0]; true metric; restart or stop
// The steps form an inner WHILE node and the cycles an outer WHILE node of a
// CUDA graph, so a whole solve is one graph launch.
//
// Stopping (Sec. 2.2): a cycle ends when |g_{j+1}| < tau * ||r0|| (the
// least-squares residual relative to the initial residual), at numerical
// breakdown h_{j+1,j} <= hbrk ||A v_j|| (hbrk = 1e-14 in FP64; ||A v_j|| from
// the CGS coefficients and h_{j+1,j}, equal to the direct norm up to rounding), after m
// steps, or at maxit.  The
// true metric ||W(b - Ax)|| / ||W(b - Ax0)|| (W = GS(2) scales of A) decides
// convergence; if the estimate met tau but the metric did not, tau is
// tightened by tol / metric before the restart.
#pragma once

#include <cfloat>

#include "internal.hpp"
#include "spmv_tma.cuh"

namespace gsk {

struct GmState {
  double rho0, mu0, tau, tol, est, mu_true, inv_rho0, hbrk;
  int m, maxit, iters, restarts, conv, j, kcols, stop, est_hit, w_identity, cont;
};

template <typename T>
struct GmArgs {
  int n, nnz, m;
  long long ldv;
  const int* rowptr;
  const int* colidx;
  const T* val;
  const T* b;
  T* x;
  T* V;
  double *H, *g, *cs, *sn, *y, *h1, *h2, *sig;
  const double* w;
  GmState* S;
  GridRed red;
  unsigned* cnt;
  int* err;
  cudaGraphConditionalHandle h_outer, h_inner;
  int in_graph;
  int vec_ok;  // x is 16-byte aligned: 128-bit loads in the x update
  // right preconditioning (x = M^-1 u): the product of a step takes
  // zin = M^-1 v_j instead of v_j, and the cycle's update V (sig .* y) goes
  // to u_out (then x += M^-1 u_out); both null without a preconditioner
  const T* zin;
  T* u_out;
  // Arnoldi mode: gm_gc also stores each Hessenberg column before the Givens
  // rotations ((m+1) x m, column-major); null in the solvers
  double* Hraw;
  // unrolled cycle: the graph holds the m steps of a cycle as a chain (step j
  // with the basis kernels of class gm_kclass(j + 1)) instead of an inner
  // WHILE node; once the cycle has ended (S->cont == 0) the remaining steps'
  // kernels return at entry
  int unrolled;
};

// Basis-kernel class of a step with k columns: the kernels of class c hold
// per-column accumulators for up to kGmClassKP[c] columns, so small k runs
// with few registers and many resident blocks.
constexpr int kGmClasses = 5;
constexpr int kGmClassKP[kGmClasses] = {4, 8, 16, 32, 64};
__host__ __device__ __forceinline__ int gm_kclass(int k) {
  return k <= 4 ? 0 : (k <= 8 ? 1 : (k <= 16 ? 2 : (k <= 32 ? 3 : 4)));
}

template <typename T>
__device__ __forceinline__ void gm_set_cond(const GmArgs<T>& a, cudaGraphConditionalHandle h, unsigned v) {
  if (a.in_graph) cudaGraphSetConditional(h, v);
}

#define GM_ROW_LOOP(a) for (int i = blockIdx.x * kBlock + threadIdx.x; i < (a).n; i += gridDim.x * kBlock)

__device__ __forceinline__ double gm_wgt(const double* w, bool wid, int i) { return wid ? 1.0 : __ldg(w + i); }

// Block sum of NV register accumulators (only the first nv are needed), in
// chunks of 16 rows of a [min(NV, 16)][kBlock] shared table, added in the
// accumulators' type: FP64 for the FP64 solver; FP32 for the FP32 inner
// solves, whose per-thread sums are FP32 already (an FP64 tree there would
// spend the scarce FP64 pipe on k x 255 additions per block).  The block
// totals go on to the grid-wide sum in FP64.
template <int NV>
__host__ __device__ constexpr int chunk_rows() { return NV < 16 ? NV : 16; }
template <int NV, typename A>
__device__ __forceinline__ void block_sum_chunked(const A (&v)[NV], int nv, A* table, double* res) {
#pragma unroll
  for (int c0 = 0; c0 < NV; c0 += 16) {
    if (c0 < nv) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (c0 + q < NV) table[q * kBlock + threadIdx.x] = v[c0 + q];
      block_sum_table<kBlock>(table, min(16, nv - c0), res + c0);
    }
  }
}

template <typename T>
union GmSmem {
  PipeSmem<T> pipe;
  double table[16 * kBlock];
};

// r = b - A x into V[:, 0]; the true metric; start (init) or restart a cycle.
template <typename T, bool INIT>
__global__ void __launch_bounds__(kBlock) gm_residual(GmArgs<T> a) {
  __shared__ GmSmem<T> sm;
  __shared__ double blk[2], tot[2];
  GmState* S = a.S;
  const bool wid = S->w_identity;
  double acc[2] = {0.0, 0.0};
  spmv_rows_tma(a.rowptr, a.colidx, a.val, a.x, a.n, a.nnz, sm.pipe, a.err, [&](int i, T ax) {
    const T r = a.b[i] - ax;
    a.V[i] = r;
    const double wr = gm_wgt(a.w, wid, i) * (double)r;
    acc[0] = fma(wr, wr, acc[0]);
    acc[1] = fma((double)r, (double)r, acc[1]);
  });
  block_sum_chunked<2>(acc, 2, sm.table, blk);
  if (grid_sum(blk, 2, a.red, tot) && threadIdx.x == 0) {
    const int e = *(volatile int*)a.err;
    const double rn = sqrt(tot[1]);
    int stop = 0;
    if (INIT) {
      const double mu0 = sqrt(tot[0]);
      S->mu0 = mu0;
      S->rho0 = rn;
      S->inv_rho0 = 1.0 / rn;
      S->iters = 0;
      S->restarts = 0;
      S->tau = S->tol;
      S->conv = GSK_MAXIT;
      S->mu_true = 1.0;
      S->est = 1.0;
      if (e) {
        stop = 1;
      } else if (!isfinite(mu0)) {
        atomicOr(a.err, kErrNonFinite);
        stop = 1;
      } else if (mu0 == 0.0) {
        S->conv = GSK_CONVERGED;
        S->mu_true = 0.0;
        S->est = 0.0;
        stop = 1;
      } else if (S->maxit <= 0) {
        stop = 1;
      }
    } else {
      const double mu = sqrt(tot[0]) / S->mu0;
      S->mu_true = mu;
      if (e) {
        stop = 1;
      } else if (mu < S->tol) {
        S->conv = GSK_CONVERGED;
        stop = 1;
      } else if (S->iters >= S->maxit || S->kcols == 0) {
        S->conv = GSK_MAXIT;
        stop = 1;
      } else {
        if (S->est_hit) S->tau = S->tau * (S->tol / mu);
        S->restarts += 1;
      }
    }
    if (!stop) {
      a.sig[0] = 1.0 / rn;
      a.g[0] = rn;
      for (int q = 1; q <= a.m; ++q) a.g[q] = 0.0;
      S->j = 0;
      S->est_hit = 0;
      S->kcols = 0;
    }
    S->stop = stop;
    S->cont = !stop;
    gm_set_cond(a, a.h_outer, (unsigned)!stop);
    if (!a.unrolled) gm_set_cond(a, a.h_inner, (unsigned)!stop);
  }
}

// Arnoldi step, product: w = A v_j stored in V[:, j+1].  No reduction here:
// the breakdown reference ||A v_j|| follows from the CGS coefficients and
// the final norm (Pythagoras over the orthonormal basis), taken in gm_gc.
template <typename T>
__global__ void __launch_bounds__(kBlock) gm_ga(GmArgs<T> a) {
  __shared__ PipeSmem<T> pipe;
  const GmState* S = a.S;
  if (a.unrolled && !S->cont) return;  // the cycle ended at an earlier step
  const int j = S->j;
  const T* vj = a.zin ? a.zin : a.V + (long long)j * a.ldv;
  T* __restrict__ wout = a.V + (long long)(j + 1) * a.ldv;
  using Acc = typename AccOf<T>::type;
  const Acc sj = (Acc)a.sig[j];
  spmv_rows_tma(a.rowptr, a.colidx, a.val, vj, a.n, a.nnz, pipe, a.err,
                [&](int i, T av) { wout[i] = (T)(sj * (Acc)av); });
}

// Row loop of the CGS passes: each thread takes R = 16/sizeof(T) consecutive
// rows (one 128-bit load per basis column); V's columns are 16-byte aligned
// (leading dimension a multiple of 64) and only the last partial group of
// rows takes the scalar path.
#define GM_VEC_LOOP(a, R)                                                                          \
  for (int i0 = (R) * (blockIdx.x * kBlock + threadIdx.x), vstride_ = (R) * gridDim.x * kBlock; \
       i0 < (a).n; i0 += vstride_)

// Calls f(c) for c = 0 .. k-1 in groups of four, c a compile-time constant
// after unrolling (so per-column accumulators stay in registers).  The
// ragged last group takes one uniform branch per count: no FP64 instruction
// is issued for a column c >= k (on this part a predicated-off FP64
// instruction still costs its pipe time).
template <int KP, typename F>
__device__ __forceinline__ void for_columns(int k, F&& f) {
#pragma unroll
  for (int c0 = 0; c0 < KP; c0 += 4) {
    if (c0 + 4 <= k) {
      f(c0);
      f(c0 + 1);
      f(c0 + 2);
      f(c0 + 3);
    } else if (c0 < k) {
      switch (k - c0) {
        case 3:
          f(c0);
          f(c0 + 1);
          f(c0 + 2);
          break;
        case 2:
          f(c0);
          f(c0 + 1);
          break;
        default:
          f(c0);
          break;
      }
    }
  }
}

// CGS pass 1: h1 = sig .* (V_k^T w).
template <typename T, int KP>
__global__ void __launch_bounds__(kBlock) gm_gd(GmArgs<T> a) {
  using Acc = typename AccOf<T>::type;
  constexpr int R = Vec16<T>::R;
  __shared__ Acc table[chunk_rows<KP>() * kBlock];
  __shared__ double res[KP], tot[KP];
  const GmState* S = a.S;
  if (a.unrolled && !S->cont) return;  // the cycle ended at an earlier step
  const int j = S->j, k = j + 1;
  const T* __restrict__ wv = a.V + (long long)(j + 1) * a.ldv;
  Acc acc[KP];
#pragma unroll
  for (int c = 0; c < KP; ++c) acc[c] = Acc(0);
  GM_VEC_LOOP(a, R) {
    if (i0 + R <= a.n) {
      const Vec16<T> w = vload(wv + i0);
      for_columns<KP>(k, [&](int c) {
        const Vec16<T> v = vload(a.V + (long long)c * a.ldv + i0);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[c] = fma((Acc)v.v[r], (Acc)w.v[r], acc[c]);
      });
    } else {
      for (int i = i0; i < a.n; ++i) {
        const Acc w = (Acc)wv[i];
        for (int c = 0; c < k; ++c)
#pragma unroll
          for (int q = 0; q < KP; ++q)
            if (q == c) acc[q] = fma((Acc)a.V[(long long)c * a.ldv + i], w, acc[q]);
      }
    }
  }
  block_sum_chunked<KP>(acc, k, table, res);
  if (grid_sum<(KP >= 16 ? 16 : 8)>(res, k, a.red, tot)) {
    for (int c = threadIdx.x; c < k; c += kBlock) a.h1[c] = a.sig[c] * tot[c];
  }
}

// CGS pass 2: w -= V_k (sig .* h1); h2 = sig .* (V_k^T w).
template <typename T, int KP>
__global__ void __launch_bounds__(kBlock) gm_gb(GmArgs<T> a) {
  using Acc = typename AccOf<T>::type;
  constexpr int R = Vec16<T>::R;
  __shared__ Acc coef[KP];
  __shared__ Acc table[chunk_rows<KP>() * kBlock];
  __shared__ double res[KP], tot[KP];
  const GmState* S = a.S;
  if (a.unrolled && !S->cont) return;  // the cycle ended at an earlier step
  const int j = S->j, k = j + 1;
  T* wv = a.V + (long long)(j + 1) * a.ldv;
  for (int c = threadIdx.x; c < k; c += kBlock) coef[c] = (Acc)(a.sig[c] * a.h1[c]);
  __syncthreads();
  Acc acc[KP];
#pragma unroll
  for (int c = 0; c < KP; ++c) acc[c] = Acc(0);
  GM_VEC_LOOP(a, R) {
    if (i0 + R <= a.n) {
      const Vec16<T> w0 = vload(wv + i0);
      Acc w[R];
#pragma unroll
      for (int r = 0; r < R; ++r) w[r] = (Acc)w0.v[r];
      for_columns<KP>(k, [&](int c) {
        const Vec16<T> v = vload(a.V + (long long)c * a.ldv + i0);
#pragma unroll
        for (int r = 0; r < R; ++r) w[r] = fma(-(Acc)v.v[r], coef[c], w[r]);
      });
      Vec16<T> wt;
#pragma unroll
      for (int r = 0; r < R; ++r) wt.v[r] = (T)w[r];
      vstore(wv + i0, wt);
      for_columns<KP>(k, [&](int c) {
        const Vec16<T> v = vload(a.V + (long long)c * a.ldv + i0);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[c] = fma((Acc)v.v[r], (Acc)wt.v[r], acc[c]);
      });
    } else {
      for (int i = i0; i < a.n; ++i) {
        Acc w = (Acc)wv[i];
        for (int c = 0; c < k; ++c) w = fma(-(Acc)a.V[(long long)c * a.ldv + i], coef[c], w);
        const T wt = (T)w;
        wv[i] = wt;
        for (int c = 0; c < k; ++c)
#pragma unroll
          for (int q = 0; q < KP; ++q)
            if (q == c) acc[q] = fma((Acc)a.V[(long long)c * a.ldv + i], (Acc)wt, acc[q]);
      }
    }
  }
  block_sum_chunked<KP>(acc, k, table, res);
  if (grid_sum<(KP >= 16 ? 16 : 8)>(res, k, a.red, tot)) {
    for (int c = threadIdx.x; c < k; c += kBlock) a.h2[c] = a.sig[c] * tot[c];
  }
}

// CGS pass 3: w -= V_k (sig .* h2); ||w||; then the Hessenberg column, the
// Givens rotations and the cycle's stopping tests.
//
// Every block stages, at entry, what the closing block will need (the
// column h = h1 + h2, the earlier rotations, g_j and the state's scalars):
// the loads are a few hundred bytes per block from L2 and complete during
// the pass, so the closing block starts its scalar work with no memory
// round trip.  There warp 0 forms ||h||^2 and the products c_q h_{q+1}
// across its lanes while warp 1 forms hnext = ||w|| and 1/hnext; lane 0 of
// warp 0 then applies the earlier rotations as a chain of one FMA per
// rotation through the one carried entry (the rotated entries themselves are
// formed afterwards by all threads at once), forms the new rotation and
// takes the decisions.  A lone thread's FP64 instruction waits its full
// latency on this part, so the chain keeps few of them: squared comparisons
// instead of roots, one reciprocal for c and s, 1/rho0 kept in the state,
// and sqrt(a^2 + b^2) for hypot(a, b) where the squares are safe.
struct GcStage {
  double gj, inv_rho0, tau, hbrk, hh, hnext, inv_hnext;
  int iters, maxit, err;
};

template <typename T, int KP>
__global__ void __launch_bounds__(kBlock) gm_gc(GmArgs<T> a) {
  using Acc = typename AccOf<T>::type;
  __shared__ Acc coef[KP];
  __shared__ double table[kBlock], res[1], tot[1];
  __shared__ double hs[kMaxM + 1], css[kMaxM], sns[kMaxM], chq[kMaxM], hcar[kMaxM];
  __shared__ GcStage st;
  GmState* S = a.S;
  if (a.unrolled && !S->cont) return;  // the cycle ended at an earlier step
  const int j = S->j, k = j + 1;
  T* wv = a.V + (long long)(j + 1) * a.ldv;
  for (int c = threadIdx.x; c < k; c += kBlock) {
    const double h2 = a.h2[c];
    coef[c] = (Acc)(a.sig[c] * h2);
    hs[c] = a.h1[c] + h2;
    if (c < j) {
      css[c] = a.cs[c];
      sns[c] = a.sn[c];
    }
  }
  if (threadIdx.x == 0) {
    st.gj = a.g[j];
    st.inv_rho0 = S->inv_rho0;
    st.tau = S->tau;
    st.hbrk = S->hbrk;
    st.iters = S->iters;
    st.maxit = S->maxit;
    st.err = *(volatile int*)a.err;  // set by earlier kernels only: this one flags nothing
  }
  __syncthreads();
  constexpr int R = Vec16<T>::R;
  Acc acc[1] = {Acc(0)};
  GM_VEC_LOOP(a, R) {
    if (i0 + R <= a.n) {
      const Vec16<T> w0 = vload(wv + i0);
      Acc w[R];
#pragma unroll
      for (int r = 0; r < R; ++r) w[r] = (Acc)w0.v[r];
      for_columns<KP>(k, [&](int c) {
        const Vec16<T> v = vload(a.V + (long long)c * a.ldv + i0);
#pragma unroll
        for (int r = 0; r < R; ++r) w[r] = fma(-(Acc)v.v[r], coef[c], w[r]);
      });
      Vec16<T> wt;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        wt.v[r] = (T)w[r];
        acc[0] = fma((Acc)wt.v[r], (Acc)wt.v[r], acc[0]);
      }
      vstore(wv + i0, wt);
    } else {
      for (int i = i0; i < a.n; ++i) {
        Acc w = (Acc)wv[i];
        for (int c = 0; c < k; ++c) w = fma(-(Acc)a.V[(long long)c * a.ldv + i], coef[c], w);
        const T wt = (T)w;
        wv[i] = wt;
        acc[0] = fma((Acc)wt, (Acc)wt, acc[0]);
      }
    }
  }
  const double accd[1] = {(double)acc[0]};
  block_sum<1, kBlock>(accd, table, res);
  if (!grid_sum(res, 1, a.red, tot)) return;
  // the closing block
  const int ld = a.m + 1;
  const double hn2 = tot[0];
  if (threadIdx.x < 32) {
    double part = 0.0;
    for (int c = threadIdx.x; c <= j; c += 32) {
      part = fma(hs[c], hs[c], part);
      if (c < j) chq[c] = css[c] * hs[c + 1];
      if (a.Hraw) a.Hraw[(long long)j * ld + c] = hs[c];
    }
    const double hh = warp_allsum(part);  // ||h1 + h2||^2
    if (threadIdx.x == 0) st.hh = hh;
  } else if (threadIdx.x == 32) {
    const double hnext = sqrt(hn2);
    st.hnext = hnext;
    st.inv_hnext = 1.0 / hnext;
    if (a.Hraw) a.Hraw[(long long)j * ld + j + 1] = hnext;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double* hcol = a.H + (long long)j * ld;
    const double hnext = st.hnext;
    // ||A v_j||^2 = ||h1 + h2||^2 + hnext^2 (w's parts along the orthonormal
    // basis and orthogonal to it)
    const double aw2 = st.hh + hn2;
    const int iters = st.iters + 1;
    S->iters = iters;
    double hq = hs[0];
    for (int q = 0; q < j; ++q) {
      hcar[q] = hq;  // the entry carried into rotation q
      hq = fma(-sns[q], hq, chq[q]);
    }
    const double r2 = fma(hq, hq, hn2);
    const double rho = (r2 > 1e-290 && r2 < 1e290) ? sqrt(r2) : hypot(hq, hnext);
    double c_, s_;
    if (rho == 0.0) {
      c_ = 1.0;
      s_ = 0.0;
    } else {
      const double inv = 1.0 / rho;
      c_ = hq * inv;
      s_ = hnext * inv;
    }
    a.cs[j] = c_;
    a.sn[j] = s_;
    hcol[j] = rho;
    hcol[j + 1] = 0.0;
    const double gj = st.gj;
    const double gn = -s_ * gj;
    a.g[j + 1] = gn;
    a.g[j] = c_ * gj;
    const double est = fabs(gn) * st.inv_rho0;
    S->est = est;
    S->kcols = k;
    int cont = 1;
    if (est < st.tau) {
      S->est_hit = 1;
      cont = 0;
    } else if (hn2 <= st.hbrk * st.hbrk * aw2) {  // hnext <= hbrk ||A v_j||
      cont = 0;
    } else if (k >= a.m || iters >= st.maxit || st.err) {
      cont = 0;
    }
    if (cont) {
      a.sig[j + 1] = st.inv_hnext;
      S->j = j + 1;
    }
    S->cont = cont;
    if (!a.unrolled) gm_set_cond(a, a.h_inner, (unsigned)cont);
  }
  __syncthreads();
  // the rotated entries of column j above the diagonal
  for (int q = threadIdx.x; q < j; q += kBlock) a.H[(long long)j * ld + q] = css[q] * hcar[q] + sns[q] * hs[q + 1];
}

// Back substitution H(0:k, 0:k) y = g(0:k), bottom row first, by one warp:
// the triangle is staged in shared memory and each row's sum is split over
// the lanes (a fixed shuffle tree).
template <typename T>
__global__ void gm_gy(GmArgs<T> a) {
  __shared__ double Hs[kMaxM * kMaxM];
  __shared__ double ys[kMaxM], gs[kMaxM];
  const int k = a.S->kcols, ld = a.m + 1, lane = lane_id();
  // the whole block stages the triangle (its loads in flight together), then
  // one warp solves
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int col = e / k, row = e - col * k;
    if (row <= col) Hs[row * kMaxM + col] = a.H[(long long)col * ld + row];
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) gs[i] = a.g[i];
  __syncthreads();
  if (threadIdx.x >= 32) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = 0.0;
    for (int q = i + 1 + lane; q < k; q += 32) s = fma(Hs[i * kMaxM + q], ys[q], s);
    s = warp_allsum(s);
    if (lane == 0) ys[i] = (gs[i] - s) / Hs[i * kMaxM + i];
    __syncwarp();
  }
  for (int i = lane; i < k; i += 32) a.y[i] = ys[i];
}

// x += V_k (sig .* y): two rows per thread (128-bit loads of every basis
// column; the caller's x must be 16-byte aligned for that, else scalar), the
// columns in order for each row.
template <typename T, int KP>
__global__ void __launch_bounds__(kBlock) gm_gx(GmArgs<T> a) {
  __shared__ double coef[KP];
  const int k = a.S->kcols;
  for (int c = threadIdx.x; c < k; c += kBlock) coef[c] = a.sig[c] * a.y[c];
  __syncthreads();
  constexpr int R = Vec16<T>::R;
  // without a preconditioner x += V (sig .* y); with one u = V (sig .* y)
  T* dst = a.u_out ? a.u_out : a.x;
  const bool add = a.u_out == nullptr;
  const bool vec = add ? a.vec_ok != 0 : true;  // u_out is workspace (aligned)
  GM_VEC_LOOP(a, R) {
    if (i0 + R <= a.n && vec) {
      double x[R];
      if (add) {
        const Vec16<T> x0 = vload(a.x + i0);
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = (double)x0.v[r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = 0.0;
      }
      for_columns<KP>(k, [&](int c) {
        const Vec16<T> v = vload(a.V + (long long)c * a.ldv + i0);
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = fma((double)v.v[r], coef[c], x[r]);
      });
      Vec16<T> xo;
#pragma unroll
      for (int r = 0; r < R; ++r) xo.v[r] = (T)x[r];
      vstore(dst + i0, xo);
    } else {
      for (int i = i0; i < min(i0 + R, a.n); ++i) {
        double x = add ? (double)a.x[i] : 0.0;
        for_columns<KP>(k, [&](int c) { x = fma((double)a.V[(long long)c * a.ldv + i], coef[c], x); });
        dst[i] = (T)x;
      }
    }
  }
}

// x += z (the preconditioned cycle's correction z = M^-1 V (sig .* y), in zin).
template <typename T>
__global__ void __launch_bounds__(kBlock) gm_xadd(GmArgs<T> a) {
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < a.n; i += gridDim.x * kBlock) a.x[i] += a.zin[i];
}

}  // namespace gsk
