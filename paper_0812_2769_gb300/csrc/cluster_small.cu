// Bi-CGSTAB (Sec. 2; van der Vorst 1992) for small systems on one thread-block
// cluster: the whole solve in one launch of kClusterCtas CTAs that share their
// shared memory (distributed shared memory, DSMEM).
//
// Why: a system of a few thousand rows is too small to fill the GPU, and the
// grid-wide solver then pays kernel boundaries (launch ramp, the closing of
// every cross-block sum) on each of its five kernels per iteration: about
// 28 us per iteration on a 1,024-row system, for ~30 thousand FP64 operations.
// A single block is no better: one SM's two FP64 lanes per clock need ~7 us
// for that work alone.  A cluster spreads the FP64 work over 16 SMs and
// replaces each kernel boundary by a hardware cluster barrier.
//
// Layout: CTA c owns rows [c * rpc, (c + 1) * rpc) (rpc = ceil(n / 16)); the
// iteration vectors x, r, r^, p, v, s, t of those rows live in its shared
// memory.  A product gathers the entries of p, s or x that other CTAs own
// through DSMEM (the matrix itself is read from global memory, where it stays
// L2-resident).  A dot product is summed per CTA (fixed warp and lane order),
// published in the CTA's shared memory, and after a cluster barrier every CTA
// adds the 16 partials in rank order: every CTA holds bit-identical scalars
// and takes the same decisions, with no further exchange.
//
// The arithmetic per row (the order of each product row, the FMA forms of the
// vector updates) and every decision (breakdown tests, the half-step exit,
// true-residual confirmation with refreshes, maxit, the metric weights) are
// those of the grid-wide solver (bicgstab_kernels.cuh); only the order of the
// additions inside the dot products differs.
#include <algorithm>
#include <cfloat>

#include "cluster.cuh"

namespace gsk {

constexpr int kClusterVecs = 8;     // x, r, r^, p, v, s, t, W in shared memory

struct ClusterBcgArgs {
  int n, nnz, rpc;  // rows per CTA
  const int* rowptr;
  const int* colidx;
  const double* val;
  const double* b;
  double* x;
  const double* wglob;  // metric weights from the caller, or null
  int wmode;            // 0: GS(2) weights of A (identity if within 4 ulp), 1: none, 2: wglob
  double tol, brk;
  int maxit, refresh;
  int cap;              // matrix entries a CTA stages in shared memory
  gsk_info* out;        // device: the outcome
  int* err;             // device: kErr* bits
};

// The solve.  One cluster; every CTA runs the same control flow on the same
// scalars.  Outcome and counts are written to a.out by rank 0.
__global__ void __launch_bounds__(kClusterThreads, 1) bcg_cluster(ClusterBcgArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double cs_dyn[];
  const int rpc = a.rpc, n = a.n;
  double* xs = cs_dyn;
  double* rs = xs + rpc;
  double* rhs = rs + rpc;
  double* ps = rhs + rpc;
  double* vs = ps + rpc;
  double* ss = vs + rpc;
  double* ts = ss + rpc;
  double* ws = ts + rpc;
  double* red = ws + rpc;  // [2][8] published partial sums
  double* wsum = red + 16;  // [16 warps][4]
  double* tot = wsum + 64;  // [8] totals
  // this CTA's rows of the matrix, staged once: values, then the local row
  // pointers and the columns packed as (owning CTA << 20 | local row)
  double* sval = tot + 8;
  int* srp = reinterpret_cast<int*>(sval + a.cap);
  int* scol = srp + rpc + 1;
  const int rank = (int)cl.block_rank();
  const int row0 = rank * rpc;
  const int nloc = max(0, min(rpc, n - row0));
  const int nw = (min(nloc, kClusterThreads) + 31) / 32;  // warps that hold rows
  int round = 0;
  const int e0 = nloc > 0 ? __ldg(a.rowptr + row0) : 0;
  const int e1 = nloc > 0 ? __ldg(a.rowptr + row0 + nloc) : 0;
  const bool staged = e0 >= 0 && e1 >= e0 && e1 <= a.nnz && e1 - e0 <= a.cap;
  // (a CTA that owns no row stages nothing: its row0 may lie past rowptr's
  // last entry)
  if (staged && nloc > 0) {
    for (int k = threadIdx.x; k < e1 - e0; k += kClusterThreads) {
      const int j = __ldg(a.colidx + e0 + k);
      const int o = (unsigned)j < (unsigned)n ? j / rpc : -1;
      scol[k] = o < 0 ? -1 : (o << 20) | (j - o * rpc);
      sval[k] = __ldg(a.val + e0 + k);
    }
    for (int li = threadIdx.x; li <= nloc; li += kClusterThreads) srp[li] = __ldg(a.rowptr + row0 + li) - e0;
  }
  __syncthreads();

  // entry j of a vector distributed like the rows (this CTA's part `mine`)
  auto gather = [&](double* mine, int j) -> double {
    const int o = j / rpc, l = j - o * rpc;
    if (o == rank) return mine[l];
    return cl.map_shared_rank(mine, o)[l];
  };
  // (A vec)_i for local row li, in the row's column order: from the staged
  // copy (the columns' owners decoded once), or from global memory when this
  // CTA's rows did not fit the stage
  auto rowprod = [&](int li, double* vec) -> double {
    double sum = 0.0;
    if (staged) {
      const int k0 = srp[li], k1 = srp[li + 1];
      if (k0 < 0 || k1 < k0 || k1 > e1 - e0) return sum;  // reported by the set-up check
#pragma unroll 4
      for (int k = k0; k < k1; ++k) {
        const int c = scol[k];
        double xv = 0.0;
        if (c >= 0) {
          const int o = c >> 20, l = c & 0xFFFFF;
          xv = o == rank ? vec[l] : cl.map_shared_rank(vec, o)[l];
        }
        sum = fma(sval[k], xv, sum);
      }
      return sum;
    }
    const int gi = row0 + li;
    const int k0 = __ldg(a.rowptr + gi), k1 = __ldg(a.rowptr + gi + 1);
    if (k0 < 0 || k1 < k0 || k1 > a.nnz) return sum;
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
      const int j = __ldg(a.colidx + k);
      double xv = 0.0;
      if ((unsigned)j < (unsigned)n) xv = gather(vec, j);
      sum = fma(__ldg(a.val + k), xv, sum);
    }
    return sum;
  };
#define CL_ROWS(li) for (int li = threadIdx.x; li < nloc; li += kClusterThreads)

  // ---- set-up: structure checks, metric weights, x0
  double nbad = 0.0, nfar = 0.0;
  CL_ROWS(li) {
    const int gi = row0 + li;
    const int k0 = __ldg(a.rowptr + gi), k1 = __ldg(a.rowptr + gi + 1);
    bool ok = k0 >= 0 && k1 >= k0 && k1 <= a.nnz && (!staged || (k0 >= e0 && k1 <= e1));
    if (ok)
      for (int k = k0; k < k1; ++k) ok = ok && (unsigned)__ldg(a.colidx + k) < (unsigned)n;
    if (!ok) {
      atomicOr(a.err, kErrIndex);
      nbad += 1.0;
    }
    double w = 1.0;
    if (a.wmode == 0 && ok) {
      w = row_inv_norm_pm<kP2>(a.val + k0, k1 - k0, 2.0, a.err);
      if (dbits(w) == 0ull) nbad += 1.0;  // zero row or non-finite entry
      // outside [1 - 4 eps, 1 + 4 eps]: the weights are not the identity
      const long long bw = (long long)dbits(w);
      const long long lo = __double_as_longlong(1.0 - 4.0 * 2.220446049250313e-16);
      const long long hi = __double_as_longlong(1.0 + 4.0 * 2.220446049250313e-16);
      nfar += (bw < lo || bw > hi) ? 1.0 : 0.0;
    } else if (a.wmode == 2) {
      w = __ldg(a.wglob + gi);
    }
    ws[li] = w;
    xs[li] = a.x[gi];
  }
  {
    const double v2[2] = {nbad, nfar};
    cluster_sum<2>(cl, v2, red, wsum, tot, round, nw);  // also publishes x0 to the cluster
  }
  const bool err0 = tot[0] != 0.0;
  const bool wid = a.wmode == 1 || (a.wmode == 0 && tot[1] == 0.0);

  // ---- r = b - A x0, r^ = p = r; mu0, rho
  double acc0 = 0.0, acc1 = 0.0;
  CL_ROWS(li) {
    const double r = __ldg(a.b + row0 + li) - rowprod(li, xs);
    rs[li] = r;
    rhs[li] = r;
    ps[li] = r;
    const double wr = (wid ? 1.0 : ws[li]) * r;
    acc0 = fma(wr, wr, acc0);
    acc1 = fma(r, r, acc1);
  }
  {
    const double v2[2] = {acc0, acc1};
    cluster_sum<2>(cl, v2, red, wsum, tot, round, nw);  // also publishes p
  }
  // The scalar recurrences and every decision are taken by thread 0 of each
  // CTA (from the totals, which are identical in every CTA) and broadcast
  // through shared memory: FP64 divisions and square roots repeated by all
  // 512 threads of 16 CTAs would cost more than the rest of an iteration.
  __shared__ struct {
    double mu0, inv_mu0, rho, rhn, alpha, omega, beta, mu_true, mu_rec;
    int iters, refreshes, refresh_left, conv, next;  // next: what the CTA does next
  } sc;
  enum { kNext = 0, kStop = 1, kHalf = 2, kUpdate = 3, kConfirm = 4, kRefresh = 5, kIterate = 6 };
  if (threadIdx.x == 0) {
    sc.mu0 = sqrt(tot[0]);
    sc.inv_mu0 = 1.0 / sc.mu0;
    sc.rho = tot[1];
    sc.rhn = sqrt(tot[1]);
    sc.iters = 0;
    sc.refreshes = 0;
    sc.refresh_left = a.refresh;
    sc.conv = GSK_MAXIT;
    sc.mu_true = 1.0;
    sc.mu_rec = 1.0;
    sc.next = kNext;
    if (err0) {
      sc.next = kStop;
    } else if (!isfinite(sc.mu0)) {
      if (rank == 0) atomicOr(a.err, kErrNonFinite);
      sc.next = kStop;
    } else if (sc.mu0 == 0.0) {
      sc.conv = GSK_CONVERGED;
      sc.mu_true = 0.0;
      sc.mu_rec = 0.0;
      sc.next = kStop;
    } else if (a.maxit <= 0) {
      sc.next = kStop;
    }
  }
  __syncthreads();
  bool confirmed = false;  // the loop ended with a true-residual check
  while (sc.next != kStop) {
    // v = A p; sigma = <r^, v>, ||v||
    {
      double a2 = 0.0, a3 = 0.0;
      CL_ROWS(li) {
        const double v = rowprod(li, ps);
        vs[li] = v;
        a2 = fma(rhs[li], v, a2);
        a3 = fma(v, v, a3);
      }
      const double v2[2] = {a2, a3};
      cluster_sum<2>(cl, v2, red, wsum, tot, round, nw);
    }
    if (threadIdx.x == 0) {
      const double sigma = tot[0], vn = sqrt(tot[1]);
      if (!(fabs(sigma) > a.brk * sc.rhn * vn)) {
        sc.conv = GSK_BREAKDOWN;
        sc.next = kStop;
      } else {
        sc.alpha = sc.rho / sigma;
      }
    }
    __syncthreads();
    if (sc.next == kStop) break;
    const double alpha = sc.alpha;
    // s = r - alpha v, then visible to the cluster
    CL_ROWS(li) ss[li] = fma(-alpha, vs[li], rs[li]);
    cl.sync();
    // t = A s; <t, s>, <t, t>, ||W s||
    {
      double b0 = 0.0, b1 = 0.0, b2 = 0.0;
      CL_ROWS(li) {
        const double t = rowprod(li, ss);
        ts[li] = t;
        const double si = ss[li];
        b0 = fma(t, si, b0);
        b1 = fma(t, t, b1);
        const double wsi = wid ? si : ws[li] * si;
        b2 = fma(wsi, wsi, b2);
      }
      const double v3[3] = {b0, b1, b2};
      cluster_sum<3>(cl, v3, red, wsum, tot, round, nw);
    }
    if (threadIdx.x == 0) {
      const double mus = sqrt(tot[2]) * sc.inv_mu0;
      if (mus < a.tol) {
        sc.iters += 1;
        sc.mu_rec = mus;
        sc.next = kHalf;
      } else if (!(tot[1] > 0.0)) {
        sc.conv = GSK_BREAKDOWN;
        sc.next = kStop;
      } else {
        sc.omega = tot[0] / tot[1];
        sc.next = kUpdate;
      }
    }
    __syncthreads();
    if (sc.next == kStop) break;
    if (sc.next == kHalf) {
      // half-step exit: x += alpha p; confirmed below
      CL_ROWS(li) xs[li] = fma(alpha, ps[li], xs[li]);
    } else {
      // x += alpha p + omega s; r = s - omega t; <r^, r>, ||W r||, ||r||
      const double omega = sc.omega;
      double c0 = 0.0, c1 = 0.0, c2 = 0.0;
      CL_ROWS(li) {
        const double si = ss[li];
        xs[li] = fma(omega, si, fma(alpha, ps[li], xs[li]));
        const double r = fma(-omega, ts[li], si);
        rs[li] = r;
        c0 = fma(rhs[li], r, c0);
        if (wid) {
          c1 = fma(r, r, c1);
        } else {
          const double wr = ws[li] * r;
          c1 = fma(wr, wr, c1);
          c2 = fma(r, r, c2);
        }
      }
      const double v3[3] = {c0, c1, c2};
      cluster_sum<3>(cl, v3, red, wsum, tot, round, nw);
      if (threadIdx.x == 0) {
        sc.iters += 1;
        const double mur = sqrt(tot[1]) * sc.inv_mu0;
        sc.mu_rec = mur;
        if (mur < a.tol) {
          sc.next = kConfirm;
        } else if (sc.omega == 0.0) {
          sc.conv = GSK_BREAKDOWN;
          sc.next = kStop;
        } else {
          const double rho1 = tot[0], rn = sqrt(wid ? tot[1] : tot[2]);
          if (!(fabs(rho1) > a.brk * sc.rhn * rn)) {
            sc.conv = GSK_BREAKDOWN;
            sc.next = kStop;
          } else {
            sc.beta = (rho1 * sc.alpha) / (sc.rho * sc.omega);
            sc.rho = rho1;
            sc.next = sc.iters >= a.maxit ? kStop : kIterate;
          }
        }
      }
      __syncthreads();
      if (sc.next == kStop) break;
      if (sc.next == kIterate) {
        // p = r + beta (p - omega v), then visible to the cluster
        const double beta = sc.beta;
        CL_ROWS(li) ps[li] = fma(beta, fma(-omega, vs[li], ps[li]), rs[li]);
        cl.sync();
        continue;
      }
    }
    // ---- the recursive residual met tol: confirm with t = b - A x
    cl.sync();  // x visible
    {
      double d0 = 0.0, d1 = 0.0;
      CL_ROWS(li) {
        const double t = __ldg(a.b + row0 + li) - rowprod(li, xs);
        ts[li] = t;
        const double wt = (wid ? 1.0 : ws[li]) * t;
        d0 = fma(wt, wt, d0);
        d1 = fma(t, t, d1);
      }
      const double v2[2] = {d0, d1};
      cluster_sum<2>(cl, v2, red, wsum, tot, round, nw);
    }
    if (threadIdx.x == 0) {
      sc.mu_true = sqrt(tot[0]) * sc.inv_mu0;
      if (sc.mu_true < a.tol) {
        sc.conv = GSK_CONVERGED;
        sc.next = kStop;
      } else if (sc.refresh_left == 0) {
        sc.conv = GSK_STAGNATED;
        sc.next = kStop;
      } else {
        sc.refresh_left -= 1;
        sc.refreshes += 1;
        sc.rho = tot[1];
        sc.rhn = sqrt(tot[1]);
        sc.next = kRefresh;
      }
    }
    __syncthreads();
    confirmed = true;
    if (sc.next == kStop) break;
    confirmed = false;
    // refresh: r = r^ = p = t
    CL_ROWS(li) {
      const double t = ts[li];
      rs[li] = t;
      rhs[li] = t;
      ps[li] = t;
    }
    if (sc.iters >= a.maxit) {  // (the same value in every thread)
      if (threadIdx.x == 0) sc.conv = GSK_MAXIT;
      __syncthreads();
      break;
    }
    cl.sync();  // p visible
  }
  // ---- the true residual of the returned x when the loop stopped without a
  // confirmation (breakdown, maxit), as the grid-wide solver reports it
  if (!confirmed && sc.conv != GSK_CONVERGED && !err0 && isfinite(sc.mu0) && sc.mu0 > 0.0) {
    cl.sync();
    double d0 = 0.0;
    CL_ROWS(li) {
      const double t = __ldg(a.b + row0 + li) - rowprod(li, xs);
      const double wt = (wid ? 1.0 : ws[li]) * t;
      d0 = fma(wt, wt, d0);
    }
    const double v1[1] = {d0};
    cluster_sum<1>(cl, v1, red, wsum, tot, round, nw);
    if (threadIdx.x == 0) sc.mu_true = sqrt(tot[0]) * sc.inv_mu0;
    __syncthreads();
  }
  // ---- x back to global memory; the outcome
  CL_ROWS(li) a.x[row0 + li] = xs[li];
  if (rank == 0 && threadIdx.x == 0)
    *a.out = gsk_info{sc.iters, 0, sc.refreshes, 0, sc.conv, sc.mu_true, sc.mu_rec, 0.f};
  cl.sync();  // no CTA leaves while another may still read its shared memory
#undef CL_ROWS
}


// Shared memory of the cluster kernel: the vectors of rpc rows, the
// reduction buffers, and a stage of cap matrix entries (12 bytes each) with
// the local row pointers.
static size_t bcg_cluster_smem(int rpc, int cap) {
  return sizeof(double) * ((size_t)kClusterVecs * rpc + 16 + 64 + 8 + cap) + sizeof(int) * ((size_t)rpc + 1 + cap);
}
// The largest stage that fits beside the vectors in `bytes` of shared memory.
static int bcg_cluster_cap(int rpc, size_t bytes) {
  const long long fixed = (long long)bcg_cluster_smem(rpc, 0);
  const long long cap = ((long long)bytes - fixed) / 12;
  return cap > 0 ? (int)cap : 0;
}

// Whether this context can launch the cluster kernel for n rows (cached per
// context: the attributes, and whether a 16-CTA cluster with the largest
// shared memory fits on the device).
static bool bcg_cluster_fits(gsk_ctx* ctx, int n) {
  if (ctx->cluster_max_n < 0) {
    ctx->cluster_max_n = 0;
    const int smem = cluster_smem_limit(bcg_cluster, ctx->device);
    if (smem <= 0) return false;
    ctx->cluster_smem = smem;
    const int rpc_max = (int)((smem / sizeof(double) - (16 + 64 + 8)) / (kClusterVecs + 1));
    ctx->cluster_max_n = rpc_max * kClusterCtas;
  }
  return n <= ctx->cluster_max_n && n <= ctx->small_n;
}

// The cluster path is taken only where a CTA's rows of the matrix are
// expected to fit its stage beside the vectors (an even split of the nonzeros
// with 25% to spare): unstaged, the products wait on global memory and the
// grid-wide solver is faster.
static bool bcg_cluster_takes(gsk_ctx* ctx, int n, int nnz) {
  if (!bcg_cluster_fits(ctx, n)) return false;
  const int rpc = (n + kClusterCtas - 1) / kClusterCtas;
  const long long expect = (long long)nnz / kClusterCtas + nnz / (4 * kClusterCtas) + 64;
  return bcg_cluster_cap(rpc, (size_t)ctx->cluster_smem) >= expect;
}

// Bi-CGSTAB on one cluster when the system is small enough (FP64, no
// preconditioner).  *used = false: not taken, the caller runs the grid-wide
// solver.
gsk_status bcg_cluster_solve(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, double tol,
                             const gsk_opts& opts, gsk_info* info, cudaStream_t st, bool* used) {
  *used = false;
  if (A->dtype != GSK_F64 || opts.precision != GSK_PREC_F64 || opts.precond || A->n <= 0) return GSK_OK;
  if (!(tol >= 0.0) || opts.maxit < 0 || opts.refresh < 0) return GSK_OK;  // the caller reports it
  if (!b || !x) return GSK_OK;
  if (!bcg_cluster_takes(ctx, A->n, A->nnz)) return GSK_OK;
  *used = true;
  Arena sz;
  sz.take<int>(64);
  sz.take<gsk_info>(1);
  gsk_status s = ctx->reserve(sz.off);
  if (s != GSK_OK) return s;
  Arena ar{(char*)ctx->ws, ctx->ws_bytes, 0};
  int* err = ar.take<int>(64);
  gsk_info* dout = ar.take<gsk_info>(1);
  ClusterBcgArgs a;
  a.n = A->n;
  a.nnz = A->nnz;
  a.rpc = (A->n + kClusterCtas - 1) / kClusterCtas;
  a.rowptr = A->rowptr;
  a.colidx = A->colidx;
  a.val = (const double*)A->val;
  a.b = (const double*)b;
  a.x = (double*)x;
  a.wglob = opts.weights;
  a.wmode = opts.weights ? 2 : (opts.metric == GSK_METRIC_PLAIN ? 1 : 0);
  a.tol = tol;
  a.brk = 1e-16 * DBL_EPSILON;
  a.maxit = opts.maxit;
  a.refresh = opts.refresh;
  a.cap = bcg_cluster_cap(a.rpc, (size_t)ctx->cluster_smem);
  a.out = dout;
  a.err = err;
  GSK_CK(cudaEventRecord(ctx->ev0, st));
  GSK_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  GSK_CK(cluster_launch(bcg_cluster, a, (size_t)ctx->cluster_smem, st));
  GSK_CK(cudaEventRecord(ctx->ev1, st));
  if (!info) return GSK_OK;
  char* hp = (char*)ctx->host_pinned;
  GSK_CK(cudaMemcpyAsync(hp, dout, sizeof(gsk_info), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaMemcpyAsync(hp + 512, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GSK_CK(cudaStreamSynchronize(st));
  std::memcpy(info, hp, sizeof(gsk_info));
  int bits = 0;
  std::memcpy(&bits, hp + 512, sizeof(int));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  info->ms = ms;
  return err_bits_status(ctx, bits);
}

}  // namespace gsk

extern "C" gsk_status gsk_small_system_rows(gsk_ctx* ctx, int* rows) {
  if (!ctx || !rows) return GSK_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ctx->fail(GSK_ERR_CUDA, "cudaSetDevice");
  *rows = gsk::bcg_cluster_fits(ctx, 1) ? std::min(ctx->cluster_max_n, ctx->small_n) : 0;
  return GSK_OK;
}
