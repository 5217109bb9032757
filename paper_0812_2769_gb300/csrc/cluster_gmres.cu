// Restarted GMRES(m) with classical Gram-Schmidt applied twice (Sec. 2) for
// small systems on one thread-block cluster: the whole solve in one launch
// of kClusterCtas CTAs that share their shared memory.
//
// Why: on a system of a few thousand rows the grid-wide solver spends an
// Arnoldi step in four kernel boundaries (launch ramp, the closing of each
// cross-block sum): about 36 us per step on a 1,024-row system whose step is
// ~100 thousand FP64 operations.  Here every CTA keeps its rows of the basis
// V, of x and of the metric weights in shared memory (and its rows of the
// matrix, staged once), the products gather the other CTAs' entries through
// distributed shared memory, and each kernel boundary becomes one hardware
// cluster barrier (cluster.cuh).
//
// The recurrences and every decision are those of the grid-wide solver
// (gmres_kernels.cuh), in the same order: unnormalised basis columns with
// scales sig (v_c = sig[c] V[:, c]); CGS pass 1 (h1), pass 2 (w -= V h1,
// h2), pass 3 (w -= V h2, ||w||); the Hessenberg column h1 + h2, the earlier
// rotations, the new rotation and g; the cycle ends when |g_{j+1}| < tau
// ||r0||, at numerical breakdown h_{j+1,j} <= hbrk ||A v_j||, after m steps
// or at maxit; then the back substitution, x += V (sig .* y) and the true
// metric, which decides convergence, with tau tightened by tol / metric
// when the estimate met tau but the metric did not.  Only the order of the
// additions inside the sums differs, and the scalar recurrences multiply by
// reciprocals and compare squares where the grid-wide solver divides and
// takes roots (a lone thread's FP64 operation waits its whole latency on this
// part).  The Hessenberg columns are kept rotated (the triangle R of the
// least-squares problem), one copy per CTA: every CTA does the scalar work
// itself on identical totals.
#include <algorithm>
#include <cfloat>

#include "cluster.cuh"

namespace gsk {

struct ClusterGmArgs {
  int n, nnz, rpc, m;
  const int* rowptr;
  const int* colidx;
  const double* val;
  const double* b;
  double* x;
  const double* wglob;  // metric weights from the caller, or null
  int wmode;            // 0: GS(2) weights of A (identity if within 4 ulp), 1: none, 2: wglob
  double tol, hbrk;
  int maxit;
  int cap;              // matrix entries a CTA stages in shared memory
  gsk_info* out;        // device: the outcome
  int* err;             // device: kErr* bits
};

// Doubles of dynamic shared memory besides the matrix stage: the basis
// (m + 1 columns of rpc rows), x and the weights, the publication buffers
// and totals, and the small vectors of the least-squares problem.
__host__ __device__ inline long long gm_cluster_doubles(int rpc, int m) {
  const long long M1 = m + 1;
  return M1 * rpc + 2LL * rpc + 2 * M1 + 16 + 64 + 6 * M1 + 2LL * m + (m + 2) + (long long)m * (m + 1) / 2 + m;
}

// Dot products of w with the first k basis columns, summed over the cluster:
// tot[c] = sum over every row i of V[c][i] w[i], c < k.  Warp q of the CTA
// takes columns q, q + 16, ..., each lane a fixed strided set of the CTA's
// rows, then a fixed shuffle tree; the CTAs' partials meet as in
// cluster_sum (redk: two publication buffers of m + 1 values, alternating
// by `round`).
__device__ __forceinline__ void cluster_multidot(cg::cluster_group& cl, const double* V, const double* w, int rpc,
                                                 int nloc, int k, double* redk, int M1, double* tot, int& round) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* mine = redk + (round & 1) * M1;
  for (int c = wid; c < k; c += kClusterThreads / 32) {
    const double* vc = V + (long long)c * rpc;
    double s = 0.0;
    for (int li = lane; li < nloc; li += 32) s = fma(vc[li], w[li], s);
    s = warp_allsum(s);
    if (lane == 0) mine[c] = s;
  }
  cl.sync();
  for (int c = threadIdx.x; c < k; c += kClusterThreads) tot[c] = cluster_gather_sum(cl, mine, c);
  __syncthreads();
  round += 1;
}

__global__ void __launch_bounds__(kClusterThreads, 1) gm_cluster(ClusterGmArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double gc_dyn[];
  const int rpc = a.rpc, n = a.n, m = a.m, M1 = m + 1;
  double* V = gc_dyn;                 // M1 * rpc
  double* xs = V + (long long)M1 * rpc;
  double* ws = xs + rpc;
  double* redk = ws + rpc;            // 2 * M1
  double* red = redk + 2 * M1;        // 16: cluster_sum's buffers
  double* wsum = red + 16;            // 64
  double* tot = wsum + 64;            // M1
  double* h1 = tot + M1;
  double* h2 = h1 + M1;
  double* cf = h2 + M1;               // coefficients of the current update
  double* sig = cf + M1;
  double* g = sig + M1;
  double* csn = g + M1;               // m
  double* snn = csn + m;              // m
  double* hs = snn + m;               // m + 2
  double* R = hs + (m + 2);           // m (m + 1) / 2: column j at j (j + 1) / 2
  double* y = R + (long long)m * (m + 1) / 2;  // m
  double* sval = y + m;               // cap
  int* srp = reinterpret_cast<int*>(sval + a.cap);
  int* scol = srp + rpc + 1;
  const int rank = (int)cl.block_rank();
  const int row0 = rank * rpc;
  const int nloc = max(0, min(rpc, n - row0));
  const int nw = (min(nloc, kClusterThreads) + 31) / 32;  // warps that hold rows
  int round = 0, kround = 0;
  const int e0 = nloc > 0 ? __ldg(a.rowptr + row0) : 0;
  const int e1 = nloc > 0 ? __ldg(a.rowptr + row0 + nloc) : 0;
  const bool staged = e0 >= 0 && e1 >= e0 && e1 <= a.nnz && e1 - e0 <= a.cap;
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

  // (A vec)_i for local row li, vec distributed like the rows (this CTA's
  // part), in the row's column order
  auto rowprod = [&](int li, const double* vec) -> double {
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
      if ((unsigned)j < (unsigned)n) {
        const int o = j / rpc, l = j - o * rpc;
        xv = o == rank ? vec[l] : cl.map_shared_rank(vec, o)[l];
      }
      sum = fma(__ldg(a.val + k), xv, sum);
    }
    return sum;
  };
#define GC_ROWS(li) for (int li = threadIdx.x; li < nloc; li += kClusterThreads)

  // ---- set-up: structure checks, metric weights, x0
  double nbad = 0.0, nfar = 0.0;
  GC_ROWS(li) {
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

  __shared__ struct {
    double mu0, rho0, inv_rho0, tau, est, mu_true;
    int iters, restarts, conv, kcols, est_hit, j, cont, stop;
  } sc;
  bool first = true;
  for (;;) {
    // ---- r = b - A x into V[:, 0]; the true metric; start or restart a cycle
    {
      double acc0 = 0.0, acc1 = 0.0;
      GC_ROWS(li) {
        const double r = __ldg(a.b + row0 + li) - rowprod(li, xs);
        V[li] = r;
        const double wr = (wid ? 1.0 : ws[li]) * r;
        acc0 = fma(wr, wr, acc0);
        acc1 = fma(r, r, acc1);
      }
      const double v2[2] = {acc0, acc1};
      cluster_sum<2>(cl, v2, red, wsum, tot, round, nw);  // also publishes V[:, 0]
    }
    if (threadIdx.x == 0) {
      const double rn = sqrt(tot[1]);
      int stop = 0;
      if (first) {
        sc.mu0 = sqrt(tot[0]);
        sc.rho0 = rn;
        sc.inv_rho0 = 1.0 / rn;
        sc.iters = 0;
        sc.restarts = 0;
        sc.tau = a.tol;
        sc.conv = GSK_MAXIT;
        sc.mu_true = 1.0;
        sc.est = 1.0;
        sc.kcols = 0;
        if (err0) {
          stop = 1;
        } else if (!isfinite(sc.mu0)) {
          if (rank == 0) atomicOr(a.err, kErrNonFinite);
          stop = 1;
        } else if (sc.mu0 == 0.0) {
          sc.conv = GSK_CONVERGED;
          sc.mu_true = 0.0;
          sc.est = 0.0;
          stop = 1;
        } else if (a.maxit <= 0) {
          stop = 1;
        }
      } else {
        const double mu = sqrt(tot[0]) / sc.mu0;
        sc.mu_true = mu;
        if (mu < a.tol) {
          sc.conv = GSK_CONVERGED;
          stop = 1;
        } else if (sc.iters >= a.maxit || sc.kcols == 0) {
          sc.conv = GSK_MAXIT;
          stop = 1;
        } else {
          if (sc.est_hit) sc.tau = sc.tau * (a.tol / mu);
          sc.restarts += 1;
        }
      }
      if (!stop) {
        sig[0] = 1.0 / rn;
        g[0] = rn;
        for (int q = 1; q <= m; ++q) g[q] = 0.0;
        sc.j = 0;
        sc.est_hit = 0;
        sc.kcols = 0;
      }
      sc.stop = stop;
    }
    __syncthreads();
    first = false;
    if (sc.stop) break;

    // ---- the cycle's Arnoldi steps
    bool ahead = false;  // this step's product was formed during the last step
    for (;;) {
      const int j = sc.j, k = j + 1;
      const double* vj = V + (long long)j * rpc;
      double* w = V + (long long)(j + 1) * rpc;
      const double sj = sig[j];
      // w = A v_j = sig[j] (A V[:, j]); A V[:, j] may already be in w
      if (ahead) {
        GC_ROWS(li) w[li] = sj * w[li];
      } else {
        GC_ROWS(li) w[li] = sj * rowprod(li, vj);
      }
      __syncthreads();
      // pass 1: h1 = sig .* (V_k^T w)
      cluster_multidot(cl, V, w, rpc, nloc, k, redk, M1, tot, kround);
      for (int c = threadIdx.x; c < k; c += kClusterThreads) {
        h1[c] = sig[c] * tot[c];
        cf[c] = sig[c] * h1[c];
      }
      __syncthreads();
      // pass 2: w -= V_k (sig .* h1); h2 = sig .* (V_k^T w)
      GC_ROWS(li) {
        double wi = w[li];
        for (int c = 0; c < k; ++c) wi = fma(-V[(long long)c * rpc + li], cf[c], wi);
        w[li] = wi;
      }
      __syncthreads();
      cluster_multidot(cl, V, w, rpc, nloc, k, redk, M1, tot, kround);
      for (int c = threadIdx.x; c < k; c += kClusterThreads) {
        h2[c] = sig[c] * tot[c];
        cf[c] = sig[c] * h2[c];
      }
      __syncthreads();
      // pass 3: w -= V_k (sig .* h2); ||w||^2
      {
        double an = 0.0;
        GC_ROWS(li) {
          double wi = w[li];
          for (int c = 0; c < k; ++c) wi = fma(-V[(long long)c * rpc + li], cf[c], wi);
          w[li] = wi;
          an = fma(wi, wi, an);
        }
        const double v1[1] = {an};
        cluster_sum<1>(cl, v1, red, wsum, tot, round, nw);  // also publishes V[:, j+1]
      }
      // Meanwhile warps 1.. form the next step's product A V[:, j+1] (the
      // column is final and visible, and its scale sig[j+1] only multiplies
      // the sums) in V[:, j+2]; if the cycle ends here it is not used
      ahead = j + 2 <= m;
      if (ahead && threadIdx.x >= 32) {
        double* wn = V + (long long)(j + 2) * rpc;
        for (int li = threadIdx.x - 32; li < nloc; li += kClusterThreads - 32) wn[li] = rowprod(li, w);
      }
      // the Hessenberg column, the rotations and the cycle's tests: warp 0
      // forms h = h1 + h2 and ||h||^2 across its lanes; lane 0 applies the
      // earlier rotations (a chain through the one carried entry, each
      // rotated entry stored straight into R), forms the new rotation and
      // takes the decisions.  A lone thread's FP64 operation waits its full
      // latency on this part, so the chain keeps few of them: squared
      // comparisons instead of roots, one reciprocal for c and s, and
      // sqrt(a^2 + b^2) for hypot(a, b) where the squares are safe
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double part = 0.0;
        for (int c = lane; c <= j; c += 32) {
          const double h = h1[c] + h2[c];
          hs[c] = h;
          part = fma(h, h, part);
        }
        const double hh = warp_allsum(part);  // ||h1 + h2||^2
        __syncwarp();
        if (lane == 0) {
          const double hn2 = tot[0];
          const double hnext = sqrt(hn2);
          const double inv_hnext = 1.0 / hnext;
          // ||A v_j||^2 = ||h1 + h2||^2 + hnext^2 (w's parts along the
          // orthonormal basis and orthogonal to it)
          const double aw2 = hh + hn2;
          sc.iters += 1;
          double* rc = R + (long long)j * (j + 1) / 2;
          double hq = hs[0];
          for (int q = 0; q < j; ++q) {
            const double c = csn[q], s = snn[q], hn = hs[q + 1];
            rc[q] = c * hq + s * hn;
            hq = -s * hq + c * hn;
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
          csn[j] = c_;
          snn[j] = s_;
          rc[j] = rho;
          const double gj = g[j];
          g[j + 1] = -s_ * gj;
          g[j] = c_ * gj;
          const double est = fabs(g[j + 1]) * sc.inv_rho0;
          sc.est = est;
          sc.kcols = k;
          int cont = 1;
          if (est < sc.tau) {
            sc.est_hit = 1;
            cont = 0;
          } else if (hn2 <= a.hbrk * a.hbrk * aw2) {  // hnext <= hbrk ||A v_j||
            cont = 0;
          } else if (k >= m || sc.iters >= a.maxit) {
            cont = 0;
          }
          if (cont) {
            sig[j + 1] = inv_hnext;
            sc.j = j + 1;
          }
          sc.cont = cont;
        }
      }
      __syncthreads();
      if (!sc.cont) break;
    }

    // ---- the cycle's update: R y = g (back substitution), x += V (sig .* y)
    if (threadIdx.x == 0) {
      const int k = sc.kcols;
      for (int i = k - 1; i >= 0; --i) {
        double s = 0.0;
        for (int q = i + 1; q < k; ++q) s = fma(R[(long long)q * (q + 1) / 2 + i], y[q], s);
        y[i] = (g[i] - s) / R[(long long)i * (i + 1) / 2 + i];
      }
      for (int c = 0; c < k; ++c) cf[c] = sig[c] * y[c];
    }
    __syncthreads();
    {
      const int k = sc.kcols;
      GC_ROWS(li) {
        double xv = xs[li];
        for (int c = 0; c < k; ++c) xv = fma(V[(long long)c * rpc + li], cf[c], xv);
        xs[li] = xv;
      }
    }
    cl.sync();  // x visible to the residual's gathers
  }
  // ---- x back to global memory; the outcome
  GC_ROWS(li) a.x[row0 + li] = xs[li];
  if (rank == 0 && threadIdx.x == 0)
    *a.out = gsk_info{sc.iters, sc.restarts, 0, 0, sc.conv, sc.mu_true, sc.est, 0.f};
  cl.sync();  // no CTA leaves while another may still read its shared memory
#undef GC_ROWS
}

// ------------------------------------------------------------------ host

// Dynamic shared memory of the kernel on a device (0: a cluster of this
// shape does not fit), cached per device.
static int gm_cluster_smem(int device) {
  static int cache[64];  // 0: not looked up; -1: unavailable; else bytes
  if (device < 0 || device >= 64) return 0;
  if (cache[device] == 0) {
    const int s = cluster_smem_limit(gm_cluster, device);
    cache[device] = s > 0 ? s : -1;
  }
  return cache[device] > 0 ? cache[device] : 0;
}

// The matrix entries a CTA can stage beside everything else, for rpc rows
// and restart length m, in `smem` bytes.
static long long gm_cluster_cap(int rpc, int m, int smem) {
  const long long fixed = 8 * gm_cluster_doubles(rpc, m) + 4LL * (rpc + 1);
  return ((long long)smem - fixed) / 12;
}

// The cluster path is taken for systems of at most ctx->small_n rows whose
// basis fits and whose rows of the matrix are expected to fit each CTA's
// stage (an even split of the nonzeros with 25% to spare).
static bool gm_cluster_takes(gsk_ctx* ctx, int n, int nnz, int m) {
  if (n <= 0 || n > ctx->small_n) return false;
  const int smem = gm_cluster_smem(ctx->device);
  if (smem <= 0) return false;
  const int rpc = (n + kClusterCtas - 1) / kClusterCtas;
  const long long expect = (long long)nnz / kClusterCtas + nnz / (4 * kClusterCtas) + 64;
  return gm_cluster_cap(rpc, m, smem) >= expect;
}

// The most rows the cluster path takes with restart length m (for systems
// with about 7 nonzeros per row), 0 when it is off or unavailable.
int gm_cluster_rows(gsk_ctx* ctx, int m) {
  int lo = 0, hi = std::min(ctx->small_n, 1 << 20);
  while (lo < hi) {
    const int mid = lo + (hi - lo + 1) / 2;
    if (gm_cluster_takes(ctx, mid, 7 * mid, m)) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// GMRES(m) on one cluster when the system is small enough (FP64, no
// preconditioner).  *used = false: not taken, the caller runs the grid-wide
// solver.
gsk_status gm_cluster_solve(gsk_ctx* ctx, const gsk_csr* A, const void* b, void* x, int m, double tol,
                            const gsk_opts& opts, gsk_info* info, cudaStream_t st, bool* used) {
  *used = false;
  if (A->dtype != GSK_F64 || opts.precision != GSK_PREC_F64 || opts.precond || A->n <= 0) return GSK_OK;
  if (!(tol >= 0.0) || opts.maxit < 0 || m < 1 || m > kMaxM) return GSK_OK;  // the caller reports it
  if (!b || !x) return GSK_OK;
  if (!gm_cluster_takes(ctx, A->n, A->nnz, m)) return GSK_OK;
  *used = true;
  Arena sz;
  sz.take<int>(64);
  sz.take<gsk_info>(1);
  gsk_status s = ctx->reserve(sz.off);
  if (s != GSK_OK) return s;
  Arena ar{(char*)ctx->ws, ctx->ws_bytes, 0};
  int* err = ar.take<int>(64);
  gsk_info* dout = ar.take<gsk_info>(1);
  const int smem = gm_cluster_smem(ctx->device);
  ClusterGmArgs a;
  a.n = A->n;
  a.nnz = A->nnz;
  a.rpc = (A->n + kClusterCtas - 1) / kClusterCtas;
  a.m = m;
  a.rowptr = A->rowptr;
  a.colidx = A->colidx;
  a.val = (const double*)A->val;
  a.b = (const double*)b;
  a.x = (double*)x;
  a.wglob = opts.weights;
  a.wmode = opts.weights ? 2 : (opts.metric == GSK_METRIC_PLAIN ? 1 : 0);
  a.tol = tol;
  a.hbrk = 1e-14;
  a.maxit = opts.maxit;
  a.cap = (int)std::min<long long>(gm_cluster_cap(a.rpc, m, smem), 1 << 30);
  a.out = dout;
  a.err = err;
  GSK_CK(cudaEventRecord(ctx->ev0, st));
  GSK_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  GSK_CK(cluster_launch(gm_cluster, a, (size_t)smem, st));
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

extern "C" gsk_status gsk_gmres_small_system_rows(gsk_ctx* ctx, int m, int* rows) {
  if (!ctx || !rows || m < 1 || m > gsk::kMaxM) return GSK_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ctx->fail(GSK_ERR_CUDA, "cudaSetDevice");
  *rows = gsk::gm_cluster_rows(ctx, m);
  return GSK_OK;
}
