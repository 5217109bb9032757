// Device-side building blocks shared by the GS, SpMV and Krylov kernels.
//
// Design notes for GB300 (sm_103a):
//  * FP64 arithmetic is scarce on this part (about two FP64 FMA lanes per SM
//    per clock), so every helper here keeps FP64 work proportional to the
//    useful work: row sums are accumulated by the thread that owns the row
//    (no shuffle tree per row), and reductions across threads spread the
//    additions over all 32 lanes of a warp.
//  * Reductions are deterministic: the assignment of rows to threads depends
//    only on (n, grid), and every sum is taken in a fixed order, so repeated
//    runs give bit-identical scalars.
//  * Cross-block sums use the "last block finishes" pattern, so no kernel
//    ever waits on another block and no spin loop exists.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gsk {

constexpr unsigned kFull = 0xffffffffu;

// error bits written by kernels into a device status word
enum : int { kErrIndex = 1, kErrZeroRow = 2, kErrNonFinite = 4, kErrTimeout = 8 };

// Scratch for one grid-wide reduction site.
struct GridRed {
  double* partials;    // [nv_max * maxgrid]
  unsigned* counters;  // [1], zero between uses
  int maxgrid;         // launches using this site must have gridDim.x <= maxgrid
};

// Per-thread accumulation type: FP64 data is accumulated in FP64; FP32 data
// (the inner solves of the mixed-precision path) in FP32, so that an FP32
// kernel does no FP64 work per element.  Grid sums are FP64.
template <typename T>
struct AccOf {
  using type = double;
};
template <>
struct AccOf<float> {
  using type = float;
};

// 16-byte vectors of consecutive entries (2 doubles or 4 floats) for
// 128-bit loads and stores on 16-byte aligned addresses.
template <typename T>
struct Vec16 {
  static constexpr int R = 16 / sizeof(T);
  T v[R];
} __attribute__((aligned(16)));

template <typename T>
__device__ __forceinline__ Vec16<T> vload(const T* p) {
  return *reinterpret_cast<const Vec16<T>*>(p);
}
template <typename T>
__device__ __forceinline__ void vstore(T* p, const Vec16<T>& x) {
  *reinterpret_cast<Vec16<T>*>(p) = x;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// Block-wide sum of nv per-thread values held in shared memory as
// tab[k * BLOCK + t] (the table is consumed), added in the table's type.
// Result in res[k] (shared), valid after the call.  Tree as in block_sum.
template <int BLOCK, typename TT>
__device__ __forceinline__ void block_sum_table(TT* tab, int nv, double* res) {
  __syncthreads();
#pragma unroll
  for (int s = BLOCK / 2; s >= 32; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < nv; ++k) tab[k * BLOCK + threadIdx.x] += tab[k * BLOCK + threadIdx.x + s];
    __syncthreads();
  }
  // the remaining 32 partial sums of each value: one warp per value
  for (int k = warp_id(); k < nv; k += BLOCK / 32) {
    const TT t = warp_allsum(tab[k * BLOCK + lane_id()]);
    if (lane_id() == 0) res[k] = (double)t;
  }
  __syncthreads();
}

// Block-wide sum of NV register values (all threads contribute).  Uses the
// caller's shared scratch sm[NV * BLOCK]; totals in res[NV] (shared).
// The values go through a shared-memory tree (BLOCK/2, BLOCK/4, ... 32
// active threads) and one warp finishes with shuffles: about 12 warp-wide
// FP64 additions per value instead of 45 for a shuffle tree in every warp,
// which matters on a part with little FP64 throughput.
// The tree runs in the values' type A: FP64 for FP64 data, FP32 for the
// FP32 inner solves (whose per-thread sums are FP32 already); the totals are
// returned in FP64 for the grid-wide sum.
template <int NV, int BLOCK, typename A>
__device__ __forceinline__ void block_sum(const A (&v)[NV], A* sm, double* res) {
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) sm[k * BLOCK + threadIdx.x] = v[k];
  __syncthreads();
#pragma unroll
  for (int s = BLOCK / 2; s >= 32; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < NV; ++k) sm[k * BLOCK + threadIdx.x] += sm[k * BLOCK + threadIdx.x + s];
    }
    __syncthreads();
  }
  if (warp_id() == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const A t = warp_allsum(sm[k * BLOCK + lane_id()]);
      if (lane_id() == 0) res[k] = (double)t;
    }
  }
  __syncthreads();
}

// Grid-wide deterministic sum of nv block totals blk[k] (shared memory, valid
// in every thread).  Returns true in every thread of the one block that
// finishes last; that block then finds the totals in tot[k] (shared).  The
// counter is reset so the site can be reused by the next launch.
// One level: each block publishes its totals and counts itself in; the last
// one sums all G partials of each value (one warp per value, lanes over the
// partials in a fixed order, a fixed shuffle tree).  The serial tail of a
// launch is then one fence, one atomic and one round of loads: a two-level
// scheme (groups of blocks, then the group totals) measured longer, its
// second atomic and fence sitting on the path that every other SM idles on.
__device__ __forceinline__ bool grid_sum(const double* blk, int nv, const GridRed& R, double* tot) {
  __shared__ int s_last;
  const int G = gridDim.x, b = blockIdx.x;
  const int nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    for (int k = 0; k < nv; ++k) R.partials[k * G + b] = blk[k];
    __threadfence();
    const unsigned t = atomicAdd(&R.counters[0], 1u);
    s_last = (t == (unsigned)(G - 1));
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  for (int k = warp_id(); k < nv; k += nwarps) {
    const double* p = R.partials + (long long)k * G;
    double v0 = 0.0, v1 = 0.0;
    int q = lane_id();
    for (; q + 32 < G; q += 64) {  // two independent chains, loads in flight together
      v0 += __ldcg(p + q);
      v1 += __ldcg(p + q + 32);
    }
    if (q < G) v0 += __ldcg(p + q);
    const double v = warp_allsum(v0 + v1);
    if (lane_id() == 0) tot[k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) R.counters[0] = 0u;
  return true;
}

// Last-block detection without values (for kernels whose epilogue must run
// after every block has read the shared state).
__device__ __forceinline__ bool grid_last(unsigned* counter) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
    if (s_last) *counter = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// ------------------------------------------------------------- row norms

enum PMode : int { kP1 = 0, kP2 = 1, kPInf = 2, kPGen = 3 };

__host__ __device__ inline int pmode_of(double p) {
  return p == 1.0 ? kP1 : (p == 2.0 ? kP2 : (p > 1e300 ? kPInf : kPGen));
}

// ||a||_p of one row held in shared memory (values converted to double).
// p = 2 sums squares directly unless the largest magnitude is near the ends
// of the exponent range, where the row is first scaled by an exact power of
// two; this is the definition up to rounding.  The largest magnitude and the
// finiteness test use the integer bit patterns (no FP64 work).
template <typename T>
__device__ __forceinline__ double row_norm(const T* v, int len, int pmode, double p, int* err) {
  unsigned long long mb = 0ull;
  bool nonfinite = false;
  for (int k = 0; k < len; ++k) {
    unsigned long long bits = (unsigned long long)__double_as_longlong((double)v[k]) & 0x7fffffffffffffffull;
    nonfinite |= bits >= 0x7ff0000000000000ull;
    mb = bits > mb ? bits : mb;
  }
  if (nonfinite) {
    atomicOr(err, kErrNonFinite);
    return 1.0;
  }
  if (mb == 0ull) {
    atomicOr(err, kErrZeroRow);
    return 1.0;
  }
  const double m = __longlong_as_double((long long)mb);
  if (pmode == kPInf) return m;
  if (pmode == kP1) {
    double s = 0.0;
    for (int k = 0; k < len; ++k) s += fabs((double)v[k]);
    return s;
  }
  if (pmode == kP2) {
    const int e = (int)(mb >> 52) - 1023;
    if (e > -480 && e < 480) {
      double s = 0.0;
      for (int k = 0; k < len; ++k) {
        const double a = (double)v[k];
        s = fma(a, a, s);
      }
      return sqrt(s);
    }
    const double sc = ldexp(1.0, -e), isc = ldexp(1.0, e);
    double s = 0.0;
    for (int k = 0; k < len; ++k) {
      const double a = (double)v[k] * sc;
      s = fma(a, a, s);
    }
    return sqrt(s) * isc;
  }
  double s = 0.0;
  for (int k = 0; k < len; ++k) s += pow(fabs((double)v[k]) / m, p);
  return m * pow(s, 1.0 / p);
}

// ------------------------------------------------------------- CSR tiles
//
// One warp computes the products of 32 consecutive rows r0..r0+31 with a
// vector x.  The tile's nonzeros form one contiguous range of val/colidx; the
// warp copies that range into shared memory with coalesced loads and then
// each lane sums its own row from shared memory (one FMA per nonzero, no
// cross-lane FP64 work).  Tiles whose range exceeds the staging capacity are
// read directly.  Every rowptr extent and column index is bounds-checked;
// violations set kErrIndex in *err and contribute nothing.
template <typename T, int CAP>
struct TileStage {
  T val[CAP];
  int col[CAP];
};

template <typename T, typename XT, int CAP>
__device__ __forceinline__ T csr_tile_row(const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                          const T* __restrict__ val, const XT* __restrict__ x, int n, int nnz,
                                          int r0, TileStage<T, CAP>& st, int* err) {
  const int lane = lane_id();
  const int row = r0 + lane;
  const int last = min(31, n - 1 - r0);
  int rs = 0, re = 0;
  if (row < n) {
    rs = __ldg(rowptr + row);
    re = __ldg(rowptr + row + 1);
  }
  const int e0 = __shfl_sync(kFull, rs, 0);
  const int e1 = __shfl_sync(kFull, re, last);
  bool ok = (row >= n) || (rs >= e0 && re >= rs && re <= e1);
  const bool tile_ok = (e0 >= 0) && (e1 <= nnz) && (e1 >= e0);
  ok = ok && tile_ok;
  if (!ok) atomicOr(err, kErrIndex);
  T sum = T(0);
  const int cnt = e1 - e0;
  if (tile_ok && cnt <= CAP) {
#pragma unroll 4
    for (int k = lane; k < cnt; k += 32) {
      st.val[k] = __ldg(val + e0 + k);
      st.col[k] = __ldg(colidx + e0 + k);
    }
    __syncwarp();
    if (ok && row < n) {
      const int base = rs - e0, len = re - rs;
      int k = 0;
      // pairs: two gathers of x in flight before the FMAs (column order kept)
      for (; k + 1 < len; k += 2) {
        const int c0 = st.col[base + k], c1 = st.col[base + k + 1];
        const T a0 = st.val[base + k], a1 = st.val[base + k + 1];
        T x0 = T(0), x1 = T(0);
        if ((unsigned)c0 < (unsigned)n) x0 = (T)__ldg(x + c0); else atomicOr(err, kErrIndex);
        if ((unsigned)c1 < (unsigned)n) x1 = (T)__ldg(x + c1); else atomicOr(err, kErrIndex);
        sum = fma(a0, x0, sum);
        sum = fma(a1, x1, sum);
      }
      if (k < len) {
        const int c0 = st.col[base + k];
        if ((unsigned)c0 < (unsigned)n) sum = fma(st.val[base + k], (T)__ldg(x + c0), sum);
        else atomicOr(err, kErrIndex);
      }
    }
    __syncwarp();
  } else if (ok && row < n) {
    for (int k = rs; k < re; ++k) {
      const int cc = __ldg(colidx + k);
      if ((unsigned)cc < (unsigned)n) sum = fma(__ldg(val + k), (T)__ldg(x + cc), sum);
      else atomicOr(err, kErrIndex);
    }
  }
  return sum;
}

}  // namespace gsk
