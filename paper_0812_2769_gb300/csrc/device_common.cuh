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
//  * Cross-block sums use the "last block finishes" pattern in two levels
//    (groups of kGroup blocks, then the group totals), so no kernel ever waits
//    on another block and no spin loop exists.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gsk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGroup = 16;  // blocks per first-level reduction group

// error bits written by kernels into a device status word
enum : int { kErrIndex = 1, kErrZeroRow = 2, kErrNonFinite = 4 };

// Scratch for one grid-wide reduction site.
struct GridRed {
  double* partials;    // [nv_max * maxgrid]
  double* gpartials;   // [nv_max * ngroups(maxgrid)]
  unsigned* counters;  // [ngroups(maxgrid) + 1], zero between uses
  int maxgrid;         // launches using this site must have gridDim.x <= maxgrid
};

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// Sum of cnt entries src[k*stride + q] (q < cnt) for each k < nv, computed by
// one full warp in a fixed order; the totals are returned in out[k] (written
// by lane 0 when nv is small, by lane k % 32 otherwise).
template <int NVMAX>
__device__ __forceinline__ void warp_sum_table(const double* src, int stride, int cnt, int nv,
                                               double* out, bool cached) {
  const int lane = lane_id();
  if (nv >= 8) {
    for (int k = lane; k < nv; k += 32) {
      double s = 0.0;
      for (int q = 0; q < cnt; ++q) s += cached ? src[k * stride + q] : __ldcg(src + k * stride + q);
      out[k] = s;
    }
  } else {
    for (int k = 0; k < nv; ++k) {
      double s = 0.0;
      for (int q = lane; q < cnt; q += 32) s += cached ? src[k * stride + q] : __ldcg(src + k * stride + q);
      s = warp_allsum(s);
      if (lane == 0) out[k] = s;
    }
  }
}

// Block-wide sum of nv per-thread values held in shared memory as
// tab[k * BLOCK + t].  Result in res[k] (shared), valid after the call.
template <int BLOCK>
__device__ __forceinline__ void block_sum_table(double* tab, int nv, double* res) {
  __syncthreads();
  constexpr int NW = BLOCK / 32;
  const int w = warp_id();
  // each warp takes whole rows k; a row of BLOCK entries is summed by the
  // warp's lanes (BLOCK/32 each, sequential) and a fixed shuffle tree
  for (int k = w; k < nv; k += NW) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < BLOCK / 32; ++q) s += tab[k * BLOCK + lane_id() * (BLOCK / 32) + q];
    s = warp_allsum(s);
    if (lane_id() == 0) res[k] = s;
  }
  __syncthreads();
}

// Block-wide sum of NV register values (all threads contribute).  Uses the
// caller's shared scratch sm[NV * BLOCK]; totals in res[NV] (shared).
template <int NV, int BLOCK>
__device__ __forceinline__ void block_sum(const double (&v)[NV], double* sm, double* res) {
  if (NV <= 4) {
    // few values: warp trees, then one warp over the warp totals
    constexpr int NW = BLOCK / 32;
    __syncthreads();
    double t[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] = warp_allsum(v[k]);
    if (lane_id() == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) sm[k * NW + warp_id()] = t[k];
    }
    __syncthreads();
    if (warp_id() == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double s = lane_id() < NW ? sm[k * NW + lane_id()] : 0.0;
        s = warp_allsum(s);
        if (lane_id() == 0) res[k] = s;
      }
    }
    __syncthreads();
  } else {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k * BLOCK + threadIdx.x] = v[k];
    block_sum_table<BLOCK>(sm, NV, res);
  }
}

// Grid-wide deterministic sum of nv block totals blk[k] (shared memory, valid
// in every thread).  Returns true in every thread of the one block that
// finishes last; that block then finds the totals in tot[k] (shared).  The
// counters are reset so the site can be reused by the next launch.
__device__ __forceinline__ bool grid_sum(const double* blk, int nv, const GridRed& R, double* tot) {
  __shared__ int s_last;
  const int G = gridDim.x, b = blockIdx.x;
  const int g = b / kGroup;
  const int ng = (G + kGroup - 1) / kGroup;
  const int gsize = min(kGroup, G - g * kGroup);
  if (threadIdx.x == 0) {
    for (int k = 0; k < nv; ++k) R.partials[k * G + b] = blk[k];
    __threadfence();
    unsigned t = atomicAdd(&R.counters[g], 1u);
    s_last = (t == (unsigned)(gsize - 1));
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  if (warp_id() == 0) {
    // this block closes group g: sum its gsize partials per value
    double* gout = R.gpartials;  // [k * ng + g]
    if (nv >= 8) {
      for (int k = lane_id(); k < nv; k += 32) {
        double s = 0.0;
        for (int q = 0; q < gsize; ++q) s += __ldcg(R.partials + k * G + g * kGroup + q);
        gout[k * ng + g] = s;
      }
    } else {
      for (int k = 0; k < nv; ++k) {
        double s = lane_id() < gsize ? __ldcg(R.partials + k * G + g * kGroup + lane_id()) : 0.0;
        s = warp_allsum(s);
        if (lane_id() == 0) gout[k * ng + g] = s;
      }
    }
    __syncwarp();
    if (lane_id() == 0) {
      R.counters[g] = 0u;
      __threadfence();
      unsigned t = atomicAdd(&R.counters[ng], 1u);
      s_last = (t == (unsigned)(ng - 1));
    }
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  if (warp_id() == 0) {
    warp_sum_table<64>(R.gpartials, ng, ng, nv, tot, false);
    __syncwarp();
    if (lane_id() == 0) R.counters[ng] = 0u;
  }
  __syncthreads();
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
      for (int k = rs - e0; k < re - e0; ++k) {
        const int c = st.col[k];
        if ((unsigned)c < (unsigned)n) sum = fma(st.val[k], (T)__ldg(x + c), sum);
        else atomicOr(err, kErrIndex);
      }
    }
    __syncwarp();
  } else if (ok && row < n) {
    for (int k = rs; k < re; ++k) {
      const int c = __ldg(colidx + k);
      if ((unsigned)c < (unsigned)n) sum = fma(__ldg(val + k), (T)__ldg(x + c), sum);
      else atomicOr(err, kErrIndex);
    }
  }
  return sum;
}

}  // namespace gsk
