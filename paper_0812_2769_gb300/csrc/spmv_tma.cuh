// CSR products with the matrix streamed into shared memory by TMA bulk copies.
//
// A block owns a sequence of 256-row chunks (chunk c = blockIdx.x + q * grid).
// One thread is the producer: for each chunk it reads the chunk's nonzero
// range [e0, e1) from rowptr and issues two cp.async.bulk copies (values and
// column indices) into one stage of a double-buffered shared-memory ring,
// completing on that stage's mbarrier.  Every thread then waits for the stage,
// sums its own row from shared memory (one FMA per nonzero, the gathers of x
// issued in pairs) and hands (row, value) to the caller's epilogue.  While a
// chunk is being summed the next one is already in flight, so the HBM stream
// does not wait on the arithmetic.
//
// TMA rules respected here: both addresses of a bulk copy are 16-byte aligned
// and its size is a multiple of 16 bytes.  The copied range starts at e0
// rounded down to a 16-byte boundary (a few leading entries are ignored) and
// ends at e1 rounded up, inside the array; only where that would pass the
// array's end (the matrix's last chunk) does it end at e1 rounded down, the
// producer loading the last few entries itself.  Chunks whose range does not fit a
// stage (very long rows), or matrices whose arrays are not 16-byte aligned,
// are summed straight from global memory.  Every mbarrier wait is bounded:
// on time-out the kernel records kErrTimeout and stops using the ring.
#pragma once

#include "device_common.cuh"

namespace gsk {

constexpr int kPipeRows = 256;    // rows per chunk = threads per block
constexpr int kPipeCap = 1856;    // nonzeros per stage (7-point rows: 1792)
constexpr int kPipeSpin = 1 << 22;  // bounded mbarrier polls per wait

template <typename T>
struct __align__(16) PipeSmem {
  T val[2][kPipeCap];
  int col[2][kPipeCap];
  unsigned long long mbar[2];
  // per stage: offsets of the copied ranges, the chunk's nonzero range
  // [e0, e1) and whether its rows are read from global memory instead
  int va0[2], ca0[2], e0[2], e1[2], direct[2];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(tx) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Copy range of one array for nonzeros [e0, e1): start rounded down to a
// 16-byte boundary; end rounded up when that stays inside the array (all but
// possibly the matrix's last chunk), else rounded down, the rest loaded
// with plain loads.
template <int EV>
struct CopyRange {
  int a0, a1, tail;  // copy [a0, a1), then plain loads [tail, e1)
  __device__ __forceinline__ CopyRange(int e0, int e1, int nnz) {
    a0 = e0 & ~(EV - 1);
    const int up = (e1 + EV - 1) & ~(EV - 1);
    if (up <= nnz) {
      a1 = up;
      tail = e1;
    } else {
      a1 = e1 & ~(EV - 1);
      tail = a1;
    }
  }
};

// Producer side: stage `st` receives the chunk whose nonzeros are [e0, e1).
// Thread 0 only.
template <typename T>
__device__ __forceinline__ void pipe_issue(PipeSmem<T>& sm, int st, int e0, int e1,
                                           const int* __restrict__ colidx, const T* __restrict__ val, int nnz,
                                           bool aligned, int* err) {
  int direct = 1;
  int va0 = 0, ca0 = 0;
  unsigned vbytes = 0, cbytes = 0;
  if (e0 < 0 || e1 > nnz || e1 < e0) {
    atomicOr(err, kErrIndex);
    e0 = e1 = 0;  // the chunk's rows then all fail their range check
  } else if (aligned) {
    const CopyRange<16 / sizeof(T)> vr(e0, e1, nnz);
    const CopyRange<4> cr(e0, e1, nnz);
    // the stage receives [a0, max(a1, e1)): the bulk copy up to a1, then, on
    // the matrix's last chunk, the plain loads of [tail, e1), which end past
    // a1 when e1 was rounded down
    const int vspan = (vr.a1 > e1 ? vr.a1 : e1) - vr.a0;
    const int cspan = (cr.a1 > e1 ? cr.a1 : e1) - cr.a0;
    if (vspan <= kPipeCap && cspan <= kPipeCap) {
      direct = 0;
      va0 = vr.a0;
      ca0 = cr.a0;
      vbytes = (unsigned)(vr.a1 - vr.a0) * (unsigned)sizeof(T);
      cbytes = (unsigned)(cr.a1 - cr.a0) * 4u;
      for (int k = vr.tail; k < e1; ++k) sm.val[st][k - va0] = __ldg(val + k);
      for (int k = cr.tail; k < e1; ++k) sm.col[st][k - ca0] = __ldg(colidx + k);
    }
  }
  sm.va0[st] = va0;
  sm.ca0[st] = ca0;
  sm.e0[st] = e0;
  sm.e1[st] = e1;
  sm.direct[st] = direct;
  fence_proxy_async();
  mbar_arrive_tx(&sm.mbar[st], vbytes + cbytes);
  if (vbytes) bulk_g2s(&sm.val[st][0], val + va0, vbytes, &sm.mbar[st]);
  if (cbytes) bulk_g2s(&sm.col[st][0], colidx + ca0, cbytes, &sm.mbar[st]);
}

// Sum of the products of one row with nonzeros [rs, re), from stage `st`
// (or from global memory when the stage holds no copy).  Gathers of x are
// issued four at a time ahead of their FMAs; the FMAs keep column order and
// no FMA is issued for an entry the row does not have (on this part an FP64
// instruction costs its pipe time even with every lane predicated off).
template <typename T, typename XT>
__device__ __forceinline__ T pipe_row(const PipeSmem<T>& sm, int st, int rs, int re,
                                      const int* __restrict__ colidx, const T* __restrict__ val,
                                      const XT* __restrict__ x, int n, int* err) {
  T sum = T(0);
  if (rs < sm.e0[st] || re < rs || re > sm.e1[st]) {
    atomicOr(err, kErrIndex);
    return sum;
  }
  const bool direct = sm.direct[st] != 0;
  const T* v = direct ? val + rs : &sm.val[st][rs - sm.va0[st]];
  const int* c = direct ? colidx + rs : &sm.col[st][rs - sm.ca0[st]];
  const int len = re - rs;
  int k = 0;
  for (; k + 4 <= len; k += 4) {
    T xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int cc = c[k + u];
      xv[u] = T(0);
      if ((unsigned)cc < (unsigned)n) xv[u] = (T)__ldg(x + cc);
      else atomicOr(err, kErrIndex);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) sum = fma(v[k + u], xv[u], sum);
  }
  // the last 1..3 entries: their gathers together, then exactly as many FMAs
  const int rem = len - k;
  if (rem > 0) {
    T xv[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int u = 0; u < 3; ++u)
      if (u < rem) {
        const int cc = c[k + u];
        if ((unsigned)cc < (unsigned)n) xv[u] = (T)__ldg(x + cc);
        else atomicOr(err, kErrIndex);
      }
    sum = fma(v[k], xv[0], sum);
    if (rem > 1) {
      sum = fma(v[k + 1], xv[1], sum);
      if (rem > 2) sum = fma(v[k + 2], xv[2], sum);
    }
  }
  return sum;
}

// y_i = (A x)_i for every row, delivered to epi(i, y_i) by the thread that
// owns row i.  Must be called by all threads of a kPipeRows-thread block.
// Latency hiding: the producer loads the bounds of the chunk it will issue
// next one chunk ahead, and every thread loads its next row's extent before
// it waits for the current stage.
template <typename T, typename XT, typename Epi>
__device__ __forceinline__ void spmv_rows_tma(const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                              const T* __restrict__ val, const XT* __restrict__ x, int n, int nnz,
                                              PipeSmem<T>& sm, int* err, Epi&& epi) {
  const int nchunks = (n + kPipeRows - 1) / kPipeRows;
  const int G = gridDim.x;
  const bool aligned = (((uintptr_t)val | (uintptr_t)colidx) & 15u) == 0;
  auto chunk_lo = [&](int c) { return __ldg(rowptr + c * kPipeRows); };
  auto chunk_hi = [&](int c) { return __ldg(rowptr + min(c * kPipeRows + kPipeRows, n)); };
  if (threadIdx.x == 0) {
    mbar_init(&sm.mbar[0], 1);
    mbar_init(&sm.mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // thread 0 tracks, per stage (bit st), whether a copy is outstanding and
  // the phase it completes
  unsigned pending = 0u, next_parity = 0u;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 2; ++q) {
      const int c = blockIdx.x + q * G;
      if (c < nchunks) {
        pipe_issue(sm, q, chunk_lo(c), chunk_hi(c), colidx, val, nnz, aligned, err);
        pending |= 1u << q;
      }
    }
  }
  // this thread's row extent in the first chunk
  int rs = 0, re = 0;
  {
    const int row = blockIdx.x * kPipeRows + threadIdx.x;
    if (blockIdx.x < nchunks && row < n) {
      rs = __ldg(rowptr + row);
      re = __ldg(rowptr + row + 1);
    }
  }
  bool ring_ok = true;
  for (int q = 0;; ++q) {
    const int c = blockIdx.x + q * G;
    if (c >= nchunks) break;
    const int st = q & 1;
    const unsigned parity = (unsigned)((q >> 1) & 1);
    // prefetch: the producer's bounds for chunk c + 2G, every thread's row
    // extent in chunk c + G
    const int cf = c + 2 * G;
    int f0 = 0, f1 = 0;
    if (threadIdx.x == 0 && cf < nchunks) {
      f0 = chunk_lo(cf);
      f1 = chunk_hi(cf);
    }
    const int rown = (c + G) * kPipeRows + threadIdx.x;
    int rsn = 0, ren = 0;
    if (c + G < nchunks && rown < n) {
      rsn = __ldg(rowptr + rown);
      ren = __ldg(rowptr + rown + 1);
    }
    if (ring_ok) {
      int it = 0;
      while (!mbar_try_wait(&sm.mbar[st], parity) && ++it < kPipeSpin) {
      }
      if (it >= kPipeSpin) {
        atomicOr(err, kErrTimeout);
        ring_ok = false;
      } else if (threadIdx.x == 0) {
        pending &= ~(1u << st);
        next_parity ^= 1u << st;
      }
    }
    const int row = c * kPipeRows + threadIdx.x;
    if (row < n) {
      T y;
      if (ring_ok) {
        y = pipe_row(sm, st, rs, re, colidx, val, x, n, err);
      } else {  // the ring is not trusted any more: read straight from global memory
        y = T(0);
        if (rs >= 0 && re >= rs && re <= nnz)
          for (int k = rs; k < re; ++k) {
            const int cc = __ldg(colidx + k);
            if ((unsigned)cc < (unsigned)n) y = fma(__ldg(val + k), (T)__ldg(x + cc), y);
          }
      }
      epi(row, y);
    }
    rs = rsn;
    re = ren;
    __syncthreads();  // every thread is done with stage st
    if (threadIdx.x == 0 && ring_ok && cf < nchunks) {
      pipe_issue(sm, st, f0, f1, colidx, val, nnz, aligned, err);
      pending |= 1u << st;
    }
  }
  // only after a time-out can a copy still be in flight: wait for it (again
  // bounded) before the block's shared memory is released
  if (threadIdx.x == 0 && !ring_ok) {
    for (int st = 0; st < 2; ++st) {
      int it = 0;
      while (((pending >> st) & 1u) && !mbar_try_wait(&sm.mbar[st], (next_parity >> st) & 1u) &&
             ++it < kPipeSpin) {
      }
    }
  }
  __syncthreads();
}

}  // namespace gsk
