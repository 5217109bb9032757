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

#include <type_traits>

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

// Block-wide sum of nv <= 16 per-thread values held in shared memory as
// tab[k * BLOCK + t] (the table is consumed), added in the table's type.
// Result in res[k] (shared), valid after the call.
// On this part each SM sub-partition has a narrow FP64 unit and a warp's FP64
// instruction costs its pipe time whatever its active lanes, so the work is
// dealt over every warp instead of narrowing to one: each value's BLOCK
// entries first fold to 32 (fold q adds entries q, q + 32, q + 64, ... in
// that order; the nv * 32 folds are spread over all threads), then each warp
// finishes two values, its half-warps adding folds l and l + 16 and meeting
// in a fixed four-level shuffle tree.
template <int BLOCK, typename TT>
__device__ __forceinline__ void block_sum_table(TT* tab, int nv, double* res) {
  static_assert(BLOCK % 32 == 0 && BLOCK >= 64, "block of whole warps, at least two");
  __syncthreads();
  for (int o = threadIdx.x; o < nv * 32; o += BLOCK) {
    TT* p = tab + (o >> 5) * BLOCK + (o & 31);
    TT t = p[0];
#pragma unroll
    for (int r = 1; r < BLOCK / 32; ++r) t += p[32 * r];
    p[0] = t;  // each fold reads and writes only its own entries
  }
  __syncthreads();
  const int half = lane_id() >> 4, l = lane_id() & 15;
  for (int v0 = 2 * warp_id(); v0 < nv; v0 += 2 * (BLOCK / 32)) {  // warp-uniform
    const int v = v0 + half;
    TT t = TT(0);
    if (v < nv) t = tab[v * BLOCK + l] + tab[v * BLOCK + l + 16];
#pragma unroll
    for (int off = 8; off; off >>= 1) t += __shfl_xor_sync(kFull, t, off);
    if (l == 0 && v < nv) res[v] = (double)t;
  }
  __syncthreads();
}

// Block-wide sum of NV register values (all threads contribute).  Uses the
// caller's shared scratch sm[NV * BLOCK]; totals in res[NV] (shared).  The
// sum runs in the values' type A (FP64 for FP64 data, FP32 for the FP32
// inner solves, whose per-thread sums are FP32 already), the same fixed
// order as block_sum_table; the totals are returned in FP64 for the
// grid-wide sum.
template <int NV, int BLOCK, typename A>
__device__ __forceinline__ void block_sum(const A (&v)[NV], A* sm, double* res) {
  static_assert(NV <= 16, "at most 16 values per call");
  __syncthreads();  // the scratch may still be read by an earlier sum
#pragma unroll
  for (int k = 0; k < NV; ++k) sm[k * BLOCK + threadIdx.x] = v[k];
  block_sum_table<BLOCK>(sm, NV, res);
}

// Block-wide sum of NV register values with the shortest dependent chain
// and few registers, for block sums on a latency-bound path (the batched
// solvers, one block per system): a shared-memory tree (BLOCK/2, BLOCK/4,
// ... 32 active threads) and one warp's shuffle tree.  Uses the caller's
// shared scratch sm[NV * BLOCK]; totals in res[NV] (shared).
template <int NV, int BLOCK, typename A>
__device__ __forceinline__ void block_sum_tree(const A (&v)[NV], A* sm, double* res) {
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
// one sums all G partials of each value with all its threads.  Value v's
// partials go to tpv threads (the largest power of two up to 32 with
// nv * tpv <= blockDim.x, so that a value's threads are neighbouring lanes of
// one warp); thread q adds partials q, q + tpv, q + 2 tpv, ... in that order,
// issuing their loads B at a time ahead of the additions (B = 16 in kernels
// with many values, whose registers are free by then), and the tpv
// sums meet in a fixed shuffle tree.  The serial tail of a launch is then one
// fence, one atomic and a round or two of loads: a two-level scheme (groups
// of blocks, then the group totals) measured longer, its second atomic and
// fence sitting on the path that every other SM idles on.
template <int B = 8>
__device__ __forceinline__ bool grid_sum(const double* blk, int nv, const GridRed& R, double* tot) {
  __shared__ int s_last;
  const int G = gridDim.x, b = blockIdx.x;
  if (threadIdx.x == 0) {
    for (int k = 0; k < nv; ++k) R.partials[k * G + b] = blk[k];
    __threadfence();
    const unsigned t = atomicAdd(&R.counters[0], 1u);
    s_last = (t == (unsigned)(G - 1));
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  int tpv = 32;
  while (tpv > 1 && tpv * nv > (int)blockDim.x) tpv >>= 1;
  const int per_round = (int)blockDim.x / tpv;
  for (int v0 = 0; v0 < nv; v0 += per_round) {  // one round unless nv > blockDim.x
    const int v = v0 + (int)threadIdx.x / tpv, q = (int)threadIdx.x % tpv;
    double s = 0.0;
    if (v < nv) {
      const double* p = R.partials + (long long)v * G;
      for (int i = q; i < G; i += B * tpv) {
        double t[B];
#pragma unroll
        for (int u = 0; u < B; ++u) t[u] = i + u * tpv < G ? __ldcg(p + i + u * tpv) : 0.0;
#pragma unroll
        for (int u = 0; u < B; ++u) s += t[u];
      }
    }
    for (int off = tpv >> 1; off; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
    if (v < nv && q == 0) tot[v] = s;
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

// The bit pattern of v, through an opaque move.  Tests on a double's bits
// (finiteness, the largest magnitude) are then done as integer instructions:
// written on the reinterpreted bits directly, the compiler recognises them and
// turns them into FP64 compares, which occupy the scarce FP64 pipe (measured:
// a finiteness test and a maximum doubled the FP64 instructions of a row-norm
// loop).
__device__ __forceinline__ unsigned long long dbits(double v) {
  unsigned long long b;
  asm("mov.b64 %0, %1;" : "=l"(b) : "d"(v));
  return b;
}

// True when a bit pattern is a finite double (exponent field not all ones).
__device__ __forceinline__ bool finite_pattern(unsigned long long b) {
  return (b & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// Reciprocals for the GS scales.  FP64 instructions are scarce on this part
// (a correctly rounded FP64 division or square root costs tens of them per
// row), so d = 1/||a||_p is formed from an FP32 seed (the hardware
// approximation of 1/x or 1/sqrt(x), about 22 correct bits, taken on the
// FP32 pipe) and one cubically convergent Householder correction in FP64 (a
// published method: Householder's iteration of order 3 for the reciprocal
// and the reciprocal square root).  With e = 1 - s y or e = 1 - s y^2 of
// size 2^-22, the corrections
//     1/s:        y + y (e + e^2)
//     1/sqrt(s):  y + y e (1/2 + 3/8 e)
// leave a relative error of order e^3 (2^-66), below the rounding of the
// few FP64 operations that form them: the result is within a few ulp of the
// exact value.  The seed's exponent is moved by integer operations on the bit
// pattern, so only 3 (1/s) or 5 (1/sqrt(s)) FP64 instructions are issued.
// Both take a positive, finite, normal s; the callers route the rare
// subnormal or near-overflow cases to the plain division.

// 1/s for a positive normal s whose reciprocal is normal too (s < 2^1022).
__device__ __forceinline__ double recip_pos(double s) {
  const long long bits = (long long)dbits(s);
  const int ex = (int)(bits >> 52);  // biased exponent
  if (ex == 0 || ex >= 2045) return 1.0 / s;
  // s = 2^(ex-1023) f with f in [1, 2): seed 1/f in FP32
  const unsigned fb = 0x3f800000u | (unsigned)((bits >> 29) & 0x7fffffll);
  const unsigned yb = __float_as_uint(__frcp_rn(__uint_as_float(fb)));
  const int fe = (int)((yb >> 23) & 0xffu) - 127;  // -1 or 0
  const double y =
      __longlong_as_double(((long long)(fe - ex + 2046) << 52) | ((long long)(yb & 0x7fffffu) << 29));
  const double e = fma(-s, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// 1/sqrt(s) for a positive normal s.
__device__ __forceinline__ double rsqrt_pos(double s) {
  const long long bits = (long long)dbits(s);
  const int ex = (int)(bits >> 52);
  if (ex == 0 || ex == 2047) return 1.0 / sqrt(s);
  const int e2 = ex - 1023;  // s = 2^e2 f, f in [1, 2)
  const int k = e2 >> 1;     // s = 2^(2k) g, g = f 2^(e2 - 2k) in [1, 4)
  const unsigned gb = ((unsigned)(127 + (e2 - 2 * k)) << 23) | (unsigned)((bits >> 29) & 0x7fffffll);
  const unsigned yb = __float_as_uint(rsqrtf(__uint_as_float(gb)));  // 1/sqrt(g) in (1/2, 1]
  const int fe = (int)((yb >> 23) & 0xffu) - 127;
  const double y =
      __longlong_as_double(((long long)(fe - k + 1023) << 52) | ((long long)(yb & 0x7fffffu) << 29));
  const double t = s * y;
  const double e = fma(-t, y, 1.0);
  return fma(y, e * fma(0.375, e, 0.5), y);
}

// Sums of |a| and of a^2 over a row of doubles in the integer pipes.  On
// this part a row of GS(2) needs about 20 FP64 instructions (squares,
// scaling products, the reciprocal square root) for 88 bytes of traffic, so
// the FP64 pipe, not HBM, bounds the one-pass kernel; the sums move to the
// integer units, which are many times wider.  Every entry a = m 2^(E-1075)
// (m the 53-bit significand, E the biased exponent; subnormals have E = 0
// and no implicit bit, and are taken as E = 1) is aligned to the row's
// largest biased exponent emax and added as an integer: |a| as
// (m 2^48) >> (emax - E) into a 128-bit accumulator with unit 2^(emax -
// 1123), a^2 as the square of the 64-bit (m 2^5) >> (emax - E) (one wide
// multiply, no 128-bit shift) with unit 2^(2 emax - 2160).  The only loss is
// the bits shifted out below the unit (against a largest term of at least
// 2^100 or 2^114 units), so the sum is the exact one to within a relative
// len 2^-55 (a^2) or len 2^-100 (|a|) before its final rounding to double,
// closer than an FP64 loop; the accumulators hold rows of up to 4,096 (a^2)
// and 2^20 (|a|) entries, longer rows take the FP64 route.  `int_sum_to_double` rounds it to the nearest double; the callers
// use these only where that double is normal (the row's largest exponent is
// far from the ends of the range).
__device__ __forceinline__ double int_sum_to_double(unsigned __int128 acc, int unit_exp) {
  // acc > 0; value = acc 2^unit_exp
  const unsigned long long hi = (unsigned long long)(acc >> 64), lo = (unsigned long long)acc;
  const int lead = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  unsigned long long mant;
  int shift = lead - 52;  // bits below the 53 kept
  if (shift <= 0) {
    mant = lo << (-shift);
  } else {
    mant = (unsigned long long)(acc >> shift);
    const unsigned __int128 rem = acc & ((((unsigned __int128)1) << shift) - 1);
    const unsigned __int128 half = ((unsigned __int128)1) << (shift - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      mant += 1ull;
      if (mant >> 53) {
        mant >>= 1;
        shift += 1;
      }
    }
  }
  const long long ef = (long long)shift + unit_exp + 52 + 1023;  // biased exponent of mant 2^(shift + unit_exp)
  return __longlong_as_double((ef << 52) | (long long)(mant & 0x000fffffffffffffull));
}

// sum |a_k| (P2 false) or sum a_k^2 (P2 true) over a row of doubles whose
// largest magnitude has biased exponent emax (1 <= emax <= 2046).
template <bool P2>
__device__ __forceinline__ double row_int_sum(const double* v, int len, int emax) {
  unsigned __int128 acc = 0;
  for (int k = 0; k < len; ++k) {
    const unsigned long long b = dbits(v[k]);
    const int E = (int)((b >> 52) & 0x7ffull);
    const unsigned long long m = (b & 0x000fffffffffffffull) | ((unsigned long long)(E != 0) << 52);
    const int d = emax - (E == 0 ? 1 : E);  // >= 0
    if (P2) {
      if (d < 58) {
        const unsigned long long q = (m << 5) >> d;
        acc += (unsigned __int128)q * q;
      }
    } else {
      if (d < 101) acc += ((unsigned __int128)m << 48) >> d;
    }
  }
  return P2 ? int_sum_to_double(acc, 2 * emax - 2160) : int_sum_to_double(acc, emax - 1123);
}

// The rare cases of row_inv_norm, out of line so that the common path keeps
// few registers: a row whose largest exponent e is far from 0 (its sum could
// overflow or lose the small terms) and general p.  The row is summed again
// after an exact scaling by sc = 2^-e, which puts its largest term in [1, 2);
// then 1/||a|| = (1/||a sc||) sc.
template <typename T>
__device__ __noinline__ double row_inv_norm_rescaled(const T* v, int len, int pmode, double p, int e,
                                                     unsigned long long mb) {
  const double sc = ldexp(1.0, -e);
  double t = 0.0;
  if (pmode == kPInf) {
    t = __longlong_as_double((long long)mb) * sc;
  } else {
    for (int k = 0; k < len; ++k) {
      const double q = fabs((double)v[k]) * sc;
      if (pmode == kP1) t += q;
      else if (pmode == kP2) t = fma(q, q, t);
      else t += pow(q, p);
    }
  }
  double dt;
  if (pmode == kP2) dt = rsqrt_pos(t);
  else if (pmode == kPGen) dt = 1.0 / pow(t, 1.0 / p);
  else dt = recip_pos(t);
  return dt * sc;
}

// d = 1/||a||_p of one row (entries converted to double), for GS(p)
// (Sec. 2, Eq. (2)).  One pass over the row for p = 1, 2 and inf: the
// largest magnitude, the finiteness test (both on the integer bit patterns,
// no FP64 work) and the sum are taken together.  When the largest exponent is
// far from 0 the sum could overflow or lose the small terms, and the row is
// summed again after an exact power-of-two scaling; the result is the
// definition up to rounding.  A non-finite entry, an all-zero row or a norm
// whose reciprocal is not a finite double (every entry below 2^-1024) records
// an error bit in *err and returns 0 (the row is then not scaled).
template <int PM, typename T, bool INT_SUM = true>
__device__ __forceinline__ double row_inv_norm_pm(const T* v, int len, double p, int* err) {
  constexpr int pmode = PM;
  // FP64 rows take the sums of |a| and a^2 in the integer pipes (a second
  // sweep over the row once its largest exponent is known); FP32 rows, and
  // callers that pass INT_SUM = false (the FP64 batched kernels, whose
  // threads walk many rows from global memory one after another, where the
  // second sweep's latency costs more than the FP64 it saves), sum in FP64
  // as they go
  constexpr bool kIntSum = INT_SUM && std::is_same<T, double>::value && (PM == kP1 || PM == kP2);
  unsigned long long mb = 0ull;  // largest |a| (its bit pattern)
  unsigned long long nf = 0ull;  // nonzero when an entry is Inf or NaN
  double s = 0.0;
  for (int k = 0; k < len; ++k) {
    const double a = (double)v[k];
    const unsigned long long bits = dbits(a) & 0x7fffffffffffffffull;
    nf |= (bits + 0x0010000000000000ull) & 0x8000000000000000ull;  // exponent field all ones
    mb = bits > mb ? bits : mb;
    if (!kIntSum) {
      if (pmode == kP1) s += fabs(a);
      else if (pmode == kP2) s = fma(a, a, s);
    }
  }
  if (nf) {
    atomicOr(err, kErrNonFinite);
    return 0.0;
  }
  if (mb == 0ull) {
    atomicOr(err, kErrZeroRow);
    return 0.0;
  }
  const int e = (int)(mb >> 52) - 1023;  // exponent of the largest magnitude
  double d;
  if (pmode == kP2 && e > -480 && e < 480 && len < (1 << 12)) {
    if constexpr (kIntSum) s = row_int_sum<true>(reinterpret_cast<const double*>(v), len, e + 1023);
    d = rsqrt_pos(s);
  } else if (pmode == kP1 && e > -1000 && e < 1000 && len < (1 << 20)) {
    if constexpr (kIntSum) s = row_int_sum<false>(reinterpret_cast<const double*>(v), len, e + 1023);
    d = recip_pos(s);
  } else if (pmode == kPInf && e > -1000 && e < 1000) {
    d = recip_pos(__longlong_as_double((long long)mb));
  } else {
    d = row_inv_norm_rescaled(v, len, pmode, p, e, mb);
  }
  if (!finite_pattern(dbits(d))) {  // the norm underflows the reciprocal's range
    atomicOr(err, kErrZeroRow);
    return 0.0;
  }
  return d;
}

// The same with p chosen at run time (the one-block batched solvers).
template <bool INT_SUM = true, typename T>
__device__ __forceinline__ double row_inv_norm(const T* v, int len, int pmode, double p, int* err) {
  switch (pmode) {
    case kP1: return row_inv_norm_pm<kP1, T, INT_SUM>(v, len, p, err);
    case kP2: return row_inv_norm_pm<kP2, T, INT_SUM>(v, len, p, err);
    case kPInf: return row_inv_norm_pm<kPInf, T, INT_SUM>(v, len, p, err);
    default: return row_inv_norm_pm<kPGen, T, INT_SUM>(v, len, p, err);
  }
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
