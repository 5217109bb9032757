// ILU(0) on the device: the handle's layout and the triangular-solve kernel
// the preconditioned solvers record into their graphs.
//
// Rows are processed by level sets of their dependency graph (row i waits
// for the rows k < i of its pattern in the forward sweep and the factor, for
// the rows j > i in the backward sweep).  One cooperative launch runs all the
// levels of a sweep: its blocks are co-resident, sweep a level's rows, and
// meet at a grid barrier before the next level.  Every barrier wait is
// bounded: on time-out the kernel records kErrTimeout and carries on (the
// result is then wrong, and the caller reports GSK_ERR_TIMEOUT); later
// barriers of the launch see the flag and no longer wait.
// Values that other blocks wrote during the launch (z in the sweeps, the
// factors of earlier rows) are read with L2-only loads: L1 is not coherent
// between SMs.
#pragma once

#include "internal.hpp"

struct gsk_ilu0 {
  // unique per handle: solver graphs record pointers into the handle's device
  // memory, so their cache key names the handle by this number, never by
  // its address (a new handle may reuse a destroyed one's host address)
  unsigned long long serial = 0;
  int device = 0;
  int n = 0, nnz = 0;
  const int* rowptr = nullptr;  // A's structure (caller-owned)
  const int* colidx = nullptr;
  // one device allocation, carved into:
  void* mem = nullptr;
  double* lu = nullptr;    // [nnz] L (strictly lower part) and U, A's layout
  int* dpos = nullptr;     // [n] position of the diagonal in each row
  int* orderL = nullptr;   // [n] rows by forward level
  int* lptrL = nullptr;    // [nlevL + 1]
  int* orderU = nullptr;   // [n] rows by backward level
  int* lptrU = nullptr;    // [nlevU + 1]
  unsigned* bar = nullptr; // grid-barrier counter, zeroed before each launch
  int* err = nullptr;      // error bits of the factorisation and applications
  int nlevL = 0, nlevU = 0;
  int grid = 0;            // blocks of the cooperative launches (all resident)
  // one-CTA sweep for systems whose z fits in shared memory: the rows of each
  // sweep in level order with their first kIluPack entries packed, in a
  // second allocation; smem_bytes = 0 means the cooperative grid sweep
  void* pmem = nullptr;
  int smem_bytes = 0;
  int *prowL = nullptr, *pk0L = nullptr, *pk1L = nullptr, *pcolL = nullptr, *psrcL = nullptr;
  int *prowU = nullptr, *pk0U = nullptr, *pk1U = nullptr, *pcolU = nullptr, *psrcU = nullptr, *ppsrc = nullptr;
  double *pvalL = nullptr, *pvalU = nullptr, *ppiv = nullptr;
};

namespace gsk {

constexpr int kIluBlock = 256;
constexpr unsigned kIluSpin = 1u << 20;  // bounded polls per barrier

// Where an application reads its right-hand side and whether it runs at all
// (the solvers' graphs skip it after their iteration has stopped).
struct IluGate {
  const double* base;  // r = base + (*col) * stride (col may be null: r = base)
  const int* col;
  long long stride;
  const int* skip0;    // skip when any of these is nonzero (may be null)
  const int* skip1;
  const int* skip2;
  const int* run_if;   // skip when this is zero (may be null)
};

struct IluArgs {
  int n;
  const int* rowptr;
  const int* colidx;
  const double* lu;
  const int* dpos;
  const int* orderL;
  const int* lptrL;
  const int* orderU;
  const int* lptrU;
  int nlevL, nlevU;
  unsigned* bar;
  int* err;
  IluGate gate;
  double* z;
};

__device__ __forceinline__ bool ilu_gate_closed(const IluGate& g) {
  if (g.skip0 && *g.skip0) return true;
  if (g.skip1 && *g.skip1) return true;
  if (g.skip2 && *g.skip2) return true;
  if (g.run_if && !*g.run_if) return true;
  return false;
}

// Grid barrier number `k` (0-based) of a cooperative launch: every block
// arrives once per barrier, so barrier k completes at gridDim.x * (k + 1)
// arrivals.  Bounded.
__device__ __forceinline__ void ilu_barrier(unsigned* bar, unsigned k, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned target = gridDim.x * (k + 1);
    unsigned it = 0;
    while (*(volatile unsigned*)bar < target) {
      // after one time-out no barrier of the launch waits any more: the
      // result is already wrong, and the launch must end promptly
      if (++it >= kIluSpin || (*(volatile int*)err & kErrTimeout)) {
        atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

// z = U^-1 L^-1 r, level by level.
__global__ void __launch_bounds__(kIluBlock) ilu_solve_kernel(IluArgs a);

// The same sweeps by one CTA with z in shared memory, for systems small
// enough: a level then ends at __syncthreads instead of a grid barrier, and
// the rows of the next level (level-ordered, their first kIluPack columns
// and factor entries packed) are loaded while the current one is summed.
// The arithmetic of every row is the grid sweep's, in the same order, so the
// results are bit-identical.
constexpr int kIluPack = 4;
constexpr int kIluSBlock = 1024;
struct IluPackedSweep {
  const int* row;     // [n] row of level-ordered position p
  const int* k0;      // [n] first entry of the row's triangle (index into lu / colidx)
  const int* k1;      // [n] one past its last
  const int* col;     // [kIluPack n] the first kIluPack columns (0 where the row has fewer)
  const double* val;  // [kIluPack n] their factor entries (0 where the row has fewer)
  const double* piv;  // [n] u_ii (backward sweep only; null forward)
};
__global__ void __launch_bounds__(kIluSBlock) ilu_solve_smem(IluArgs a, IluPackedSweep L, IluPackedSweep U);

// One application recorded on `st` (capturable into a graph): the barrier
// counter is cleared, then the cooperative sweep runs (or returns at once if
// the gate is closed).
gsk_status ilu_launch_apply(gsk_ctx* ctx, const gsk_ilu0* h, const IluGate& gate, double* z, cudaStream_t st);

// Error bits the handle's launches recorded (synchronises `st`).
gsk_status ilu_read_err(gsk_ctx* ctx, const gsk_ilu0* h, cudaStream_t st);

}  // namespace gsk
