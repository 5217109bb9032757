// Pieces shared by the solvers that run a whole small system on one
// thread-block cluster (cluster_small.cu: Bi-CGSTAB; cluster_gmres.cu:
// GMRES(m)): the cluster shape, the deterministic cluster-wide sums and the
// launch.
//
// CTA c of the cluster owns rows [c * rpc, (c + 1) * rpc) (rpc = ceil(n / 16))
// and keeps its part of every vector in its shared memory; products gather
// the entries other CTAs own through distributed shared memory.  A sum over
// the cluster is formed per CTA in a fixed order, published in the CTA's
// shared memory, and after one cluster barrier every CTA adds the 16 partials
// in the same fixed tree, so every CTA holds bit-identical totals and takes
// the same decisions without further exchange.  The cluster barrier is the
// hardware's (all CTAs of a cluster are resident together): no spin-wait.
#pragma once

#include <cooperative_groups.h>

#include "internal.hpp"

namespace gsk {

namespace cg = cooperative_groups;

constexpr int kClusterCtas = 16;  // CTAs per cluster (a non-portable size)
constexpr int kClusterThreads = 512;

// The 16 published partials of value v (mine: this CTA's publication
// buffer; the same offset in every CTA), loaded at once and added in a fixed
// pairwise tree.
__device__ __forceinline__ double cluster_gather_sum(cg::cluster_group& cl, double* mine, int v) {
  double q[kClusterCtas];
#pragma unroll
  for (int c = 0; c < kClusterCtas; ++c) q[c] = cl.map_shared_rank(mine, c)[v];
#pragma unroll
  for (int h = kClusterCtas / 2; h >= 1; h >>= 1)
#pragma unroll
    for (int c = 0; c < h; ++c) q[c] += q[c + h];
  return q[0];
}

// Sum over the CTA's threads of NV values, then over the cluster's CTAs.
// red: this CTA's two publication buffers of 8 values (alternating by
// `round`, so that a CTA may publish the next sums while another still reads
// the previous ones); wsum: per-warp scratch [16][NV]; the totals land in
// tot (shared; valid in every thread of every CTA after the call).  Only the
// first `nw` warps hold rows (the others' values are zero and are left out:
// on this part an FP64 addition costs its pipe time whatever its operands).
template <int NV>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, const double (&v)[NV], double* red,
                                            double* wsum, double* tot, int& round, int nw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < nw) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double s = warp_allsum(v[k]);
      if (lane == 0) wsum[wid * NV + k] = s;
    }
  }
  __syncthreads();
  double* mine = red + (round & 1) * 8;
  if (threadIdx.x < NV) {
    // the warps' sums in a fixed pairwise tree over the nw warps that hold
    // rows (the additions of the empty slots' zeros are skipped: the same
    // sums, and on this part every FP64 instruction costs its pipe time)
    double q[kClusterThreads / 32];
#pragma unroll
    for (int w = 0; w < kClusterThreads / 32; ++w) q[w] = w < nw ? wsum[w * NV + threadIdx.x] : 0.0;
#pragma unroll
    for (int h = kClusterThreads / 64; h >= 1; h >>= 1)
#pragma unroll
      for (int w = 0; w < h; ++w)
        if (w + h < nw) q[w] += q[w + h];
    mine[threadIdx.x] = q[0];
  }
  cl.sync();
  if (threadIdx.x < NV) tot[threadIdx.x] = cluster_gather_sum(cl, mine, threadIdx.x);
  __syncthreads();
  round += 1;
}

// Launch of a cluster kernel: one cluster of kClusterCtas CTAs of
// kClusterThreads threads with `smem` bytes of dynamic shared memory.
template <typename Args>
inline cudaError_t cluster_launch(void (*kernel)(Args), const Args& a, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kClusterCtas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, a);
}

// The dynamic shared memory a cluster kernel can have on this device (the
// opt-in limit less its static shared memory), after checking that a
// cluster of that shape fits; 0 when it does not (the kernel is then not
// used).  Sets the kernel's attributes on the way.
template <typename Args>
inline int cluster_smem_limit(void (*kernel)(Args), int device) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, (const void*)kernel) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  optin -= (int)fa.sharedSizeBytes;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kClusterCtas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = (size_t)optin;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&nclusters, (const void*)kernel, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return 0;
  }
  return optin;
}

}  // namespace gsk
