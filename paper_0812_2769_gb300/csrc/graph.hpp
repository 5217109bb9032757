// Helpers to build solver graphs: kernels are recorded by stream capture
// into graphs (or conditional-node bodies), and device-evaluated WHILE / IF
// nodes carry the iteration control, so a whole solve is one graph launch
// with no host round trip.
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace gsk {

// Records kernels launched on `s` into graph `g` after `deps`; on end() the
// nodes the next addition must depend on are kept in `tail`.
struct Capture {
  cudaStream_t s = nullptr;
  cudaGraph_t g = nullptr;
  std::vector<cudaGraphNode_t> tail;

  cudaError_t begin(cudaStream_t s_, cudaGraph_t g_, const std::vector<cudaGraphNode_t>& deps = {}) {
    s = s_;
    g = g_;
    return cudaStreamBeginCaptureToGraph(s, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                         cudaStreamCaptureModeThreadLocal);
  }
  cudaError_t end() {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &d, nullptr, &nd);
    if (e == cudaSuccess) tail.assign(d, d + nd);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &out);
    return e != cudaSuccess ? e : e2;
  }
};

// Adds a conditional node to `g`; its body graphs are returned in bodies[].
inline cudaError_t add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                                   cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                   unsigned size, cudaGraphNode_t* node, cudaGraph_t* bodies) {
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = size;
  cudaError_t e = cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &np);
  if (e != cudaSuccess) return e;
  for (unsigned i = 0; i < size; ++i) bodies[i] = np.conditional.phGraph_out[i];
  return cudaSuccess;
}

}  // namespace gsk
