// CUDA graphs with a data-dependent loop: a captured prefix followed by a
// conditional while node whose body is captured separately.  The node's
// handle starts at 1 on every launch; the body's kernels set it (a first
// kernel clears it, a closing kernel sets it again when another iteration is
// due), so the loop stops by default.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace cgk {

// prefix(handle, stream) and body(handle, stream) enqueue kernels on the
// capturing stream `cap`; *out receives the instantiated graph.
template <class Prefix, class Body>
cudaError_t build_loop_graph(cudaStream_t cap, Prefix prefix, Body body, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  do {
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    if ((e = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      break;
    prefix(h, cap);
    cudaGraph_t captured = g;
    if ((e = cudaStreamEndCapture(cap, &captured)) != cudaSuccess) break;
    // the captured prefix is a chain: its one node without dependents
    size_t nn = 0;
    if ((e = cudaGraphGetNodes(g, nullptr, &nn)) != cudaSuccess) break;
    std::vector<cudaGraphNode_t> nodes(nn);
    if ((e = cudaGraphGetNodes(g, nodes.data(), &nn)) != cudaSuccess) break;
    cudaGraphNode_t leaf = nullptr;
    for (cudaGraphNode_t node : nodes) {
      size_t nd = 0;
      if ((e = cudaGraphNodeGetDependentNodes(node, nullptr, nullptr, &nd)) != cudaSuccess) break;
      if (nd == 0) leaf = node;
    }
    if (e != cudaSuccess) break;
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((e = cudaGraphAddNode(&loop, g, leaf ? &leaf : nullptr, nullptr, leaf ? 1 : 0, &p)) != cudaSuccess) break;
    cudaGraph_t bodyg = p.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cap, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      break;
    body(h, cap);
    if ((e = cudaStreamEndCapture(cap, &bodyg)) != cudaSuccess) break;
    e = cudaGraphInstantiate(out, g, 0);
  } while (0);
  cudaGraphDestroy(g);
  return e;
}

}  // namespace cgk
