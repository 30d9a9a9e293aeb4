// CUDA graphs with a data-dependent loop: a captured prefix, a conditional
// while node, then a captured suffix.  The node's handle starts at 1 on every
// launch; the body's kernels set it (a first kernel clears it, a closing
// kernel sets it again when another iteration is due), so the loop stops by
// default.  The prefix may fork work onto other streams; the loop node waits
// for everything the capturing stream waits for at its end, and the suffix
// joins whatever is still outstanding.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace cgk {

// prefix(handle, stream), body(handle, stream) and suffix(stream) enqueue
// work on the capturing stream `cap`; *out receives the instantiated graph.
// instantiate_flags: e.g. cudaGraphInstantiateFlagUseNodePriority.
template <class Prefix, class Body, class Suffix>
cudaError_t build_loop_graph(cudaStream_t cap, Prefix prefix, Body body, Suffix suffix, cudaGraphExec_t* out,
                             unsigned long long instantiate_flags = 0) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  bool capturing = false;
  do {
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    if ((e = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      break;
    capturing = true;
    prefix(h, cap);
    // the loop node follows what the capturing stream currently depends on
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(cap, &status, nullptr, nullptr, &deps, nullptr, &nd)) != cudaSuccess) break;
    std::vector<cudaGraphNode_t> dep(deps, deps + nd);
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((e = cudaGraphAddNode(&loop, g, dep.data(), nullptr, dep.size(), &p)) != cudaSuccess) break;
    if ((e = cudaStreamUpdateCaptureDependencies(cap, &loop, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
      break;
    suffix(cap);
    cudaGraph_t captured = g;
    capturing = false;
    if ((e = cudaStreamEndCapture(cap, &captured)) != cudaSuccess) break;
    cudaGraph_t bodyg = p.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cap, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      break;
    body(h, cap);
    if ((e = cudaStreamEndCapture(cap, &bodyg)) != cudaSuccess) break;
    e = cudaGraphInstantiate(out, g, instantiate_flags);
  } while (0);
  if (capturing) {  // leave the stream usable after a failure inside the capture
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(cap, &junk);
  }
  cudaGraphDestroy(g);
  return e;
}

}  // namespace cgk
