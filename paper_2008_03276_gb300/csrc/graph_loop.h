// graph_loop.h -- device-driven loops for CUDA graphs: while-nodes whose condition a kernel
// sets on the device (the Newton, GMRES and line-search loops of a solve as one graph).
#pragma once
#include <cuda_runtime.h>

#include "ehl_internal.h"

namespace ehl {

// next = 0: *counter = 0 (before the loop); next = 1: *counter += 1 and *total += 1 (end of a
// pass).  Sets the loop's condition: continue while *counter < cap and some instance z has
// done[z] == 0 and other[z] == 0 (other nullable).  One block.
__global__ void k_nk_loop(cudaGraphConditionalHandle h, int* __restrict__ counter, int* __restrict__ total, int cap,
                          int next, const int* __restrict__ done, const int* __restrict__ other, int ni);

// A while-node appended to the graph captured on `outer`: `start` (launched on outer) sets the
// first condition, the body is captured from what `body` launches on `inner`; c->st follows.
template <class Ctx, class Start, class Body>
cudaError_t capture_while(Ctx* c, cudaStream_t outer, cudaStream_t inner, Start start, Body body,
                          long long* body_launches) {
  cudaStreamCaptureStatus stt;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(outer, &stt, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (stt != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle h = 0;
  e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  if (e != cudaSuccess) return e;
  c->st = outer;
  e = start(h);
  if (e != cudaSuccess) return e;
  e = cudaStreamGetCaptureInfo(outer, &stt, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
  if (e != cudaSuccess) return e;
  cudaGraph_t bg = p.conditional.phGraph_out[0];
  e = cudaStreamUpdateCaptureDependencies(outer, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(inner, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  c->st = inner;
  const unsigned long long l0 = thread_launches();
  const cudaError_t eb = body(h);
  if (body_launches) *body_launches = (long long)(thread_launches() - l0);
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(inner, &out);
  c->st = outer;
  return eb != cudaSuccess ? eb : e;
}


}  // namespace ehl
