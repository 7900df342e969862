// Device-driven loops for CUDA-graph execution.
//
// A Krylov solve normally runs a host loop that reads the convergence flags
// every few iterations.  While a stream is being captured into a CUDA graph the
// host cannot read anything, so the solve is emitted instead as a conditional
// WHILE node: its body graph holds a few iterations plus a one-thread kernel
// that sets the loop condition from the device-side solver state.  The whole
// PISO step then runs as one graph launch with no host round trip.
#include <mutex>

#include "difvm_internal.cuh"

namespace difvm {

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus s = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &s) == cudaSuccess && s == cudaStreamCaptureStatusActive;
}

// one non-blocking stream per device, used only to capture loop bodies
static std::mutex g_side_mu;
static cudaStream_t g_side[64] = {nullptr};

static difvm_status side_stream(cudaStream_t* out) {
  int dev = 0;
  DIFVM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(DIFVM_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_side_mu);
  if (!g_side[dev]) DIFVM_CUDA(cudaStreamCreateWithFlags(&g_side[dev], cudaStreamNonBlocking));
  *out = g_side[dev];
  return DIFVM_OK;
}

difvm_status while_open(cudaStream_t st, WhileLoop& L) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  DIFVM_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &ndeps));
  if (cs != cudaStreamCaptureStatusActive) return set_error(DIFVM_EINVAL, "stream is not capturing");
  DIFVM_CUDA(cudaGraphConditionalHandleCreate(&L.h, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = L.h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  DIFVM_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
  L.body = np.conditional.phGraph_out[0];
  DIFVM_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  DIFVM_TRY(side_stream(&L.side));
  g_side_mu.lock();   // one body capture at a time on the side stream
  cudaError_t e = cudaStreamBeginCaptureToGraph(L.side, L.body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    g_side_mu.unlock();
    return set_error(DIFVM_ECUDA, "capture of a loop body: %s", cudaGetErrorString(e));
  }
  L.open = true;
  return DIFVM_OK;
}

difvm_status while_close(WhileLoop& L) {
  if (!L.open) return DIFVM_OK;
  cudaGraph_t g = L.body;
  cudaError_t e = cudaStreamEndCapture(L.side, &g);
  L.open = false;
  g_side_mu.unlock();
  if (e != cudaSuccess) return set_error(DIFVM_ECUDA, "end of a loop-body capture: %s", cudaGetErrorString(e));
  return DIFVM_OK;
}

// condition of a solver loop: 1 while any state is active and the body has run
// fewer than `cap` times (the cap bounds the loop even if a state never closes)
__global__ void k_loop_cond(const int* done_flags, int stride_ints, int n, int* counter, int cap,
                            cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int any = 0;
  for (int c = 0; c < n; ++c) any |= done_flags[c * stride_ints] == 0;
  const int k = *counter + 1;
  *counter = k;
  cudaGraphSetConditional(h, (any && k < cap) ? 1u : 0u);
}

}  // namespace difvm
