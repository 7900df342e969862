// Device-driven loops for CUDA-graph execution.
//
// A Krylov solve normally runs a host loop that reads the convergence flags
// every few iterations.  While a stream is being captured into a CUDA graph the
// host cannot read anything, so the solve is emitted instead as a conditional
// WHILE node: its body graph holds a few iterations plus a one-thread kernel
// that sets the loop condition from the device-side solver state.  The whole
// PISO step then runs as one graph launch with no host round trip.
#include "difvm_internal.cuh"

namespace difvm {

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus s = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &s) == cudaSuccess && s == cudaStreamCaptureStatusActive;
}

// sets a loop's condition to 1 just before the loop node runs
__global__ void k_loop_start(cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, 1u);
}

// Non-blocking streams used only to capture loop bodies: one per device and
// nesting depth (a loop inside a loop body captures on the next one), per host
// thread, so concurrent captures on different threads never share one.
constexpr int kMaxLoopDepth = 4;
static thread_local cudaStream_t t_side[64][kMaxLoopDepth] = {};
static thread_local int t_depth = 0;

difvm_status while_open(cudaStream_t st, WhileLoop& L) {
  int dev = 0;
  DIFVM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(DIFVM_EINVAL, "device %d out of range", dev);
  if (t_depth >= kMaxLoopDepth) return set_error(DIFVM_EINVAL, "device loops nested too deeply");
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  DIFVM_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &ndeps));
  if (cs != cudaStreamCaptureStatusActive) return set_error(DIFVM_EINVAL, "stream is not capturing");
  DIFVM_CUDA(cudaGraphConditionalHandleCreate(&L.h, g, 1u, cudaGraphCondAssignDefault));
  // The default value is applied when the top-level graph is launched, not each
  // time a loop nested in another loop's body starts: set it from the graph
  // itself, with a kernel that runs just before the loop node.
  k_loop_start<<<1, 32, 0, st>>>(L.h);
  DIFVM_TRY(check_error("loop_start"));
  DIFVM_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &ndeps));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = L.h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  DIFVM_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
  L.body = np.conditional.phGraph_out[0];
  DIFVM_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaStream_t& side = t_side[dev][t_depth];
  if (!side) DIFVM_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
  L.side = side;
  DIFVM_CUDA(cudaStreamBeginCaptureToGraph(L.side, L.body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed));
  ++t_depth;
  L.open = true;
  return DIFVM_OK;
}

difvm_status while_close(WhileLoop& L) {
  if (!L.open) return DIFVM_OK;
  cudaGraph_t g = L.body;
  cudaError_t e = cudaStreamEndCapture(L.side, &g);
  L.open = false;
  --t_depth;
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
