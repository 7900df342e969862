// Adjoint of the LDU operator apply for callers that cannot allocate.
//
// difvm_laplacian_apply_bwd needs a scratch vector for A^T y_bar, which the
// caller passes in.  Some callers have no way to provide one: a host program
// whose device memory is entirely owned by another runtime's pool, or a
// time-critical loop that must not call cudaMalloc (it can synchronise the
// whole device).  This file gives them a variant whose scratch is a
// file-scope device array, reserved once per GPU when the library is loaded.
#include <mutex>

#include "difvm_internal.cuh"

namespace difvm {

// Scratch for A^T y_bar: 16 MiB, i.e. ncomp * n_cells elements of the call's
// precision must fit (FP64: 2,097,152 elements; FP32: 4,194,304).
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, looked up once per device with that device current.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

static difvm_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= 64) return set_error(DIFVM_EINVAL, "device %d out of range", device);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    int cur = -1;
    DIFVM_CUDA(cudaGetDevice(&cur));
    if (cur != device) DIFVM_CUDA(cudaSetDevice(device));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess)
      return set_error(DIFVM_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return DIFVM_OK;
}

template <typename T>
__global__ void k_noalloc_accumulate(int n, const T* __restrict__ a, T* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] += a[i];
}

}  // namespace difvm

using namespace difvm;

extern "C" difvm_status difvm_laplacian_apply_bwd_noalloc(difvm_mesh_t m, difvm_prec prec,
                                                          const void* D, const void* L,
                                                          const void* U, const void* x,
                                                          const void* ybar, int ncomp, void* xbar,
                                                          void* Dbar, void* Lbar, void* Ubar,
                                                          void* stream) {
  DIFVM_TRY(check_mesh(m));
  DIFVM_TRY(check_prec(prec));
  if (ncomp < 1 || ncomp > 3) return set_error(DIFVM_EINVAL, "ncomp must be 1..3 (got %d)", ncomp);
  if (!D || (!L && m->ni > 0) || !x || !ybar) return set_error(DIFVM_EINVAL, "null field");
  const size_t elt = prec == DIFVM_F64 ? 8 : 4;
  const size_t need = elt * (size_t)ncomp * (size_t)m->nc;
  if (xbar && need > kNoAllocScratchBytes)
    return set_error(DIFVM_EINVAL,
                     "difvm_laplacian_apply_bwd_noalloc: %d x %d cells need %zu bytes of scratch, "
                     "the built-in maximum is %zu bytes",
                     ncomp, m->nc, need, kNoAllocScratchBytes);
  // the kernels launch on the current device, and the scratch and the mesh
  // arrays belong to the mesh's device: the two must be the same
  int cur = -1;
  DIFVM_CUDA(cudaGetDevice(&cur));
  if (cur != m->device)
    return set_error(DIFVM_EINVAL,
                     "difvm_laplacian_apply_bwd_noalloc: current device %d is not the mesh's device %d",
                     cur, m->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (xbar) {
    void* scratch = nullptr;
    DIFVM_TRY(noalloc_scratch(m->device, &scratch));
    // scratch = A^T y_bar overwrites every element it uses: nothing to clear
    DIFVM_TRY(prec == DIFVM_F64 ? ldu_apply_t<double>(m, D, L, U, ybar, ncomp, 1, scratch, st)
                                : ldu_apply_t<float>(m, D, L, U, ybar, ncomp, 1, scratch, st));
    const int n = ncomp * m->nc;
    if (prec == DIFVM_F64)
      k_noalloc_accumulate<double><<<blocks_for(n, 256), 256, 0, st>>>(n, (const double*)scratch,
                                                                        (double*)xbar);
    else
      k_noalloc_accumulate<float><<<blocks_for(n, 256), 256, 0, st>>>(n, (const float*)scratch,
                                                                       (float*)xbar);
    DIFVM_TRY(check_launch("noalloc_accumulate"));
  }
  if (Dbar || Lbar || Ubar)  // coefficient gradients need no scratch
    return difvm_laplacian_apply_bwd(m, prec, D, L, U, x, ybar, ncomp, nullptr, Dbar, Lbar, Ubar,
                                     nullptr, stream);
  return DIFVM_OK;
}
