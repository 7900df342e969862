// Internal declarations of the sm_103a face-operator / PISO library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/difvm.h"

namespace difvm {

// ----------------------------------------------------------------- errors
difvm_status set_error(difvm_status st, const char* fmt, ...);
void count_launch();
// algorithmic bytes of the kernels launched (each array a kernel must read or
// write counted once at its logical size: no padding, re-reads or caching);
// the solver kernels (Krylov, multigrid) add theirs at launch time
void count_bytes(uint64_t bytes);
void count_bytes_pause(bool paused);   // while paused (tuning runs), count_bytes adds nothing
difvm_status check_launch(const char* what);   // counts one launch, then check_error
difvm_status check_error(const char* what);    // pending launch error -> ECUDA

// --------------------------------------------------- per-kernel event timing
// When difvm_prof_start(tag) is active, launches wrapped in prof_before /
// prof_after with the same tag get a pair of CUDA events on their stream.
void prof_before(int tag, cudaStream_t s);
void prof_after(int tag, cudaStream_t s);
void prof_bytes(int tag, uint64_t bytes);   // algorithmic bytes of the launch prof_before bracketed
// PISO phase timing (difvm_phase_prof_start): phase_mark records an event on s
// that starts `phase` (DIFVM_PHASE_*, or -1: the step ended) and opens the
// matching NVTX range (the previous one closes); a no-op under stream capture.
void phase_mark(int phase, cudaStream_t s);
bool prof_active();

#define DIFVM_CUDA(call)                                                            \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::difvm::set_error(DIFVM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define DIFVM_TRY(expr)                                   \
  do {                                                    \
    difvm_status difvm_try_st_ = (expr);                  \
    if (difvm_try_st_ != DIFVM_OK) return difvm_try_st_;  \
  } while (0)

// ------------------------------------------- programmatic dependent launch
// A kernel started with launch_pdl may begin while the kernel before it in the
// stream is still finishing (its blocks are scheduled once every block of the
// predecessor is resident).  Such a kernel calls pdl_chain() first, in every
// thread and before any exit: griddepcontrol.wait returns once the predecessor
// has completed and its writes are visible, so completion still chains through
// every kernel; launch_dependents then lets the next kernel be scheduled.
__device__ __forceinline__ void pdl_chain() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... P, typename... A>
inline void launch_pdl(void (*k)(P...), unsigned grid, unsigned block, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, ((P)args)...);   // an error is left for check_error
}

// ------------------------------------------------------------ vector types
template <typename T> struct V4;
template <> struct __align__(16) V4<float> { float x, y, z, w; };
template <> struct __align__(32) V4<double> { double x, y, z, w; };

template <typename T>
__device__ __forceinline__ V4<T> ld4(const V4<T>* p);
template <>
__device__ __forceinline__ V4<float> ld4<float>(const V4<float>* p) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return V4<float>{v.x, v.y, v.z, v.w};
}
template <>
__device__ __forceinline__ V4<double> ld4<double>(const V4<double>* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return V4<double>{a.x, a.y, b.x, b.y};
}

// Per-precision device geometry, internal numbering.
template <typename T> struct Geo {
  const V4<T>* Sw;  // [nf] (Sx, Sy, Sz, w_f); w_f = owner weight (1 on boundary faces)
  const V4<T>* ck;  // [nf] (c_f, kx, ky, kz); k = 0 on boundary faces
  const T* V;       // [nc]
  const T* rV;      // [nc]
};

// Topology, internal numbering, passed by value to kernels.
struct Topo {
  int nc, ni, nf, nb;
  const int2* on;          // [ni] (owner, neighbour), owner < neighbour, sorted
  const int* bown;         // [nb] owner of boundary face ni + b
  const int* cptr;         // [nc+1] cell-CSR row pointers
  const int* cent;         // [nnz]  (face << 1) | side, ascending face id per cell
  const uint8_t* bkind;    // [nb] 2 bits per bc class: kind = (bkind >> (2*cls)) & 3
  const uint16_t* bpatch;  // [nb] patch id
};

// ELL layout of the off-diagonal entries of the LDU operator, used inside the
// Krylov solvers.  Uniform width W > 0: slot k of row i is at i W + k (row
// major).  Otherwise sliced ELL (slice height 32): row i lives in slice i/32 at
// lane i%32 and slot k is at soff[slice] + 32 k + lane.  col is the column (the
// row itself on padding), map the source entry (face << 1 | side, side 1 = row
// is the neighbour) or -1 on padding.
struct Ell {
  int nsl;
  int W;            // > 0: uniform row-major width; 0: sliced with per-slice widths
  const int* soff;  // [nsl+1]
  const int* col;   // [nslots]
  const int* map;   // [nslots]
  // W == 4 and every |column - row| < 2^15: the columns of row i again, as
  // 16-bit offsets from i (one 8-byte load instead of 16); else null
  const short4* c16;
};
// the four columns of row i of a uniform width-4 ELL
__device__ __forceinline__ int4 ell_cols4(const Ell& E, int i) {
  if (E.c16) {
    const short4 d = __ldg(E.c16 + i);
    return make_int4(i + d.x, i + d.y, i + d.z, i + d.w);
  }
  return __ldg(reinterpret_cast<const int4*>(E.col) + i);
}

// Boundary faces as the face operators see them: a patch is "empty" (the face
// drops out of every sum), an outlet (fixed pressure, zero-gradient velocity)
// or anything else (fixed velocity, zero-gradient pressure).  The kind of a
// face for a boundary-condition class follows from that category alone.
enum { kCatOther = 0, kCatOutlet = 1, kCatEmpty = 2 };
__host__ __device__ __forceinline__ int patch_cat(int patch_type) {
  return patch_type == DIFVM_PATCH_EMPTY ? kCatEmpty : (patch_type == DIFVM_PATCH_OUTLET ? kCatOutlet : kCatOther);
}
__host__ __device__ __forceinline__ int bc_kind(int cls, int cat) {
  if (cat == kCatEmpty) return DIFVM_FACE_EMPTY;
  switch (cls) {
    case DIFVM_BC_VELOCITY: return cat == kCatOutlet ? DIFVM_FACE_ZEROGRAD : DIFVM_FACE_FIXED;
    case DIFVM_BC_PRESSURE: return cat == kCatOutlet ? DIFVM_FACE_FIXED : DIFVM_FACE_ZEROGRAD;
    case DIFVM_BC_ALL_FIXED: return DIFVM_FACE_FIXED;
    default: return DIFVM_FACE_ZEROGRAD;
  }
}

// Half-face layout of the cell-CSR rows (every face of a cell, internal and
// boundary, in ascending face order), for the face operators: sliced ELL with
// slice height 32, column-major in a slice (slot k of row i at
// soff[i/32] + 32 k + i%32; with a uniform width W > 0 soff is not read).
// nb[slot] = 2 j + side for an internal face (j the other cell, side 1 = row is
// the neighbour), -2 - (4 b + cat) for boundary face ni + b of patch category
// cat (so a kernel knows the face's boundary kind without another load), -1 on
// padding; fid[slot] = face id; nf[slot] = (nb, fid) in one 8-byte word.  The
// Sw face records are also copied into slot order (a row's records then come
// in with coalesced loads, without the face id).
// Compact form (cw, fb; null where the mesh's numbering does not fit it): one
// 4-byte word per slot carrying both the other cell and the face id.  An
// internal slot of row i holds bit 31 = 0, bits 30..16 = j - i (15-bit signed,
// never 0; its sign gives the side: j < i means the row is the neighbour) and
// bits 15..0 = f - fb[i/32] (16-bit signed), fb[s] = the first face owned by
// row 32 s; boundary and padding slots hold the nb word (negative).  RCM keeps
// j - i within the ordering's bandwidth, so the 64^3 Kuhn mesh (|j - i| <= 7.7k,
// f - fb >= -15.4k) fits.
struct Hf {
  int W;
  const int* soff;
  const int* nb;
  const int* fid;
  const int2* nf;
  const int* cw;
  const int* fb;
  int ni;
};
// boundary face index and patch category of a boundary slot word (v <= -2)
__device__ __forceinline__ int hf_bface(int v) { return (-2 - v) >> 2; }
__device__ __forceinline__ int hf_bcat(int v) { return (-2 - v) & 3; }
// largest boundary-face count the slot words can encode
constexpr int kMaxBoundaryFaces = (1 << 29) - 1;
// face records as a face kernel reads them: by slot (sw = the slot copies,
// ck unused) or by face id (sw, ck = the face arrays)
template <typename T> struct HfGeo {
  const V4<T>* sw;
  const V4<T>* ck;
  const T* w;     // w_f by face id (internal faces)
};
__device__ __forceinline__ void hf_row(const Hf& H, int i, int& base, int& w) {
  if (H.W > 0) {
    base = (i >> 5) * 32 * H.W + (i & 31);
    w = H.W;
  } else {
    const int o = __ldg(H.soff + (i >> 5));
    base = o + (i & 31);
    w = (__ldg(H.soff + (i >> 5) + 1) - o) >> 5;
  }
}

// first slot and slot stride of row i
__device__ __forceinline__ void ell_row(const Ell& E, int i, int& base, int& step, int& w) {
  if (E.W > 0) {
    base = i * E.W;
    step = 1;
    w = E.W;
  } else {
    const int o = __ldg(E.soff + (i >> 5));
    base = o + (i & 31);
    step = 32;
    w = (__ldg(E.soff + (i >> 5) + 1) - o) >> 5;
  }
}

__device__ __forceinline__ int face_kind(const Topo& t, int b, int cls) {
  return (t.bkind[b] >> (2 * cls)) & 3;
}

struct difvm_mesh_impl;
struct AmgHier;
void amg_free(AmgHier* h);
struct DicLevels;
void dic_free(DicLevels* d);
}  // namespace difvm

// The opaque handle of the C ABI.
struct difvm_mesh {
  int device;
  int nc, ni, nf, nb, npatch, ncases;
  int64_t nnz;
  int max_row;                       // largest CSR row length
  std::vector<int32_t> cell_new_of_old, face_old_of_new, case_start;
  std::vector<int8_t> face_flip;
  std::vector<int32_t> patch_start, patch_size, patch_type;
  // device allocations
  int2* on = nullptr;
  int* bown = nullptr;
  int* cptr = nullptr;
  int* cent = nullptr;
  uint8_t* bkind = nullptr;
  uint16_t* bpatch = nullptr;
  int ell_nsl = 0;
  int ell_w = 0;      // uniform slice width, or 0
  int ell_wmax = 0;   // widest row
  int64_t ell_nslots = 0;
  int* ell_soff = nullptr;
  int* ell_col = nullptr;
  int* ell_map = nullptr;
  short4* ell_c16 = nullptr;   // see difvm::Ell
  difvm::V4<double>* Sw64 = nullptr;
  difvm::V4<double>* ck64 = nullptr;
  difvm::V4<float>* Sw32 = nullptr;
  difvm::V4<float>* ck32 = nullptr;
  double *V64 = nullptr, *rV64 = nullptr, *C64 = nullptr, *Cf64 = nullptr;
  float *V32 = nullptr, *rV32 = nullptr;
  int num_sms = 148;
  // Segmented (batched) solves: set when the mesh was created with a case
  // table.  Solver block b works on rows [cs[k] + j*seg_rows, ...) of case
  // k = seg_case[b], j = b - seg_cb0[k]; a case's blocks are contiguous.
  bool seg = false;
  int seg_nblk = 0;
  int* seg_case = nullptr;   // [seg_nblk]
  int* seg_cb0 = nullptr;    // [ncases + 1]
  int* seg_cs = nullptr;     // [ncases + 1] first cell of each case
  std::vector<int32_t> bown_host;  // boundary-face owners, internal numbering
  difvm::AmgHier* amg = nullptr;   // multigrid hierarchy, built on first use
  difvm::DicLevels* dic = nullptr; // incomplete-Cholesky dependency levels, built on first use
  // half-face layout of the CSR rows (see difvm::Hf)
  int hf_w = 0;
  int64_t hf_nslots = 0;
  int* hf_soff = nullptr;
  int* hf_nb = nullptr;
  int* hf_fid = nullptr;
  int2* hf_nf = nullptr;
  int* hf_cw = nullptr;      // compact slot words, or null (see difvm::Hf)
  int* hf_fb = nullptr;      // [slices] first face owned by each slice's first row
  // face-operator launch variants picked by first-use timing (see ops.cu):
  // key -> variant, and whether timing is allowed
  std::vector<std::pair<uint32_t, int>> tuned;
  int autotune = 1;
  // multigrid: levels below amg_tail_rows rows run in one fused launch of
  // amg_tail_bps blocks per SM (-1: the library's choice)
  int amg_tail_rows = -1, amg_tail_bps = -1;
  difvm::V4<double>* hf_sw64 = nullptr;
  difvm::V4<float>* hf_sw32 = nullptr;
  double* w64 = nullptr;     // [ni] w_f, FP64 and FP32 copies
  float* w32 = nullptr;

  difvm::Topo topo() const {
    return difvm::Topo{nc, ni, nf, nb, on, bown, cptr, cent, bkind, bpatch};
  }
  difvm::Ell ell() const { return difvm::Ell{ell_nsl, ell_w, ell_soff, ell_col, ell_map, ell_c16}; }
  difvm::Hf hf() const { return difvm::Hf{hf_w, hf_soff, hf_nb, hf_fid, hf_nf, hf_cw, hf_fb, ni}; }
  difvm::HfGeo<double> hfgeo64() const { return {hf_sw64, nullptr, w64}; }
  difvm::HfGeo<float> hfgeo32() const { return {hf_sw32, nullptr, w32}; }
  difvm::Geo<double> geo64() const { return {Sw64, ck64, V64, rV64}; }
  difvm::Geo<float> geo32() const { return {Sw32, ck32, V32, rV32}; }
};

namespace difvm {
template <typename T> inline Geo<T> geo(const difvm_mesh* m);
template <> inline Geo<double> geo<double>(const difvm_mesh* m) { return m->geo64(); }
template <> inline Geo<float> geo<float>(const difvm_mesh* m) { return m->geo32(); }
template <typename T> inline HfGeo<T> hfgeo(const difvm_mesh* m);
template <> inline HfGeo<double> hfgeo<double>(const difvm_mesh* m) { return m->hfgeo64(); }
template <> inline HfGeo<float> hfgeo<float>(const difvm_mesh* m) { return m->hfgeo32(); }

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// rows per block of the segmented (batched) Krylov kernels: 512 threads x 4 rows
constexpr int kSegRows = 2048;

// --------------------------------------------- CUDA-graph device loops (graph.cu)
bool stream_capturing(cudaStream_t st);
struct WhileLoop {
  cudaStream_t side = nullptr;  // stream that captures the loop body
  cudaGraph_t body = nullptr;
  cudaGraphConditionalHandle h = 0;
  bool open = false;
};
// Adds a conditional WHILE node at the capture point of `st` and starts
// capturing its body on L.side; while_close ends the body capture.
difvm_status while_open(cudaStream_t st, WhileLoop& L);
difvm_status while_close(WhileLoop& L);
// loop condition: any of n int flags (stride_ints apart) is 0, and the body has
// run fewer than `cap` times
__global__ void k_loop_cond(const int* done_flags, int stride_ints, int n, int* counter, int cap,
                            cudaGraphConditionalHandle h);
// iterations per loop-body execution when a solve runs inside a graph
constexpr int kGraphUnroll = 4;

// ------------------------------------- multigrid-preconditioned CG (amg.cu)
difvm_status amg_hier(difvm_mesh* m, AmgHier** out);
void amg_retune(difvm_mesh* m, int mode);   // difvm_mesh_autotune's mode, applied to the hierarchy
size_t amg_workspace_bytes(difvm_mesh* m, size_t elt);
template <typename T>
difvm_status amg_solve(difvm_mesh* m, const difvm_solve_opts* o, const T* D, const T* Lo, const T* b,
                       T* x, void* ws, size_t wsbytes, difvm_solve_info* info, cudaStream_t st);
difvm_status amg_prebuild(difvm_mesh* m, size_t elt, const void* D, const void* Lo, void* ws, size_t wsbytes,
                          cudaStream_t st);
difvm_status amg_refine(difvm_mesh* m, const difvm_solve_opts* o, const float* D, const float* Lo,
                        const double* b64, double* x64, void* ws, size_t wsbytes, difvm_solve_info* info,
                        cudaStream_t st);
// ---------------------------- incomplete-Cholesky-preconditioned CG (dic.cu)
size_t dic_workspace_bytes(difvm_mesh* m, size_t elt);
template <typename T>
difvm_status dic_solve(difvm_mesh* m, const difvm_solve_opts* o, const T* D, const T* Lo, const T* b,
                       T* x, void* ws, size_t wsbytes, difvm_solve_info* info, cudaStream_t st);
// incomplete factorisations in single-launch level sweeps (dic.cu): DILU of
// (D, L, U), DIC when U == L or null; `extra` holds ilu_extra_bytes of workspace
size_t ilu_extra_bytes(const difvm_mesh* m, size_t elt);
struct KState;
template <typename T>
difvm_status ilu_factor(difvm_mesh* m, const T* D, const T* L, const T* U, char* extra, KState* st, int nst,
                        cudaStream_t s);
template <typename T>
difvm_status ilu_apply(difvm_mesh* m, int ncomp, const T* L, const T* U, char* extra, const T* r, T* z,
                       KState* st, int nst, cudaStream_t s);
difvm_status check_mesh(const difvm_mesh* m);
difvm_status check_prec(difvm_prec p);

// cross-file launchers (ops.cu)
template <typename T>
difvm_status grad_gauss_t(difvm_mesh_t m, int cls, const void* phi, const void* phib, int ncomp,
                          void* grad, cudaStream_t s);
template <typename T>
difvm_status ldu_apply_t(difvm_mesh_t m, const void* D, const void* L, const void* U,
                         const void* x, int ncomp, int transpose, void* y, cudaStream_t s);
}  // namespace difvm
