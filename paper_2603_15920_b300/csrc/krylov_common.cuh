// Building blocks shared by the Krylov solvers (krylov.cu) and the multigrid
// preconditioner (amg.cu): device-resident solver states, the deterministic
// two-level grid reductions, and one row of the sliced-ELL SpMV.
#pragma once

#include <math.h>
#include <stddef.h>

#include "difvm_internal.cuh"

namespace difvm {

constexpr int kKB = 512;       // threads per block (four blocks per SM: few partials, few atomics)
constexpr int kMaxParts = 12;  // partial sums per block (<= 4 per component x 3)

struct KState {
  double rr, rz, bb, tol2, alpha, beta, rho, omega, pq, res0;
  int iters, done, status, sconv;
  int zero_rhs, pad0, pad1, pad2;
};

static_assert(sizeof(KState) % sizeof(int) == 0, "KState must be a whole number of ints");
constexpr int kStateInts = (int)(sizeof(KState) / sizeof(int));
inline const int* done_flags(const KState* st) {
  return reinterpret_cast<const int*>(reinterpret_cast<const char*>(st) + offsetof(KState, done));
}

struct KWork {
  KState* st;        // [ncomp]
  double* part;      // [grid * kMaxParts]
  unsigned* ticket;  // 1
  int maxit;
  double tol_rel, tol_abs;
};

// Matrix inside the solvers: diagonal + sliced-ELL off-diagonal values (filled
// from the LDU face coefficients once per solve by k_ell_fill).
template <typename T> struct Mat {
  const T* D;
  Ell E;
  const T* val;  // [nslots]
};

// val[slot] = side ? L_f : U_f  (row N holds L_f x_O, row O holds U_f x_N); 0 on padding
template <typename T>
__global__ void k_ell_fill(int nslots, const int* map, const T* L, const T* U, T* val) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nslots) return;
  const int e = map[k];
  val[k] = e < 0 ? T(0) : ((e & 1) ? L[e >> 1] : U[e >> 1]);
}

// ---------------------------------------------------------- accumulators
template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
  using part_t = double;
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double get() const { return s; }
  __device__ __forceinline__ double part() const { return s; }
};
// Dot2: error-free TwoProduct (fma) + TwoSum, errors accumulated in c.
template <> struct DotAcc<float> {
  float p = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float h = __fmul_rn(a, b);
    const float r = __fmaf_rn(a, b, -h);
    const float s = __fadd_rn(p, h);
    const float z = __fsub_rn(s, p);
    const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(s, z)), __fsub_rn(h, z));
    p = s;
    c = __fadd_rn(c, __fadd_rn(q, r));
  }
  __device__ __forceinline__ double get() const { return (double)p + (double)c; }
  // unevaluated (hi, lo) pair, reduced across threads in FP32 by ff_merge
  using part_t = float2;
  __device__ __forceinline__ float2 part() const { return make_float2(p, c); }
};

// error-free merge of two float-float pairs (TwoSum on the leading parts, then
// renormalisation), so cross-thread sums stay on the FP32 pipes
__device__ __forceinline__ float2 ff_merge(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(s, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, z)), __fsub_rn(b.x, z));
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float hi = __fadd_rn(s, e);
  return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

// block reduction of K doubles; result valid in thread 0
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double sm[K][kKB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sm[k][warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      v[k] = lane < (int)(blockDim.x >> 5) ? sm[k][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
  }
  __syncthreads();
}

// Store this block's partials; return true in the last block, with the grid
// totals in `tot` (valid in all threads of that block).
template <int K>
__device__ __forceinline__ bool grid_sum(const KWork& w, double (&v)[K], double (&tot)[K]) {
  block_sum<K>(v);
  __shared__ int amlast;
  __shared__ double res[K];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) w.part[blockIdx.x * kMaxParts + k] = v[k];
    __threadfence();
    amlast = atomicAdd(w.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  double a[K];
#pragma unroll
  for (int k = 0; k < K; ++k) a[k] = 0.0;
#pragma unroll 4
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] += __ldcg(w.part + b * kMaxParts + k);
  block_sum<K>(a);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) res[k] = a[k];
    *w.ticket = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = res[k];
  return true;
}

// FP32-pair version: warp and block trees merge (hi, lo) pairs with ff_merge;
// one conversion to FP64 per block.
template <int K>
__device__ __forceinline__ bool grid_sum(const KWork& w, float2 (&v)[K], double (&tot)[K]) {
  __shared__ float2 sm2[K][kKB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float2 t;
      t.x = __shfl_down_sync(0xffffffffu, v[k].x, o);
      t.y = __shfl_down_sync(0xffffffffu, v[k].y, o);
      v[k] = ff_merge(v[k], t);
    }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sm2[k][warp] = v[k];
  __syncthreads();
  double d[K];
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      v[k] = lane < (int)(blockDim.x >> 5) ? sm2[k][lane] : make_float2(0.f, 0.f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        float2 t;
        t.x = __shfl_down_sync(0xffffffffu, v[k].x, o);
        t.y = __shfl_down_sync(0xffffffffu, v[k].y, o);
        v[k] = ff_merge(v[k], t);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) d[k] = threadIdx.x == 0 ? (double)v[k].x + (double)v[k].y : 0.0;
  // the block result is in thread 0: store it and finish as in the FP64 path
  __shared__ int amlast;
  __shared__ double res[K];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) w.part[blockIdx.x * kMaxParts + k] = d[k];
    __threadfence();
    amlast = atomicAdd(w.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  double a[K];
#pragma unroll
  for (int k = 0; k < K; ++k) a[k] = 0.0;
#pragma unroll 4
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] += __ldcg(w.part + b * kMaxParts + k);
  block_sum<K>(a);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) res[k] = a[k];
    *w.ticket = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = res[k];
  return true;
}

template <int NC>
__device__ __forceinline__ unsigned active_mask(const KWork& w) {
  unsigned m = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (!w.st[c].done) m |= 1u << c;
  return m;
}

// One row of y = A x.  A uniform width-4 layout (Kuhn tetrahedra) reads the
// row's columns and values with one 16-byte load each; otherwise MAXW > 0
// unrolls the row to MAXW slots with predication (all loads issued before the
// gathers) and MAXW = 0 is a plain loop.
template <typename T> struct Vec4Load;
template <> struct Vec4Load<float> {
  static __device__ __forceinline__ void get(const float* v, int i, float (&a)[4]) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(v) + i);
    a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
  }
};
template <> struct Vec4Load<double> {
  static __device__ __forceinline__ void get(const double* v, int i, double (&a)[4]) {
    const double2 x = __ldg(reinterpret_cast<const double2*>(v) + 2 * i);
    const double2 y = __ldg(reinterpret_cast<const double2*>(v) + 2 * i + 1);
    a[0] = x.x; a[1] = x.y; a[2] = y.x; a[3] = y.y;
  }
};

template <typename T, int NC, int MAXW>
__device__ __forceinline__ void spmv_row(const Topo& t, const Mat<T>& A, int i, const T* x,
                                         T (&y)[NC], unsigned act) {
  const int nc = t.nc;
  const T d = __ldg(A.D + i);
#pragma unroll
  for (int c = 0; c < NC; ++c) y[c] = (act >> c & 1) ? d * __ldg(x + c * nc + i) : T(0);
  if (MAXW == 4 && A.E.W == 4) {
    const int4 j4 = ell_cols4(A.E, i);
    T a[4];
    Vec4Load<T>::get(A.val, i, a);
    const int j[4] = {j4.x, j4.y, j4.z, j4.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (act >> c & 1) y[c] += a[k] * __ldg(x + c * nc + j[k]);
    return;
  }
  int base, step, w;
  ell_row(A.E, i, base, step, w);
  const int* col = A.E.col + base;
  const T* val = A.val + base;
  if (MAXW > 0) {
    int j[MAXW > 0 ? MAXW : 1];
    T a[MAXW > 0 ? MAXW : 1];
#pragma unroll
    for (int k = 0; k < MAXW; ++k) {
      j[k] = k < w ? __ldg(col + step * k) : i;
      a[k] = k < w ? __ldg(val + step * k) : T(0);
    }
#pragma unroll
    for (int k = 0; k < MAXW; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (act >> c & 1) y[c] += a[k] * __ldg(x + c * nc + j[k]);
  } else {
    for (int k = 0; k < w; ++k) {
      const int jj = __ldg(col + step * k);
      const T aa = __ldg(val + step * k);
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (act >> c & 1) y[c] += aa * __ldg(x + c * nc + jj);
    }
  }
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }


// q = A p; alpha = rz / (p.q).  kRows rows per thread per pass (independent
// load chains); trailing row indices are clamped so all loads are unconditional.
constexpr int kRows = 4;
template <typename T, int NC, int MAXW>
__global__ void __launch_bounds__(kKB) k_pcg_spmv(Topo t, Mat<T> A, const T* p, T* q, KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  const int nc = t.nc;
  const int stride = gridDim.x * blockDim.x;
  DotAcc<T> pq[NC];
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < nc; i0 += kRows * stride) {
    T y[kRows][NC];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int i = i0 + r * stride;
      spmv_row<T, NC, MAXW>(t, A, i < nc ? i : i0, p, y[r], act);
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int i = i0 + r * stride;
      if (i < nc) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (act >> c & 1) {
            q[c * nc + i] = y[r][c];
            pq[c].add(p[c * nc + i], y[r][c]);
          }
      }
    }
  }
  typename DotAcc<T>::part_t v[NC];
  double tot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) v[c] = pq[c].part();
  if (!grid_sum<NC>(w, v, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (act >> c & 1) w.st[c].alpha = w.st[c].rz / tot[c];
}

// ---------------------------------------------------- segmented (batched)
// The same PCG / BiCGStab on a disjoint union of cases: every case keeps its
// own scalars (alpha, beta, rho, omega, ...), convergence flag and iteration
// count, as if it were solved alone.  Each solver block works inside one case
// (a chunk of kSegRows of its rows); each case has its own ticket, and the
// last of the case's blocks to arrive reduces that case's partials in block
// order.  A case's block partition depends only on its own size, so a case
// gives bitwise the same result alone as inside any batch (Jacobi or no
// preconditioning; the multigrid form in amg.cu shares its hierarchy across
// the cases and is equal to the case alone only up to rounding).
struct SWork {
  KState* st;          // [ncases * NC]
  double* part;        // [nblk * kMaxParts]
  unsigned* ticket;    // [ncases]
  const int* bcase;    // [nblk]
  const int* cb0;      // [ncases + 1]
  const int* cs;       // [ncases + 1]
  int maxit;
  double tol_rel, tol_abs;
};

struct SegBlock {
  int k, r0, r1;
};
__device__ __forceinline__ SegBlock seg_block(const SWork& w) {
  SegBlock b;
  b.k = __ldg(w.bcase + blockIdx.x);
  b.r0 = __ldg(w.cs + b.k) + (blockIdx.x - __ldg(w.cb0 + b.k)) * kSegRows;
  b.r1 = min(__ldg(w.cs + b.k + 1), b.r0 + kSegRows);
  return b;
}

template <int NC>
__device__ __forceinline__ unsigned seg_active(const SWork& w, int k) {
  unsigned m = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (!w.st[k * NC + c].done) m |= 1u << c;
  return m;
}

// Store this block's partials; true in the last block of case k, with the
// case totals in `tot` (all threads of that block).
template <int K>
__device__ __forceinline__ bool seg_sum(const SWork& w, int k, double (&v)[K], double (&tot)[K]) {
  block_sum<K>(v);
  __shared__ int amlast;
  __shared__ double res[K];
  const int b0 = __ldg(w.cb0 + k), nb = __ldg(w.cb0 + k + 1) - b0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) w.part[blockIdx.x * kMaxParts + q] = v[q];
    __threadfence();
    amlast = atomicAdd(w.ticket + k, 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  double a[K];
#pragma unroll
  for (int q = 0; q < K; ++q) a[q] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < K; ++q) a[q] += __ldcg(w.part + (b0 + b) * kMaxParts + q);
  block_sum<K>(a);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) res[q] = a[q];
    w.ticket[k] = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) tot[q] = res[q];
  return true;
}

}  // namespace difvm
