// Krylov solvers on the matrix-free LDU operator (Sec. 2.4.2 / 2.6.1): Jacobi-
// preconditioned CG for the SPD pressure system and right-Jacobi BiCGStab for
// the momentum system, for 1..3 right-hand sides at once (the matrix is read
// once per sweep for all components).
//
// All scalars live on the device.  Each kernel ends with a deterministic
// two-level reduction: block partials (warp shuffles, fixed tree) written to a
// partial buffer, then the last block to arrive (atomic ticket) sums the
// partials in block order and computes the solver scalars (alpha, beta, ...)
// and the convergence flags.  Components that have converged are skipped.
// Inner products are accumulated in FP64: directly in the F64 path, and in the
// F32 path by the compensated Dot2 scheme (Ogita, Rump & Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 2005) on FP32 pairs per thread,
// converted to FP64 for the cross-thread reduction, which keeps the B300's
// low-rate FP64 pipe off the per-element path.
//
// The host loop checks the convergence flags every `check_every` iterations;
// iterations launched after convergence exit immediately, so results do not
// depend on the check interval.
#include <math.h>

#include <algorithm>

#include "difvm_internal.cuh"

namespace difvm {

template <typename T>
difvm_status ldu_apply_t(difvm_mesh_t m, const void* D, const void* L, const void* U,
                         const void* x, int ncomp, int transpose, void* y, cudaStream_t s);

constexpr int kKB = 256;       // threads per block
constexpr int kMaxParts = 12;  // partial sums per block (<= 4 per component x 3)

struct KState {
  double rr, rz, bb, tol2, alpha, beta, rho, omega, pq, res0;
  int iters, done, status, sconv;
  int zero_rhs, pad0, pad1, pad2;
};

struct KWork {
  KState* st;        // [ncomp]
  double* part;      // [grid * kMaxParts]
  unsigned* ticket;  // 1
  int maxit;
  double tol_rel, tol_abs;
};

template <typename T> struct Mat {
  const T* D;
  const T* L;  // coefficient of x_O in row N
  const T* U;  // coefficient of x_N in row O
};

// ---------------------------------------------------------- accumulators
template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double get() const { return s; }
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
};

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

template <typename T, int NC>
__device__ __forceinline__ void spmv_row(const Topo& t, const Mat<T>& A, int i, const T* x,
                                         T (&y)[NC], unsigned act) {
  const int nc = t.nc;
  const T d = __ldg(A.D + i);
#pragma unroll
  for (int c = 0; c < NC; ++c) y[c] = (act >> c & 1) ? d * __ldg(x + c * nc + i) : T(0);
  const int e1 = __ldg(t.cptr + i + 1);
  for (int e = __ldg(t.cptr + i); e < e1; ++e) {
    const int ent = __ldg(t.cent + e);
    const int f = ent >> 1;
    if (f >= t.ni) break;
    const int2 on = __ldg(t.on + f);
    const bool nside = ent & 1;
    const int j = nside ? on.x : on.y;
    const T a = nside ? __ldg(A.L + f) : __ldg(A.U + f);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) y[c] += a * __ldg(x + c * nc + j);
  }
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// ================================================================== PCG
// init: rD = 1/D, r = b - A x, p = z = rD r;  sums bb, rr, rz
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_pcg_init(Topo t, Mat<T> A, int jacobi, const T* b, T* x,
                                                  T* r, T* p, T* rD, KWork w) {
  const int nc = t.nc;
  DotAcc<T> bb[NC], rr[NC], rz[NC];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const T di = __ldg(A.D + i);
    const T rd = jacobi ? T(1) / di : T(1);
    rD[i] = rd;
    T ax[NC];
    spmv_row<T, NC>(t, A, i, x, ax, (1u << NC) - 1);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T bi = b[c * nc + i];
      const T ri = bi - ax[c];
      const T zi = ri * rd;
      r[c * nc + i] = ri;
      p[c * nc + i] = zi;
      bb[c].add(bi, bi);
      rr[c].add(ri, ri);
      rz[c].add(ri, zi);
    }
  }
  double v[3 * NC], tot[3 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    v[3 * c] = bb[c].get();
    v[3 * c + 1] = rr[c].get();
    v[3 * c + 2] = rz[c].get();
  }
  if (!grid_sum<3 * NC>(w, v, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    KState& s = w.st[c];
    s.bb = tot[3 * c];
    s.rr = tot[3 * c + 1];
    s.rz = tot[3 * c + 2];
    s.res0 = sqrt(s.rr);
    s.tol2 = fmax(w.tol_rel * w.tol_rel * s.bb, w.tol_abs * w.tol_abs);
    s.iters = 0;
    s.status = DIFVM_OK;
    s.zero_rhs = s.bb == 0.0;
    s.done = s.zero_rhs || s.rr <= s.tol2;
    if (!finite_d(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; }
  }
}

// q = A p; alpha = rz / (p.q)
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_pcg_spmv(Topo t, Mat<T> A, const T* p, T* q, KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  const int nc = t.nc;
  DotAcc<T> pq[NC];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    T y[NC];
    spmv_row<T, NC>(t, A, i, p, y, act);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        q[c * nc + i] = y[c];
        pq[c].add(p[c * nc + i], y[c]);
      }
  }
  double v[NC], tot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) v[c] = pq[c].get();
  if (!grid_sum<NC>(w, v, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (act >> c & 1) w.st[c].alpha = w.st[c].rz / tot[c];
}

// x += alpha p; r -= alpha q; rr, rz (z = rD r); convergence test; beta
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_pcg_update(int nc, const T* p, const T* q, const T* rD,
                                                    T* x, T* r, KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  T al[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) al[c] = (T)w.st[c].alpha;
  DotAcc<T> rr[NC], rz[NC];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const T rd = rD[i];
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        const int k = c * nc + i;
        x[k] += al[c] * p[k];
        const T ri = r[k] - al[c] * q[k];
        r[k] = ri;
        rr[c].add(ri, ri);
        rz[c].add(ri, ri * rd);
      }
  }
  double v[2 * NC], tot[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    v[2 * c] = rr[c].get();
    v[2 * c + 1] = rz[c].get();
  }
  if (!grid_sum<2 * NC>(w, v, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (!(act >> c & 1)) continue;
    KState& s = w.st[c];
    s.iters += 1;
    s.rr = tot[2 * c];
    if (!finite_d(s.rr) || !finite_d(s.alpha)) { s.done = 1; s.status = DIFVM_ENONFINITE; continue; }
    if (s.rr <= s.tol2) { s.done = 1; continue; }
    if (s.iters >= w.maxit) { s.done = 1; s.status = DIFVM_ENOTCONV; continue; }
    s.beta = tot[2 * c + 1] / s.rz;
    s.rz = tot[2 * c + 1];
  }
}

// p = rD r + beta p   (components whose flag was raised this iteration are skipped)
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_pcg_pupdate(int nc, const T* r, const T* rD, T* p, KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  T be[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) be[c] = (T)w.st[c].beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const T rd = rD[i];
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        const int k = c * nc + i;
        p[k] = r[k] * rd + be[c] * p[k];
      }
  }
}

template <typename T, int NC>
__global__ void k_zero_rhs(int nc, T* x, KWork w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (w.st[c].zero_rhs) x[c * nc + i] = T(0);
}

// ============================================================= BiCGStab
// init: rD, r = rh = b - A x, p = v = 0; rho = alpha = omega = 1; bb, rr
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_bicg_init(Topo t, Mat<T> A, int jacobi, const T* b, T* x,
                                                   T* r, T* rh, T* p, T* v, T* rD, KWork w) {
  const int nc = t.nc;
  DotAcc<T> bb[NC], rr[NC];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const T di = __ldg(A.D + i);
    rD[i] = jacobi ? T(1) / di : T(1);
    T ax[NC];
    spmv_row<T, NC>(t, A, i, x, ax, (1u << NC) - 1);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int k = c * nc + i;
      const T bi = b[k];
      const T ri = bi - ax[c];
      r[k] = ri;
      rh[k] = ri;
      p[k] = T(0);
      v[k] = T(0);
      bb[c].add(bi, bi);
      rr[c].add(ri, ri);
    }
  }
  double vv[2 * NC], tot[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    vv[2 * c] = bb[c].get();
    vv[2 * c + 1] = rr[c].get();
  }
  if (!grid_sum<2 * NC>(w, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    KState& s = w.st[c];
    s.bb = tot[2 * c];
    s.rr = tot[2 * c + 1];
    s.rz = s.rr;  // rh . r with rh = r
    s.res0 = sqrt(s.rr);
    s.tol2 = fmax(w.tol_rel * w.tol_rel * s.bb, w.tol_abs * w.tol_abs);
    s.iters = 0;
    s.status = DIFVM_OK;
    s.rho = 1.0; s.alpha = 1.0; s.omega = 1.0;
    s.sconv = 0;
    s.zero_rhs = s.bb == 0.0;
    s.done = s.zero_rhs || s.rr <= s.tol2;
    if (!finite_d(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; }
  }
}

// rho1 = rh.r (kept in s.rz); beta = (rho1/rho)(alpha/omega); p = r + beta (p - omega v)
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_bicg_p(int nc, const T* r, const T* v, T* p, KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  T be[NC], om[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const KState& s = w.st[c];
    be[c] = (T)((s.rz / s.rho) * (s.alpha / s.omega));
    om[c] = (T)s.omega;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        const int k = c * nc + i;
        p[k] = r[k] + be[c] * (p[k] - om[c] * v[k]);
      }
}

// v = A (rD p); alpha = rho1 / (rh . v)
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_bicg_spmv1(Topo t, Mat<T> A, const T* rh, const T* y,
                                                    T* v, KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  const int nc = t.nc;
  DotAcc<T> rv[NC];
  // y = rD p is complete before the gather (written by k_bicg_scale)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    T a[NC];
    spmv_row<T, NC>(t, A, i, y, a, act);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        v[c * nc + i] = a[c];
        rv[c].add(rh[c * nc + i], a[c]);
      }
  }
  double vv[NC], tot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) vv[c] = rv[c].get();
  if (!grid_sum<NC>(w, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (!(act >> c & 1)) continue;
    KState& s = w.st[c];
    s.rho = s.rz;
    if (s.rho == 0.0 || tot[c] == 0.0 || s.omega == 0.0) { s.done = 1; s.status = DIFVM_EBREAKDOWN; continue; }
    s.alpha = s.rho / tot[c];
  }
}

// y = rD a  (a = p or s)
template <typename T, int NC>
__global__ void k_bicg_scale(int nc, const T* a, const T* rD, T* y, KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const T rd = rD[i];
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) y[c * nc + i] = a[c * nc + i] * rd;
  }
}

// s = r - alpha v; test ||s||; if converged x += alpha y
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_bicg_s(int nc, const T* r, const T* v, T* s_, KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  T al[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) al[c] = (T)w.st[c].alpha;
  DotAcc<T> ss[NC];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        const int k = c * nc + i;
        const T si = r[k] - al[c] * v[k];
        s_[k] = si;
        ss[c].add(si, si);
      }
  double vv[NC], tot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) vv[c] = ss[c].get();
  if (!grid_sum<NC>(w, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (!(act >> c & 1)) continue;
    KState& s = w.st[c];
    s.iters += 1;
    s.pq = tot[c];
    s.sconv = tot[c] <= s.tol2;
    if (s.sconv) s.rr = tot[c];
  }
}

// components with sconv: x += alpha y and finish
template <typename T, int NC>
__global__ void k_bicg_sfinish(int nc, const T* y, T* x, KWork w) {
  unsigned fin = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (!w.st[c].done && w.st[c].sconv) fin |= 1u << c;
  if (!fin) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (fin >> c & 1) x[c * nc + i] += (T)w.st[c].alpha * y[c * nc + i];
}

// t = A (rD s); omega = (t.s)/(t.t)
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_bicg_spmv2(Topo t, Mat<T> A, const T* z, const T* s_,
                                                    T* tv, KWork w) {
  unsigned act = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (!w.st[c].done && !w.st[c].sconv) act |= 1u << c;
  if (!act) return;
  const int nc = t.nc;
  DotAcc<T> ts[NC], tt[NC];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    T a[NC];
    spmv_row<T, NC>(t, A, i, z, a, act);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        tv[c * nc + i] = a[c];
        ts[c].add(a[c], s_[c * nc + i]);
        tt[c].add(a[c], a[c]);
      }
  }
  double vv[2 * NC], tot[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    vv[2 * c] = ts[c].get();
    vv[2 * c + 1] = tt[c].get();
  }
  if (!grid_sum<2 * NC>(w, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (act >> c & 1) w.st[c].omega = tot[2 * c + 1] > 0.0 ? tot[2 * c] / tot[2 * c + 1] : 0.0;
}

// x += alpha y + omega z; r = s - omega t; rr, rh.r; convergence
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_bicg_update(int nc, const T* y, const T* z, const T* s_,
                                                     const T* tv, const T* rh, T* x, T* r, KWork w) {
  unsigned act = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (!w.st[c].done && !w.st[c].sconv) act |= 1u << c;
  // components that converged on s are closed here (their x was updated)
  if (!act) {
    if (blockIdx.x == 0 && threadIdx.x == 0)
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (!w.st[c].done && w.st[c].sconv) w.st[c].done = 1;
    return;
  }
  T al[NC], om[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    al[c] = (T)w.st[c].alpha;
    om[c] = (T)w.st[c].omega;
  }
  DotAcc<T> rr[NC], rhr[NC];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        const int k = c * nc + i;
        x[k] += al[c] * y[k] + om[c] * z[k];
        const T ri = s_[k] - om[c] * tv[k];
        r[k] = ri;
        rr[c].add(ri, ri);
        rhr[c].add(rh[k], ri);
      }
  double vv[2 * NC], tot[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    vv[2 * c] = rr[c].get();
    vv[2 * c + 1] = rhr[c].get();
  }
  if (!grid_sum<2 * NC>(w, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    KState& s = w.st[c];
    if (!s.done && s.sconv) { s.done = 1; continue; }
    if (!(act >> c & 1)) continue;
    s.rr = tot[2 * c];
    s.rz = tot[2 * c + 1];
    if (!finite_d(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; continue; }
    if (s.rr <= s.tol2) { s.done = 1; continue; }
    if (s.iters >= w.maxit) { s.done = 1; s.status = DIFVM_ENOTCONV; continue; }
  }
}

// ------------------------------------------------------------- info output
__global__ void k_write_info(int ncomp, const KState* st, difvm_solve_info* info, int refinements) {
  int c = threadIdx.x;
  if (c >= ncomp) return;
  const KState& s = st[c];
  difvm_solve_info o;
  o.iters = s.iters;
  o.refinements = refinements;
  o.status = s.status;
  o.pad = 0;
  o.res0 = s.res0;
  o.res = sqrt(s.rr);
  o.bnorm = sqrt(s.bb);
  info[c] = o;
}

// ------------------------------------------------------------- workspace
struct WsLayout {
  size_t vec_bytes, n_vec, state_off, part_off, ticket_off, total;
};

static int grid_for(const difvm_mesh* m) {
  int need = (int)blocks_for(m->nc, kKB);
  return std::max(1, std::min(need, m->num_sms * 8));
}

static WsLayout layout(const difvm_mesh* m, size_t elt, int method, int ncomp) {
  WsLayout L;
  L.vec_bytes = ((size_t)m->nc * elt + 255) / 256 * 256;
  // PCG: r p q (per comp) + rD;  BiCGStab: r rh p v s t y z (per comp) + rD
  L.n_vec = (method == DIFVM_PCG ? 3 : 8) * (size_t)ncomp + 1;
  L.state_off = L.n_vec * L.vec_bytes;
  L.part_off = L.state_off + 256 * 4;
  L.ticket_off = L.part_off + (size_t)grid_for(m) * kMaxParts * sizeof(double);
  L.total = L.ticket_off + 256;
  return L;
}

}  // namespace difvm

using namespace difvm;

extern "C" size_t difvm_krylov_workspace_bytes(difvm_mesh_t m, difvm_prec prec, int method, int ncomp) {
  if (!m || ncomp < 1 || ncomp > 3) return 0;
  return layout(m, prec == DIFVM_F64 ? 8 : 4, method, ncomp).total;
}

namespace difvm {

template <typename T, int NC>
static difvm_status solve_nc(difvm_mesh_t m, const difvm_solve_opts* o, Mat<T> A, const T* b, T* x,
                             char* ws, const WsLayout& L, difvm_solve_info* info, int refinements,
                             cudaStream_t st, KState* host_state) {
  const int nc = m->nc;
  const int G = grid_for(m);
  Topo t = m->topo();
  auto vec = [&](int k) { return (T*)(ws + (size_t)k * L.vec_bytes); };
  KWork w;
  w.st = (KState*)(ws + L.state_off);
  w.part = (double*)(ws + L.part_off);
  w.ticket = (unsigned*)(ws + L.ticket_off);
  w.maxit = o->max_iter > 0 ? o->max_iter : 1000;
  w.tol_rel = o->tol_rel;
  w.tol_abs = o->tol_abs;
  const int jac = o->precond != DIFVM_PRECOND_NONE;
  const int chunk = o->check_every > 0 ? o->check_every : 8;
  DIFVM_CUDA(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), st));
  T* rD = vec(L.n_vec - 1);
  auto all_done = [&](bool& done) -> difvm_status {
    DIFVM_CUDA(cudaMemcpyAsync(host_state, w.st, sizeof(KState) * NC, cudaMemcpyDeviceToHost, st));
    DIFVM_CUDA(cudaStreamSynchronize(st));
    done = true;
    for (int c = 0; c < NC; ++c) done &= host_state[c].done != 0;
    return DIFVM_OK;
  };
  if (o->method == DIFVM_PCG) {
    T *r = vec(0), *p = vec(NC), *q = vec(2 * NC);
    k_pcg_init<T, NC><<<G, kKB, 0, st>>>(t, A, jac, b, x, r, p, rD, w);
    DIFVM_TRY(check_launch("pcg_init"));
    k_zero_rhs<T, NC><<<G, kKB, 0, st>>>(nc, x, w);
    DIFVM_TRY(check_launch("zero_rhs"));
    int it = 0;
    bool done = false;
    while (it < w.maxit) {
      int n = std::min(chunk, w.maxit - it);
      for (int k = 0; k < n; ++k) {
        prof_before(DIFVM_PROF_PCG_SPMV, st);
        k_pcg_spmv<T, NC><<<G, kKB, 0, st>>>(t, A, p, q, w);
        prof_after(DIFVM_PROF_PCG_SPMV, st);
        prof_before(DIFVM_PROF_PCG_UPDATE, st);
        k_pcg_update<T, NC><<<G, kKB, 0, st>>>(nc, p, q, rD, x, r, w);
        prof_after(DIFVM_PROF_PCG_UPDATE, st);
        prof_before(DIFVM_PROF_PCG_PUPDATE, st);
        k_pcg_pupdate<T, NC><<<G, kKB, 0, st>>>(nc, r, rD, p, w);
        prof_after(DIFVM_PROF_PCG_PUPDATE, st);
        count_launch(); count_launch();
        DIFVM_TRY(check_launch("pcg_iter"));
      }
      it += n;
      DIFVM_TRY(all_done(done));
      if (done) break;
    }
  } else if (o->method == DIFVM_BICGSTAB) {
    T *r = vec(0), *rh = vec(NC), *p = vec(2 * NC), *v = vec(3 * NC), *s_ = vec(4 * NC),
      *tv = vec(5 * NC), *y = vec(6 * NC), *z = vec(7 * NC);
    k_bicg_init<T, NC><<<G, kKB, 0, st>>>(t, A, jac, b, x, r, rh, p, v, rD, w);
    DIFVM_TRY(check_launch("bicg_init"));
    k_zero_rhs<T, NC><<<G, kKB, 0, st>>>(nc, x, w);
    DIFVM_TRY(check_launch("zero_rhs"));
    int it = 0;
    bool done = false;
    while (it < w.maxit) {
      int n = std::min(chunk, w.maxit - it);
      for (int k = 0; k < n; ++k) {
        k_bicg_p<T, NC><<<G, kKB, 0, st>>>(nc, r, v, p, w);
        k_bicg_scale<T, NC><<<G, kKB, 0, st>>>(nc, p, rD, y, w);
        k_bicg_spmv1<T, NC><<<G, kKB, 0, st>>>(t, A, rh, y, v, w);
        k_bicg_s<T, NC><<<G, kKB, 0, st>>>(nc, r, v, s_, w);
        k_bicg_sfinish<T, NC><<<G, kKB, 0, st>>>(nc, y, x, w);
        k_bicg_scale<T, NC><<<G, kKB, 0, st>>>(nc, s_, rD, z, w);
        k_bicg_spmv2<T, NC><<<G, kKB, 0, st>>>(t, A, z, s_, tv, w);
        k_bicg_update<T, NC><<<G, kKB, 0, st>>>(nc, y, z, s_, tv, rh, x, r, w);
        for (int q = 0; q < 7; ++q) count_launch();
        DIFVM_TRY(check_launch("bicg_iter"));
      }
      it += n;
      DIFVM_TRY(all_done(done));
      if (done) break;
    }
  } else {
    return set_error(DIFVM_EINVAL, "unknown Krylov method %d", o->method);
  }
  if (info) {
    k_write_info<<<1, 32, 0, st>>>(NC, w.st, info, refinements);
    DIFVM_TRY(check_launch("write_info"));
  }
  DIFVM_CUDA(cudaMemcpyAsync(host_state, w.st, sizeof(KState) * NC, cudaMemcpyDeviceToHost, st));
  DIFVM_CUDA(cudaStreamSynchronize(st));
  int worst = DIFVM_OK;
  for (int c = 0; c < NC; ++c) worst = std::max(worst, host_state[c].status);
  return (difvm_status)worst;
}

}  // namespace difvm

namespace difvm {

// ------------------------------------------------- mixed-precision refinement
// r64 = b64 - A x64 in FP64 (FP32 coefficients are exact in FP64), r32 = r64,
// e32 = 0; convergence of the outer iteration on ||r64||.
template <int NC>
__global__ void __launch_bounds__(kKB) k_refine_residual(Topo t, Mat<float> A, const double* b,
                                                         const double* x, float* r32, float* e32,
                                                         KWork w, int first) {
  const int nc = t.nc;
  double bb[NC], rr[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) bb[c] = rr[c] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    double y[NC];
    const double d = (double)__ldg(A.D + i);
#pragma unroll
    for (int c = 0; c < NC; ++c) y[c] = d * x[c * nc + i];
    const int e1 = __ldg(t.cptr + i + 1);
    for (int e = __ldg(t.cptr + i); e < e1; ++e) {
      const int ent = __ldg(t.cent + e);
      const int f = ent >> 1;
      if (f >= t.ni) break;
      const int2 on = __ldg(t.on + f);
      const bool nside = ent & 1;
      const int j = nside ? on.x : on.y;
      const double a = (double)(nside ? __ldg(A.L + f) : __ldg(A.U + f));
#pragma unroll
      for (int c = 0; c < NC; ++c) y[c] = fma(a, x[c * nc + j], y[c]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double bi = b[c * nc + i];
      const double ri = bi - y[c];
      r32[c * nc + i] = (float)ri;
      e32[c * nc + i] = 0.f;
      rr[c] = fma(ri, ri, rr[c]);
      bb[c] = fma(bi, bi, bb[c]);
    }
  }
  double v[2 * NC], tot[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    v[2 * c] = bb[c];
    v[2 * c + 1] = rr[c];
  }
  if (!grid_sum<2 * NC>(w, v, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    KState& s = w.st[c];
    s.bb = tot[2 * c];
    s.rr = tot[2 * c + 1];
    if (first) {
      s.res0 = sqrt(s.rr);
      s.iters = 0;
      s.status = DIFVM_OK;
      s.rho = INFINITY;  // previous outer residual norm^2
    }
    s.tol2 = fmax(w.tol_rel * w.tol_rel * s.bb, w.tol_abs * w.tol_abs);
    s.zero_rhs = s.bb == 0.0;
    if (!finite_d(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; continue; }
    s.done = s.zero_rhs || s.rr <= s.tol2;
    // stagnation: the FP32 inner solve no longer reduces the FP64 residual
    if (!s.done && !first && s.rr > 0.25 * s.rho) { s.done = 1; s.status = DIFVM_ENOTCONV; }
    s.rho = s.rr;
  }
}

template <int NC>
__global__ void k_refine_add(int nc, const float* e32, double* x, const KWork w, const KState* inner) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (!w.st[c].done) x[c * nc + i] += (double)e32[c * nc + i];
  if (blockIdx.x == 0 && threadIdx.x < NC) {
    const int c = threadIdx.x;
    if (!w.st[c].done) w.st[c].iters += inner[c].iters;
  }
}

template <int NC>
__global__ void k_zero_x64(int nc, double* x, KWork w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (w.st[c].zero_rhs) x[c * nc + i] = 0.0;
}

template <int NC>
static difvm_status refine_nc(difvm_mesh_t m, const difvm_solve_opts* o, Mat<float> A,
                              const double* b64, double* x64, char* ws, size_t wsbytes,
                              difvm_solve_info* info, cudaStream_t st) {
  const int nc = m->nc;
  const int G = grid_for(m);
  WsLayout L = layout(m, 4, o->method, NC);
  size_t vb = L.vec_bytes;
  // [inner workspace | r32 (NC vecs) | e32 (NC vecs) | outer state | outer partials | ticket]
  size_t r_off = (L.total + 255) / 256 * 256;
  size_t e_off = r_off + NC * vb;
  size_t so = e_off + NC * vb;
  size_t po = so + 256 * 4;
  size_t to = po + (size_t)G * kMaxParts * sizeof(double);
  if (wsbytes < to + 256) return set_error(DIFVM_EINVAL, "workspace too small for refinement");
  float* r32 = (float*)(ws + r_off);
  float* e32 = (float*)(ws + e_off);
  KWork w;
  w.st = (KState*)(ws + so);
  w.part = (double*)(ws + po);
  w.ticket = (unsigned*)(ws + to);
  w.maxit = o->max_iter;
  w.tol_rel = o->tol_rel;
  w.tol_abs = o->tol_abs;
  DIFVM_CUDA(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), st));
  difvm_solve_opts in = *o;
  in.tol_rel = o->inner_tol > 0 ? o->inner_tol : 1e-4;
  in.tol_abs = 0.0;
  in.refine_max = 0;
  KState hs[3], his[3];
  const int rmax = o->refine_max > 0 ? o->refine_max : 20;
  int sweeps = 0, total_inner = 0;
  Topo t = m->topo();
  for (int k = 0; k <= rmax; ++k) {
    k_refine_residual<NC><<<G, kKB, 0, st>>>(t, A, b64, x64, r32, e32, w, k == 0);
    DIFVM_TRY(check_launch("refine_residual"));
    DIFVM_CUDA(cudaMemcpyAsync(hs, w.st, sizeof(KState) * NC, cudaMemcpyDeviceToHost, st));
    DIFVM_CUDA(cudaStreamSynchronize(st));
    bool done = true;
    for (int c = 0; c < NC; ++c) done &= hs[c].done != 0;
    if (done || k == rmax) break;
    in.max_iter = std::max(1, o->max_iter - total_inner);
    difvm_status s = solve_nc<float, NC>(m, &in, A, r32, e32, ws, L, nullptr, 0, st, his);
    (void)s;  // the inner solve may stop at its own cap; the outer residual decides
    int it = 0;
    for (int c = 0; c < NC; ++c) it = std::max(it, his[c].iters);
    total_inner += it;
    k_refine_add<NC><<<G, kKB, 0, st>>>(nc, e32, x64, w, (const KState*)(ws + L.state_off));
    DIFVM_TRY(check_launch("refine_add"));
    ++sweeps;
    if (total_inner >= o->max_iter) {
      k_refine_residual<NC><<<G, kKB, 0, st>>>(t, A, b64, x64, r32, e32, w, 0);
      DIFVM_TRY(check_launch("refine_residual"));
      break;
    }
  }
  k_zero_x64<NC><<<G, kKB, 0, st>>>(nc, x64, w);
  DIFVM_TRY(check_launch("zero_x64"));
  if (info) {
    k_write_info<<<1, 32, 0, st>>>(NC, w.st, info, sweeps);
    DIFVM_TRY(check_launch("write_info"));
  }
  DIFVM_CUDA(cudaMemcpyAsync(hs, w.st, sizeof(KState) * NC, cudaMemcpyDeviceToHost, st));
  DIFVM_CUDA(cudaStreamSynchronize(st));
  int worst = DIFVM_OK;
  for (int c = 0; c < NC; ++c) {
    int sc = hs[c].status;
    if (sc == DIFVM_OK && !(hs[c].rr <= hs[c].tol2) && !hs[c].zero_rhs) sc = DIFVM_ENOTCONV;
    worst = std::max(worst, sc);
  }
  return (difvm_status)worst;
}

// coefficient adjoint of a solve: Dbar -= bbar_i x_i, Lbar -= bbar_N x_O, Ubar -= bbar_O x_N
template <typename T, int NC>
__global__ void k_solve_coeff_bwd(Topo t, const T* x, const T* bbar, T* Dbar, T* Lbar, T* Ubar,
                                  int sym) {
  const int nc = t.nc;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < t.ni) {
    const int2 on = __ldg(t.on + k);
    T lb = T(0), ub = T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      lb += bbar[c * nc + on.y] * x[c * nc + on.x];
      ub += bbar[c * nc + on.x] * x[c * nc + on.y];
    }
    if (sym) {
      if (Lbar) Lbar[k] -= lb + ub;
    } else {
      if (Lbar) Lbar[k] -= lb;
      if (Ubar) Ubar[k] -= ub;
    }
  }
  if (Dbar && k < nc) {
    T db = T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) db += bbar[c * nc + k] * x[c * nc + k];
    Dbar[k] -= db;
  }
}

template <typename T>
static difvm_status solve_t(difvm_mesh_t m, const difvm_solve_opts* o, const void* D, const void* L,
                            const void* U, const void* b, void* x, int ncomp, void* ws,
                            size_t wsbytes, difvm_solve_info* info, cudaStream_t st) {
  WsLayout Ly = layout(m, sizeof(T), o->method, ncomp);
  if (!ws || wsbytes < Ly.total)
    return set_error(DIFVM_EINVAL, "workspace of %zu bytes < %zu needed", wsbytes, Ly.total);
  Mat<T> A{(const T*)D, (const T*)L, U ? (const T*)U : (const T*)L};
  KState hs[3];
  switch (ncomp) {
    case 1: return solve_nc<T, 1>(m, o, A, (const T*)b, (T*)x, (char*)ws, Ly, info, 0, st, hs);
    case 2: return solve_nc<T, 2>(m, o, A, (const T*)b, (T*)x, (char*)ws, Ly, info, 0, st, hs);
    case 3: return solve_nc<T, 3>(m, o, A, (const T*)b, (T*)x, (char*)ws, Ly, info, 0, st, hs);
  }
  return set_error(DIFVM_EINVAL, "ncomp must be 1..3");
}

static difvm_status check_solve(difvm_mesh_t m, difvm_prec prec, const difvm_solve_opts* o, int ncomp,
                                const void* D, const void* L) {
  DIFVM_TRY(check_mesh(m));
  DIFVM_TRY(check_prec(prec));
  if (!o) return set_error(DIFVM_EINVAL, "null options");
  if (o->method != DIFVM_PCG && o->method != DIFVM_BICGSTAB)
    return set_error(DIFVM_EINVAL, "unknown Krylov method %d", o->method);
  if (ncomp < 1 || ncomp > 3) return set_error(DIFVM_EINVAL, "ncomp must be 1..3 (got %d)", ncomp);
  if (!D || (!L && m->ni > 0)) return set_error(DIFVM_EINVAL, "null matrix");
  if (o->max_iter < 0) return set_error(DIFVM_EINVAL, "negative max_iter");
  return DIFVM_OK;
}

}  // namespace difvm

extern "C" difvm_status difvm_krylov_solve(difvm_mesh_t m, difvm_prec prec, const difvm_solve_opts* o,
                                           const void* D, const void* L, const void* U, const void* b,
                                           void* x, int ncomp, void* ws, size_t wsbytes,
                                           difvm_solve_info* info, void* stream) {
  DIFVM_TRY(check_solve(m, prec, o, ncomp, D, L));
  if (!b || !x) return set_error(DIFVM_EINVAL, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  return prec == DIFVM_F64 ? solve_t<double>(m, o, D, L, U, b, x, ncomp, ws, wsbytes, info, st)
                           : solve_t<float>(m, o, D, L, U, b, x, ncomp, ws, wsbytes, info, st);
}

extern "C" size_t difvm_krylov_refine_workspace_bytes(difvm_mesh_t m, int method, int ncomp) {
  if (!m || ncomp < 1 || ncomp > 3) return 0;
  WsLayout L = layout(m, 4, method, ncomp);
  size_t r_off = (L.total + 255) / 256 * 256;
  return r_off + 2 * (size_t)ncomp * L.vec_bytes + 256 * 4 +
         (size_t)grid_for(m) * kMaxParts * sizeof(double) + 256;
}

extern "C" difvm_status difvm_krylov_solve_refine(difvm_mesh_t m, const difvm_solve_opts* o,
                                                  const float* D, const float* L, const float* U,
                                                  const double* b64, double* x64, int ncomp, void* ws,
                                                  size_t wsbytes, difvm_solve_info* info, void* stream) {
  DIFVM_TRY(check_solve(m, DIFVM_F32, o, ncomp, D, L));
  if (!b64 || !x64 || !ws) return set_error(DIFVM_EINVAL, "null vector or workspace");
  Mat<float> A{D, L, U ? U : L};
  cudaStream_t st = (cudaStream_t)stream;
  switch (ncomp) {
    case 1: return refine_nc<1>(m, o, A, b64, x64, (char*)ws, wsbytes, info, st);
    case 2: return refine_nc<2>(m, o, A, b64, x64, (char*)ws, wsbytes, info, st);
    default: return refine_nc<3>(m, o, A, b64, x64, (char*)ws, wsbytes, info, st);
  }
}

extern "C" difvm_status difvm_krylov_solve_bwd(difvm_mesh_t m, difvm_prec prec,
                                               const difvm_solve_opts* o, const void* D,
                                               const void* L, const void* U, const void* x,
                                               const void* xbar, int ncomp, void* bbar, void* Dbar,
                                               void* Lbar, void* Ubar, void* ws, size_t wsbytes,
                                               difvm_solve_info* info, void* stream) {
  DIFVM_TRY(check_solve(m, prec, o, ncomp, D, L));
  if (!x || !xbar || !bbar) return set_error(DIFVM_EINVAL, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  size_t elt = prec == DIFVM_F64 ? 8 : 4;
  DIFVM_CUDA(cudaMemsetAsync(bbar, 0, elt * (size_t)ncomp * m->nc, st));
  // A^T: swap lower and upper (symmetric matrices are their own transpose)
  const void* Lt = U ? U : L;
  const void* Ut = U ? L : nullptr;
  difvm_status s = prec == DIFVM_F64
                       ? solve_t<double>(m, o, D, Lt, Ut, xbar, bbar, ncomp, ws, wsbytes, info, st)
                       : solve_t<float>(m, o, D, Lt, Ut, xbar, bbar, ncomp, ws, wsbytes, info, st);
  if (s != DIFVM_OK && s != DIFVM_ENOTCONV) return s;
  if (Dbar || Lbar || Ubar) {
    int n = std::max(m->ni, m->nc);
    int sym = U == nullptr;
#define DIFVM_CB(T, NC)                                                                          \
  k_solve_coeff_bwd<T, NC><<<blocks_for(n, 256), 256, 0, st>>>(m->topo(), (const T*)x,            \
                                                               (const T*)bbar, (T*)Dbar, (T*)Lbar, \
                                                               (T*)Ubar, sym)
    if (prec == DIFVM_F64) {
      if (ncomp == 1) DIFVM_CB(double, 1); else if (ncomp == 2) DIFVM_CB(double, 2); else DIFVM_CB(double, 3);
    } else {
      if (ncomp == 1) DIFVM_CB(float, 1); else if (ncomp == 2) DIFVM_CB(float, 2); else DIFVM_CB(float, 3);
    }
#undef DIFVM_CB
    DIFVM_TRY(check_launch("solve_coeff_bwd"));
  }
  return s;
}
