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

#include "krylov_common.cuh"

namespace difvm {

template <typename T>
difvm_status ldu_apply_t(difvm_mesh_t m, const void* D, const void* L, const void* U,
                         const void* x, int ncomp, int transpose, void* y, cudaStream_t s);

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
    spmv_row<T, NC, 0>(t, A, i, x, ax, (1u << NC) - 1);
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
  typename DotAcc<T>::part_t v[3 * NC];
  double tot[3 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    v[3 * c] = bb[c].part();
    v[3 * c + 1] = rr[c].part();
    v[3 * c + 2] = rz[c].part();
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
  typename DotAcc<T>::part_t v[2 * NC];
  double tot[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    v[2 * c] = rr[c].part();
    v[2 * c + 1] = rz[c].part();
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
    spmv_row<T, NC, 0>(t, A, i, x, ax, (1u << NC) - 1);
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
  typename DotAcc<T>::part_t vv[2 * NC];
  double tot[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    vv[2 * c] = bb[c].part();
    vv[2 * c + 1] = rr[c].part();
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
    s.beta = (s.rz / s.rho) * (s.alpha / s.omega);   // the p-update's scalar (p = v = 0 here)
    s.sconv = 0;
    s.zero_rhs = s.bb == 0.0;
    s.done = s.zero_rhs || s.rr <= s.tol2;
    if (!finite_d(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; }
  }
}

// rho1 = rh.r (kept in s.rz); beta = (rho1/rho)(alpha/omega); p = r + beta (p - omega v);
// with rD (Jacobi) also y = rD p, the preconditioned direction, in the same pass
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_bicg_p(int nc, const T* r, const T* v, T* p, const T* rD, T* y,
                                                KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  T be[NC], om[NC];   // beta = (rho_new / rho)(alpha / omega), formed once by the last block before
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const KState& s = w.st[c];
    be[c] = (T)s.beta;
    om[c] = (T)s.omega;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const T rd = rD ? rD[i] : T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        const int k = c * nc + i;
        const T pk = r[k] + be[c] * (p[k] - om[c] * v[k]);
        p[k] = pk;
        if (rD) y[k] = pk * rd;
      }
  }
}

// v = A (rD p); alpha = rho1 / (rh . v)
template <typename T, int NC, int MAXW>
__global__ void __launch_bounds__(kKB) k_bicg_spmv1(Topo t, Mat<T> A, const T* rh, const T* y,
                                                    T* v, KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  const int nc = t.nc;
  DotAcc<T> rv[NC];
  // y = rD p is complete before the gather (written by k_bicg_scale)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    T a[NC];
    spmv_row<T, NC, MAXW>(t, A, i, y, a, act);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        v[c * nc + i] = a[c];
        rv[c].add(rh[c * nc + i], a[c]);
      }
  }
  typename DotAcc<T>::part_t vv[NC];
  double tot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) vv[c] = rv[c].part();
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

// s = r - alpha v; test ||s||; if converged x += alpha y.  With rD (Jacobi) also
// z = rD s, the preconditioned s, in the same pass
template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_bicg_s(int nc, const T* r, const T* v, T* s_, const T* rD, T* z,
                                                KWork w) {
  const unsigned act = active_mask<NC>(w);
  if (!act) return;
  T al[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) al[c] = (T)w.st[c].alpha;
  DotAcc<T> ss[NC];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const T rd = rD ? rD[i] : T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        const int k = c * nc + i;
        const T si = r[k] - al[c] * v[k];
        s_[k] = si;
        if (rD) z[k] = si * rd;
        ss[c].add(si, si);
      }
  }
  typename DotAcc<T>::part_t vv[NC];
  double tot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) vv[c] = ss[c].part();
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
template <typename T, int NC, int MAXW>
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
    spmv_row<T, NC, MAXW>(t, A, i, z, a, act);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        tv[c * nc + i] = a[c];
        ts[c].add(a[c], s_[c * nc + i]);
        tt[c].add(a[c], a[c]);
      }
  }
  typename DotAcc<T>::part_t vv[2 * NC];
  double tot[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    vv[2 * c] = ts[c].part();
    vv[2 * c + 1] = tt[c].part();
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
  typename DotAcc<T>::part_t vv[2 * NC];
  double tot[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    vv[2 * c] = rr[c].part();
    vv[2 * c + 1] = rhr[c].part();
  }
  if (!grid_sum<2 * NC>(w, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    KState& s = w.st[c];
    if (!s.done && s.sconv) { s.done = 1; continue; }
    if (!(act >> c & 1)) continue;
    s.rr = tot[2 * c];
    s.rz = tot[2 * c + 1];
    s.beta = (s.rz / s.rho) * (s.alpha / s.omega);
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
  size_t vec_bytes, n_vec, val_off, state_off, part_off, ticket_off, flag_off, total;
};

static int grid_for(const difvm_mesh* m) {
  int need = (int)blocks_for(m->nc, kKB);
  return std::max(1, std::min(need, m->num_sms * 4));
}

static size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// Grid of a grid-stride solver kernel: the blocks that are resident on the SMs
// at once (1-4 per SM, by the kernel's register use; 40 or more registers fit
// fewer than four 512-thread blocks), so that it runs in one wave and its
// reduction finishes once; never more than the rows need or than grid_for(m),
// for which the partials are sized.  The kernel is a template argument, so each
// kernel keeps its own count (kernels of one signature do not share it).
template <auto K>
static int wave_grid(const difvm_mesh* m) {
  static int per = 0;
  if (per == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, kKB, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      b = 4;
    }
    per = std::max(1, std::min(b, 4));
  }
  return std::max(1, std::min(grid_for(m), per * m->num_sms));
}

// [vectors | ELL values | solver states | block partials | ticket]
static WsLayout layout(const difvm_mesh* m, size_t elt, int method, int ncomp) {
  WsLayout L;
  L.vec_bytes = up256((size_t)m->nc * elt);
  // PCG: r p q (per comp) + rD;  BiCGStab: r rh p v s t y z (per comp) + rD
  L.n_vec = (method == DIFVM_PCG ? 3 : 8) * (size_t)ncomp + 1;
  L.val_off = L.n_vec * L.vec_bytes;
  L.state_off = L.val_off + up256((size_t)std::max<int64_t>(m->ell_nslots, 1) * elt);
  if (m->seg) {  // per-case states, partials and tickets of the segmented solvers
    L.part_off = L.state_off + up256((size_t)m->ncases * ncomp * sizeof(KState));
    L.ticket_off = L.part_off + up256((size_t)m->seg_nblk * kMaxParts * sizeof(double));
    L.flag_off = L.ticket_off + up256((size_t)m->ncases * sizeof(unsigned));
    L.total = L.flag_off + 256;
    return L;
  }
  L.part_off = L.state_off + 256 * 4;
  L.ticket_off = L.part_off + up256((size_t)grid_for(m) * kMaxParts * sizeof(double));
  L.flag_off = L.ticket_off;
  L.total = L.ticket_off + 256;
  return L;
}

template <typename T>
static difvm_status fill_ell(difvm_mesh_t m, const T* L, const T* U, T* val, cudaStream_t st) {
  if (m->ell_nslots == 0) return DIFVM_OK;
  k_ell_fill<T><<<blocks_for(m->ell_nslots, 256), 256, 0, st>>>((int)m->ell_nslots, m->ell_map, L,
                                                                 U ? U : L, val);
  return check_launch("ell_fill");
}

}  // namespace difvm

using namespace difvm;

extern "C" size_t difvm_krylov_workspace_bytes(difvm_mesh_t m, difvm_prec prec, int method, int ncomp) {
  if (!m || ncomp < 1 || ncomp > 3) return 0;
  return layout(m, prec == DIFVM_F64 ? 8 : 4, method, ncomp).total;
}

namespace difvm {

static KWork make_work(char* ws, const WsLayout& L, const difvm_solve_opts* o) {
  KWork w;
  w.st = (KState*)(ws + L.state_off);
  w.part = (double*)(ws + L.part_off);
  w.ticket = (unsigned*)(ws + L.ticket_off);
  w.maxit = o->max_iter > 0 ? o->max_iter : 1000;
  w.tol_rel = o->tol_rel;
  w.tol_abs = o->tol_abs;
  return w;
}

template <int NC>
static difvm_status read_states(KState* host, const KWork& w, cudaStream_t st, bool& all_done) {
  DIFVM_CUDA(cudaMemcpyAsync(host, w.st, sizeof(KState) * NC, cudaMemcpyDeviceToHost, st));
  DIFVM_CUDA(cudaStreamSynchronize(st));
  all_done = true;
  for (int c = 0; c < NC; ++c) all_done &= host[c].done != 0;
  return DIFVM_OK;
}

// Lraw, Uraw, extra: the LDU face coefficients and the DILU workspace, used with
// DIFVM_PRECOND_DIC (BiCGStab preconditioned by DILU in the internal order)
template <typename T, int NC, int MW>
static difvm_status solve_nc(difvm_mesh_t m, const difvm_solve_opts* o, Mat<T> A, const T* b, T* x,
                             char* ws, const WsLayout& L, difvm_solve_info* info, cudaStream_t st,
                             KState* host_state, const T* Lraw = nullptr, const T* Uraw = nullptr,
                             char* extra = nullptr) {
  const int nc = m->nc;
  const int G = grid_for(m);
  Topo t = m->topo();
  auto vec = [&](int k) { return (T*)(ws + (size_t)k * L.vec_bytes); };
  KWork w = make_work(ws, L, o);
  const int jac = o->precond != DIFVM_PRECOND_NONE;
  const int chunk = o->check_every > 0 ? o->check_every : 8;
  DIFVM_CUDA(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), st));
  T* rD = vec(L.n_vec - 1);
  bool done = false;
  const bool graph = stream_capturing(st);
  int* counter = reinterpret_cast<int*>(w.ticket) + 1;   // loop counter under a graph
  // the iterations: on the host loop, or as the body of a device WHILE node
  auto run = [&](auto&& iter) -> difvm_status {
    if (graph) {
      DIFVM_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
      WhileLoop Lw;
      DIFVM_TRY(while_open(st, Lw));
      for (int k = 0; k < kGraphUnroll; ++k) iter(Lw.side);
      k_loop_cond<<<1, 32, 0, Lw.side>>>(done_flags(w.st), kStateInts, NC, counter,
                                         w.maxit / kGraphUnroll + 2, Lw.h);
      difvm_status e = check_launch("loop_cond");
      DIFVM_TRY(while_close(Lw));
      return e;
    }
    for (int it = 0; it < w.maxit;) {
      const int n = std::min(chunk, w.maxit - it);
      for (int k = 0; k < n; ++k) iter(st);
      DIFVM_TRY(check_error("krylov_iter"));
      it += n;
      DIFVM_TRY(read_states<NC>(host_state, w, st, done));
      if (done) break;
    }
    return DIFVM_OK;
  };
  if (o->method == DIFVM_PCG) {
    T *r = vec(0), *p = vec(NC), *q = vec(2 * NC);
    k_pcg_init<T, NC><<<G, kKB, 0, st>>>(t, A, jac, b, x, r, p, rD, w);
    DIFVM_TRY(check_launch("pcg_init"));
    k_zero_rhs<T, NC><<<G, kKB, 0, st>>>(nc, x, w);
    DIFVM_TRY(check_launch("zero_rhs"));
    DIFVM_TRY(run([&](cudaStream_t s) {
      prof_before(DIFVM_PROF_PCG_SPMV, s);
      k_pcg_spmv<T, NC, MW><<<G, kKB, 0, s>>>(t, A, p, q, w);
      prof_after(DIFVM_PROF_PCG_SPMV, s);
      prof_before(DIFVM_PROF_PCG_UPDATE, s);
      k_pcg_update<T, NC><<<G, kKB, 0, s>>>(nc, p, q, rD, x, r, w);
      prof_after(DIFVM_PROF_PCG_UPDATE, s);
      prof_before(DIFVM_PROF_PCG_PUPDATE, s);
      k_pcg_pupdate<T, NC><<<G, kKB, 0, s>>>(nc, r, rD, p, w);
      prof_after(DIFVM_PROF_PCG_PUPDATE, s);
      count_launch(); count_launch(); count_launch();
    }));
  } else if (o->method == DIFVM_BICGSTAB) {
    T *r = vec(0), *rh = vec(NC), *p = vec(2 * NC), *v = vec(3 * NC), *s_ = vec(4 * NC),
      *tv = vec(5 * NC), *y = vec(6 * NC), *z = vec(7 * NC);
    const int Gi = wave_grid<k_bicg_init<T, NC>>(m), G1 = wave_grid<k_bicg_spmv1<T, NC, MW>>(m),
              G2 = wave_grid<k_bicg_spmv2<T, NC, MW>>(m), Gu = wave_grid<k_bicg_update<T, NC>>(m);
    k_bicg_init<T, NC><<<Gi, kKB, 0, st>>>(t, A, jac, b, x, r, rh, p, v, rD, w);
    DIFVM_TRY(check_launch("bicg_init"));
    k_zero_rhs<T, NC><<<G, kKB, 0, st>>>(nc, x, w);
    DIFVM_TRY(check_launch("zero_rhs"));
    // algorithmic bytes of one iteration: the LDU matrix (owner, neighbour, L, U per
    // internal face; D) in each of the two products, NC-component vectors once per kernel;
    // a DILU application reads one triangle per sweep, the factor and the vectors
    const uint64_t vb = sizeof(T), ncu = (uint64_t)nc, nq = NC;
    const uint64_t mat = (uint64_t)m->ni * (8 + 2 * vb) + ncu * vb;
    const bool dilu = o->precond == DIFVM_PRECOND_DIC;
    const uint64_t prec_bytes = dilu ? 2 * ((uint64_t)m->ni * (8 + vb) + ncu * vb + 2 * nq * ncu * vb)
                                     : ncu * vb + nq * ncu * vb;   // rD in, the scaled vector out
    const uint64_t it_bytes = 4 * nq * ncu * vb + 2 * prec_bytes + 2 * (mat + 3 * nq * ncu * vb) +
                              3 * nq * ncu * vb + 8 * nq * ncu * vb;
    if (dilu) DIFVM_TRY(ilu_factor<T>(m, A.D, Lraw, Uraw, extra, w.st, NC, st));
    auto precond = [&](const T* a, T* out, cudaStream_t s) {
      if (dilu) ilu_apply<T>(m, NC, Lraw, Uraw, extra, a, out, w.st, NC, s);
      else k_bicg_scale<T, NC><<<G, kKB, 0, s>>>(nc, a, rD, out, w);
    };
    DIFVM_TRY(run([&](cudaStream_t s) {
      count_bytes(it_bytes);
      // Jacobi: the scaling by rD rides in the p and s kernels
      k_bicg_p<T, NC><<<G, kKB, 0, s>>>(nc, r, v, p, dilu ? nullptr : rD, y, w);
      if (dilu) precond(p, y, s);
      k_bicg_spmv1<T, NC, MW><<<G1, kKB, 0, s>>>(t, A, rh, y, v, w);
      k_bicg_s<T, NC><<<G, kKB, 0, s>>>(nc, r, v, s_, dilu ? nullptr : rD, z, w);
      k_bicg_sfinish<T, NC><<<G, kKB, 0, s>>>(nc, y, x, w);
      if (dilu) precond(s_, z, s);
      k_bicg_spmv2<T, NC, MW><<<G2, kKB, 0, s>>>(t, A, z, s_, tv, w);
      k_bicg_update<T, NC><<<Gu, kKB, 0, s>>>(nc, y, z, s_, tv, rh, x, r, w);
      for (int q = 0; q < 6; ++q) count_launch();
    }));
  } else {
    return set_error(DIFVM_EINVAL, "unknown Krylov method %d", o->method);
  }
  if (info) {
    k_write_info<<<1, 32, 0, st>>>(NC, w.st, info, 0);
    DIFVM_TRY(check_launch("write_info"));
  }
  if (graph) return DIFVM_OK;   // outcome in info_dev; the host reads nothing under capture
  DIFVM_TRY(read_states<NC>(host_state, w, st, done));
  int worst = DIFVM_OK;
  for (int c = 0; c < NC; ++c) worst = std::max(worst, host_state[c].status);
  return (difvm_status)worst;
}

// ------------------------------------- mixed precision: reliable-update PCG
// Single-RHS CG whose inner arithmetic (SpMV, vector updates, preconditioner,
// reductions) is FP32 while the solution is accumulated as an unevaluated sum
// of two FP32 words (x = hi + lo, about 48 significant bits, updated with
// error-free transformations) and the residual is periodically REPLACED by the
// true FP64 residual r = b - A (hi + lo) (FP32 matrix values are exact in
// FP64).  This is the iterative-refinement residual of the pressure solve done
// without restarting the Krylov space (residual replacement, van der Vorst &
// Ye, SIAM J. Sci. Comput. 22 (2000)): p keeps its recursive update, r is
// replaced whenever the recursive residual norm has dropped by 1e-2 since the
// last replacement, has reached the tolerance, or the iteration cap is hit;
// the solve ends only when the TRUE FP64 residual meets
// ||r|| <= max(tol_rel ||b||, tol_abs).  No FP64 operation is executed per
// cell on the ordinary iterations (B300 runs FP64 at ~1/60 of FP32).

__device__ __forceinline__ double ffx(const float* hi, const float* lo, int j) {
  return (double)__ldg(hi + j) + (double)__ldg(lo + j);
}

// r64 = b - A x, over a row, x = hi + lo or the FP64 input
template <bool FROM64>
__device__ __forceinline__ double rr_row_residual(const Mat<float>& A, int i, const double* b,
                                                  const double* x64, const float* hi,
                                                  const float* lo) {
  int base, step, wd;
  ell_row(A.E, i, base, step, wd);
  double y = (double)__ldg(A.D + i) * (FROM64 ? x64[i] : ffx(hi, lo, i));
  for (int k = 0; k < wd; ++k) {
    const int j = __ldg(A.E.col + base + step * k);
    y = fma((double)__ldg(A.val + base + step * k), FROM64 ? x64[j] : ffx(hi, lo, j), y);
  }
  return b[i] - y;
}

// init: (hi, lo) = x64, r64 = b - A x64, r = (float) r64, p = rD r; bb, rr (FP64), rz
__global__ void __launch_bounds__(kKB) k_rr_init(Topo t, Mat<float> A, int jacobi, const double* b,
                                                 const double* x, float* hi, float* lo, float* r,
                                                 float* p, float* rD, KWork w) {
  const int nc = t.nc;
  double bb = 0.0, rr = 0.0;
  DotAcc<float> rz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const float di = __ldg(A.D + i);
    const float rd = jacobi ? 1.f / di : 1.f;
    rD[i] = rd;
    const double xi = x[i];
    const float h = (float)xi;
    hi[i] = h;
    lo[i] = (float)(xi - (double)h);
    const double ri = rr_row_residual<true>(A, i, b, x, nullptr, nullptr);
    const double bi = b[i];
    const float rf = (float)ri;
    r[i] = rf;
    p[i] = rf * rd;
    bb = fma(bi, bi, bb);
    rr = fma(ri, ri, rr);
    rz.add(rf, rf * rd);
  }
  double v[3] = {bb, rr, rz.get()}, tot[3];
  if (!grid_sum<3>(w, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[0];
  s.bb = tot[0];
  s.rr = tot[1];
  s.rz = tot[2];
  s.res0 = sqrt(s.rr);
  s.tol2 = fmax(w.tol_rel * w.tol_rel * s.bb, w.tol_abs * w.tol_abs);
  s.iters = 0;
  s.status = DIFVM_OK;
  s.zero_rhs = s.bb == 0.0;
  s.done = s.zero_rhs || s.rr <= s.tol2;
  s.rho = s.rr;  // residual norm^2 at the last replacement
  s.sconv = 0;   // replacement pending
  s.pad0 = 0;    // number of replacements
  if (!finite_d(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; }
}

// (hi, lo) += alpha p (error-free: TwoProduct of alpha p, TwoSum into hi,
// renormalisation); r -= alpha q; recursive rr, rz; replacement decision; beta.
// All arrays live in the 256-byte aligned workspace: 128-bit loads, four cells
// per thread step, scalar tail.
__device__ __forceinline__ void rr_update_one(float al, float pi, float qi, float rdi, float& h,
                                              float& l, float& ri, DotAcc<float>& rr,
                                              DotAcc<float>& rz) {
  const float t = __fmul_rn(al, pi);
  const float et = __fmaf_rn(al, pi, -t);
  const float s = __fadd_rn(h, t);
  const float z = __fsub_rn(s, h);
  float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, z)), __fsub_rn(t, z));
  e = __fadd_rn(e, __fadd_rn(l, et));
  const float hn = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(hn, s));
  h = hn;
  ri = ri - al * qi;
  rr.add(ri, ri);
  rz.add(ri, ri * rdi);
}

__global__ void __launch_bounds__(kKB) k_rr_update(int nc, const float* __restrict__ p,
                                                   const float* __restrict__ q,
                                                   const float* __restrict__ rD,
                                                   float* __restrict__ hi, float* __restrict__ lo,
                                                   float* __restrict__ r, KWork w) {
  if (w.st[0].done) return;
  const float al = (float)w.st[0].alpha;
  DotAcc<float> rr, rz;
  const int n4 = nc >> 2;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int g = tid; g < n4; g += stride) {
    const float4 p4 = reinterpret_cast<const float4*>(p)[g];
    const float4 q4 = reinterpret_cast<const float4*>(q)[g];
    const float4 d4 = reinterpret_cast<const float4*>(rD)[g];
    float4 h4 = reinterpret_cast<float4*>(hi)[g];
    float4 l4 = reinterpret_cast<float4*>(lo)[g];
    float4 r4 = reinterpret_cast<float4*>(r)[g];
    rr_update_one(al, p4.x, q4.x, d4.x, h4.x, l4.x, r4.x, rr, rz);
    rr_update_one(al, p4.y, q4.y, d4.y, h4.y, l4.y, r4.y, rr, rz);
    rr_update_one(al, p4.z, q4.z, d4.z, h4.z, l4.z, r4.z, rr, rz);
    rr_update_one(al, p4.w, q4.w, d4.w, h4.w, l4.w, r4.w, rr, rz);
    reinterpret_cast<float4*>(hi)[g] = h4;
    reinterpret_cast<float4*>(lo)[g] = l4;
    reinterpret_cast<float4*>(r)[g] = r4;
  }
  for (int i = 4 * n4 + tid; i < nc; i += stride) {
    float h = hi[i], l = lo[i], ri = r[i];
    rr_update_one(al, p[i], q[i], rD[i], h, l, ri, rr, rz);
    hi[i] = h;
    lo[i] = l;
    r[i] = ri;
  }
  float2 v[2] = {rr.part(), rz.part()};
  double tot[2];
  if (!grid_sum<2>(w, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[0];
  s.iters += 1;
  if (!finite_d(tot[0]) || !finite_d(s.alpha)) { s.done = 1; s.status = DIFVM_ENONFINITE; return; }
  s.beta = tot[1] / s.rz;
  s.rz = tot[1];
  s.rr = tot[0];
  s.sconv = (tot[0] <= s.tol2) || (tot[0] <= 1e-4 * s.rho) || (s.iters >= w.maxit);
}

// p = rD r + beta p (with the recursive r); on replacement steps also
// r = (float)(b - A (hi + lo)) and the FP64 true residual decides convergence.
__global__ void __launch_bounds__(kKB, 4) k_rr_pupdate(Topo t, Mat<float> A, const double* b,
                                                       const float* hi, const float* lo, float* r,
                                                       const float* rD, float* p, KWork w) {
  if (w.st[0].done) return;
  const int nc = t.nc;
  const float be = (float)w.st[0].beta;
  const bool rep = w.st[0].sconv;
  if (!rep) {
    const int n4 = nc >> 2;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int g = tid; g < n4; g += stride) {
      const float4 r4 = reinterpret_cast<const float4*>(r)[g];
      const float4 d4 = reinterpret_cast<const float4*>(rD)[g];
      float4 p4 = reinterpret_cast<float4*>(p)[g];
      p4.x = r4.x * d4.x + be * p4.x;
      p4.y = r4.y * d4.y + be * p4.y;
      p4.z = r4.z * d4.z + be * p4.z;
      p4.w = r4.w * d4.w + be * p4.w;
      reinterpret_cast<float4*>(p)[g] = p4;
    }
    for (int i = 4 * n4 + tid; i < nc; i += stride) p[i] = r[i] * rD[i] + be * p[i];
    return;
  }
  double rr = 0.0;
  DotAcc<float> rz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const float rd = rD[i];
    p[i] = r[i] * rd + be * p[i];
    const double rt = rr_row_residual<false>(A, i, b, nullptr, hi, lo);
    const float rf = (float)rt;
    r[i] = rf;
    rr = fma(rt, rt, rr);
    rz.add(rf, rf * rd);
  }
  double v[2] = {rr, rz.get()}, tot[2];
  if (!grid_sum<2>(w, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[0];
  s.sconv = 0;
  s.pad0 += 1;
  s.rr = tot[0];
  s.rz = tot[1];
  s.rho = tot[0];
  if (!finite_d(tot[0])) { s.done = 1; s.status = DIFVM_ENONFINITE; return; }
  if (tot[0] <= s.tol2) { s.done = 1; return; }
  if (s.iters >= w.maxit) { s.done = 1; s.status = DIFVM_ENOTCONV; }
}

// x64 = hi + lo (or 0 for a zero right-hand side)
__global__ void k_rr_final(int nc, const float* hi, const float* lo, double* x, KWork w) {
  const bool z = w.st[0].zero_rhs;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
    x[i] = z ? 0.0 : (double)hi[i] + (double)lo[i];
}

__global__ void k_rr_info(const KState* st, difvm_solve_info* info) {
  if (threadIdx.x != 0) return;
  const KState& s = st[0];
  difvm_solve_info o;
  o.iters = s.iters;
  o.refinements = s.pad0;
  o.status = s.status;
  o.pad = 0;
  o.res0 = s.res0;
  o.res = sqrt(s.rr);
  o.bnorm = sqrt(s.bb);
  *info = o;
}

// workspace: [r p q rD hi lo | ELL values | state | block partials | ticket]
static size_t rr_bytes(const difvm_mesh* m, size_t* val_off, size_t* st_off, size_t* part_off,
                       size_t* tick_off) {
  size_t vb = up256((size_t)m->nc * 4);
  size_t v0 = 6 * vb;
  size_t so = v0 + up256((size_t)std::max<int64_t>(m->ell_nslots, 1) * 4);
  size_t po = so + 256 * 4;
  size_t to = po + up256((size_t)grid_for(m) * kMaxParts * sizeof(double));
  if (val_off) *val_off = v0;
  if (st_off) *st_off = so;
  if (part_off) *part_off = po;
  if (tick_off) *tick_off = to;
  return to + 256;
}

template <int MW>
static difvm_status rr_pcg(difvm_mesh_t m, const difvm_solve_opts* o, const float* D, const float* L,
                           const double* b64, double* x64, char* ws, size_t wsbytes,
                           difvm_solve_info* info, cudaStream_t st) {
  size_t vo, so, po, to;
  size_t need = rr_bytes(m, &vo, &so, &po, &to);
  if (wsbytes < need) return set_error(DIFVM_EINVAL, "workspace of %zu bytes < %zu needed", wsbytes, need);
  const int nc = m->nc, G = grid_for(m);
  const size_t vb = up256((size_t)nc * 4);
  float *r = (float*)ws, *p = (float*)(ws + vb), *q = (float*)(ws + 2 * vb), *rD = (float*)(ws + 3 * vb);
  float *hi = (float*)(ws + 4 * vb), *lo = (float*)(ws + 5 * vb);
  float* val = (float*)(ws + vo);
  KWork w;
  w.st = (KState*)(ws + so);
  w.part = (double*)(ws + po);
  w.ticket = (unsigned*)(ws + to);
  w.maxit = o->max_iter > 0 ? o->max_iter : 1000;
  w.tol_rel = o->tol_rel;
  w.tol_abs = o->tol_abs;
  DIFVM_TRY(fill_ell<float>(m, L, nullptr, val, st));
  Mat<float> A{D, m->ell(), val};
  Topo t = m->topo();
  const int jac = o->precond != DIFVM_PRECOND_NONE;
  const int chunk = o->check_every > 0 ? o->check_every : 8;
  DIFVM_CUDA(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), st));
  k_rr_init<<<G, kKB, 0, st>>>(t, A, jac, b64, x64, hi, lo, r, p, rD, w);
  DIFVM_TRY(check_launch("rr_init"));
  KState hs[1];
  bool done = false;
  auto iter = [&](cudaStream_t s) {
    prof_before(DIFVM_PROF_PCG_SPMV, s);
    k_pcg_spmv<float, 1, MW><<<G, kKB, 0, s>>>(t, A, p, q, w);
    prof_after(DIFVM_PROF_PCG_SPMV, s);
    prof_before(DIFVM_PROF_PCG_UPDATE, s);
    k_rr_update<<<G, kKB, 0, s>>>(nc, p, q, rD, hi, lo, r, w);
    prof_after(DIFVM_PROF_PCG_UPDATE, s);
    prof_before(DIFVM_PROF_PCG_PUPDATE, s);
    k_rr_pupdate<<<G, kKB, 0, s>>>(t, A, b64, hi, lo, r, rD, p, w);
    prof_after(DIFVM_PROF_PCG_PUPDATE, s);
    count_launch(); count_launch(); count_launch();
  };
  const bool graph = stream_capturing(st);
  if (graph) {
    int* counter = reinterpret_cast<int*>(w.ticket) + 1;
    DIFVM_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
    WhileLoop Lw;
    DIFVM_TRY(while_open(st, Lw));
    for (int k = 0; k < kGraphUnroll; ++k) iter(Lw.side);
    k_loop_cond<<<1, 32, 0, Lw.side>>>(done_flags(w.st), kStateInts, 1, counter,
                                       w.maxit / kGraphUnroll + 2, Lw.h);
    difvm_status e = check_launch("loop_cond");
    DIFVM_TRY(while_close(Lw));
    DIFVM_TRY(e);
  } else {
    // the iteration cap is enforced on the device; the host loop is bounded as well
    for (int it = 0; it < w.maxit + chunk; it += chunk) {
      for (int k = 0; k < chunk; ++k) iter(st);
      DIFVM_TRY(check_error("rr_iter"));
      DIFVM_TRY(read_states<1>(hs, w, st, done));
      if (done) break;
    }
  }
  k_rr_final<<<G, kKB, 0, st>>>(nc, hi, lo, x64, w);
  DIFVM_TRY(check_launch("rr_final"));
  if (info) {
    k_rr_info<<<1, 32, 0, st>>>(w.st, info);
    DIFVM_TRY(check_launch("rr_info"));
  }
  if (graph) return DIFVM_OK;   // outcome in info_dev
  DIFVM_TRY(read_states<1>(hs, w, st, done));
  int s = hs[0].status;
  if (s == DIFVM_OK && !hs[0].done) s = DIFVM_ENOTCONV;
  return (difvm_status)s;
}

static int maxw_bucket(const difvm_mesh* m) { return m->ell_wmax <= 4 ? 4 : (m->ell_wmax <= 8 ? 8 : 0); }

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

// ====================================================== segmented (batched)
// (SWork, seg_block and seg_sum: krylov_common.cuh)

template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_sg_pcg_init(Topo t, Mat<T> A, int jacobi, const T* b, T* x,
                                                     T* r, T* p, T* rD, SWork w) {
  const SegBlock B = seg_block(w);
  const int nc = t.nc;
  DotAcc<T> bb[NC], rr[NC], rz[NC];
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
    const T di = __ldg(A.D + i);
    const T rd = jacobi ? T(1) / di : T(1);
    rD[i] = rd;
    T ax[NC];
    spmv_row<T, NC, 0>(t, A, i, x, ax, (1u << NC) - 1);
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
  if (!seg_sum<3 * NC>(w, B.k, v, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    KState& s = w.st[B.k * NC + c];
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

template <typename T, int NC, int MAXW>
__global__ void __launch_bounds__(kKB) k_sg_pcg_spmv(Topo t, Mat<T> A, const T* p, T* q, SWork w) {
  const SegBlock B = seg_block(w);
  const unsigned act = seg_active<NC>(w, B.k);
  if (!act) return;
  const int nc = t.nc;
  DotAcc<T> pq[NC];
#pragma unroll 4
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
    T y[NC];
    spmv_row<T, NC, MAXW>(t, A, i, p, y, act);
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
  if (!seg_sum<NC>(w, B.k, v, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (act >> c & 1) w.st[B.k * NC + c].alpha = w.st[B.k * NC + c].rz / tot[c];
}

template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_sg_pcg_update(int nc, const T* p, const T* q, const T* rD,
                                                       T* x, T* r, SWork w) {
  const SegBlock B = seg_block(w);
  const unsigned act = seg_active<NC>(w, B.k);
  if (!act) return;
  T al[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) al[c] = (T)w.st[B.k * NC + c].alpha;
  DotAcc<T> rr[NC], rz[NC];
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
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
  if (!seg_sum<2 * NC>(w, B.k, v, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (!(act >> c & 1)) continue;
    KState& s = w.st[B.k * NC + c];
    s.iters += 1;
    s.rr = tot[2 * c];
    if (!finite_d(s.rr) || !finite_d(s.alpha)) { s.done = 1; s.status = DIFVM_ENONFINITE; continue; }
    if (s.rr <= s.tol2) { s.done = 1; continue; }
    if (s.iters >= w.maxit) { s.done = 1; s.status = DIFVM_ENOTCONV; continue; }
    s.beta = tot[2 * c + 1] / s.rz;
    s.rz = tot[2 * c + 1];
  }
}

template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_sg_pcg_pupdate(int nc, const T* r, const T* rD, T* p, SWork w) {
  const SegBlock B = seg_block(w);
  const unsigned act = seg_active<NC>(w, B.k);
  if (!act) return;
  T be[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) be[c] = (T)w.st[B.k * NC + c].beta;
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
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
__global__ void k_sg_zero_rhs(int nc, T* x, SWork w) {
  const SegBlock B = seg_block(w);
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (w.st[B.k * NC + c].zero_rhs) x[c * nc + i] = T(0);
}

template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_sg_bicg_init(Topo t, Mat<T> A, int jacobi, const T* b, T* x,
                                                      T* r, T* rh, T* p, T* v, T* rD, SWork w) {
  const SegBlock B = seg_block(w);
  const int nc = t.nc;
  DotAcc<T> bb[NC], rr[NC];
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
    const T di = __ldg(A.D + i);
    rD[i] = jacobi ? T(1) / di : T(1);
    T ax[NC];
    spmv_row<T, NC, 0>(t, A, i, x, ax, (1u << NC) - 1);
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
  if (!seg_sum<2 * NC>(w, B.k, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    KState& s = w.st[B.k * NC + c];
    s.bb = tot[2 * c];
    s.rr = tot[2 * c + 1];
    s.rz = s.rr;
    s.res0 = sqrt(s.rr);
    s.tol2 = fmax(w.tol_rel * w.tol_rel * s.bb, w.tol_abs * w.tol_abs);
    s.iters = 0;
    s.status = DIFVM_OK;
    s.rho = 1.0; s.alpha = 1.0; s.omega = 1.0;
    s.beta = (s.rz / s.rho) * (s.alpha / s.omega);
    s.sconv = 0;
    s.zero_rhs = s.bb == 0.0;
    s.done = s.zero_rhs || s.rr <= s.tol2;
    if (!finite_d(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; }
  }
}

template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_sg_bicg_p(int nc, const T* r, const T* v, T* p, SWork w) {
  const SegBlock B = seg_block(w);
  const unsigned act = seg_active<NC>(w, B.k);
  if (!act) return;
  T be[NC], om[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const KState& s = w.st[B.k * NC + c];
    be[c] = (T)s.beta;   // formed once by the last block of the update
    om[c] = (T)s.omega;
  }
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) {
        const int k = c * nc + i;
        p[k] = r[k] + be[c] * (p[k] - om[c] * v[k]);
      }
}

template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_sg_bicg_scale(int nc, const T* a, const T* rD, T* y, SWork w,
                                                       int second) {
  const SegBlock B = seg_block(w);
  unsigned act = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const KState& s = w.st[B.k * NC + c];
    if (!s.done && !(second && s.sconv)) act |= 1u << c;
  }
  if (!act) return;
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
    const T rd = rD[i];
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (act >> c & 1) y[c * nc + i] = a[c * nc + i] * rd;
  }
}

template <typename T, int NC, int MAXW>
__global__ void __launch_bounds__(kKB) k_sg_bicg_spmv1(Topo t, Mat<T> A, const T* rh, const T* y, T* v,
                                                       SWork w) {
  const SegBlock B = seg_block(w);
  const unsigned act = seg_active<NC>(w, B.k);
  if (!act) return;
  const int nc = t.nc;
  DotAcc<T> rv[NC];
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
    T a[NC];
    spmv_row<T, NC, MAXW>(t, A, i, y, a, act);
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
  if (!seg_sum<NC>(w, B.k, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (!(act >> c & 1)) continue;
    KState& s = w.st[B.k * NC + c];
    s.rho = s.rz;
    if (s.rho == 0.0 || tot[c] == 0.0 || s.omega == 0.0) { s.done = 1; s.status = DIFVM_EBREAKDOWN; continue; }
    s.alpha = s.rho / tot[c];
  }
}

template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_sg_bicg_s(int nc, const T* r, const T* v, T* s_, SWork w) {
  const SegBlock B = seg_block(w);
  const unsigned act = seg_active<NC>(w, B.k);
  if (!act) return;
  T al[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) al[c] = (T)w.st[B.k * NC + c].alpha;
  DotAcc<T> ss[NC];
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x)
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
  if (!seg_sum<NC>(w, B.k, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (!(act >> c & 1)) continue;
    KState& s = w.st[B.k * NC + c];
    s.iters += 1;
    s.pq = tot[c];
    s.sconv = tot[c] <= s.tol2;
    if (s.sconv) s.rr = tot[c];
  }
}

template <typename T, int NC>
__global__ void k_sg_bicg_sfinish(int nc, const T* y, T* x, SWork w) {
  const SegBlock B = seg_block(w);
  unsigned fin = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (!w.st[B.k * NC + c].done && w.st[B.k * NC + c].sconv) fin |= 1u << c;
  if (!fin) return;
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (fin >> c & 1) x[c * nc + i] += (T)w.st[B.k * NC + c].alpha * y[c * nc + i];
}

template <typename T, int NC, int MAXW>
__global__ void __launch_bounds__(kKB) k_sg_bicg_spmv2(Topo t, Mat<T> A, const T* z, const T* s_, T* tv,
                                                       SWork w) {
  const SegBlock B = seg_block(w);
  unsigned act = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (!w.st[B.k * NC + c].done && !w.st[B.k * NC + c].sconv) act |= 1u << c;
  if (!act) return;
  const int nc = t.nc;
  DotAcc<T> ts[NC], tt[NC];
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
    T a[NC];
    spmv_row<T, NC, MAXW>(t, A, i, z, a, act);
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
  if (!seg_sum<2 * NC>(w, B.k, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (act >> c & 1)
      w.st[B.k * NC + c].omega = tot[2 * c + 1] > 0.0 ? tot[2 * c] / tot[2 * c + 1] : 0.0;
}

template <typename T, int NC>
__global__ void __launch_bounds__(kKB) k_sg_bicg_update(int nc, const T* y, const T* z, const T* s_,
                                                        const T* tv, const T* rh, T* x, T* r, SWork w) {
  const SegBlock B = seg_block(w);
  unsigned act = 0, fin = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const KState& s = w.st[B.k * NC + c];
    if (!s.done && !s.sconv) act |= 1u << c;
    if (!s.done && s.sconv) fin |= 1u << c;
  }
  // components that converged on s are closed by the case's first block
  if (!act) {
    if (fin && blockIdx.x == __ldg(w.cb0 + B.k) && threadIdx.x == 0)
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (fin >> c & 1) w.st[B.k * NC + c].done = 1;
    return;
  }
  T al[NC], om[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    al[c] = (T)w.st[B.k * NC + c].alpha;
    om[c] = (T)w.st[B.k * NC + c].omega;
  }
  DotAcc<T> rr[NC], rhr[NC];
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x)
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
  if (!seg_sum<2 * NC>(w, B.k, vv, tot) || threadIdx.x != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    KState& s = w.st[B.k * NC + c];
    if (!s.done && s.sconv) { s.done = 1; continue; }
    if (!(act >> c & 1)) continue;
    s.rr = tot[2 * c];
    s.rz = tot[2 * c + 1];
    s.beta = (s.rz / s.rho) * (s.alpha / s.omega);
    if (!finite_d(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; continue; }
    if (s.rr <= s.tol2) { s.done = 1; continue; }
    if (s.iters >= w.maxit) { s.done = 1; s.status = DIFVM_ENOTCONV; continue; }
  }
}

__global__ void k_sg_write_info(int n, const KState* st, difvm_solve_info* info) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const KState& s = st[c];
  difvm_solve_info o;
  o.iters = s.iters;
  o.refinements = 0;
  o.status = s.status;
  o.pad = 0;
  o.res0 = s.res0;
  o.res = sqrt(s.rr);
  o.bnorm = sqrt(s.bb);
  info[c] = o;
}

// 1 while any (case, component) is still iterating (host poll)
__global__ void k_sg_any_active(int n, const KState* st, int* out) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    if (!st[c].done) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) *out = any;
}

template <typename T, int NC, int MW>
static difvm_status solve_sg(difvm_mesh_t m, const difvm_solve_opts* o, Mat<T> A, const T* b, T* x,
                             char* ws, const WsLayout& L, difvm_solve_info* info, cudaStream_t st) {
  const int nc = m->nc, G = m->seg_nblk, nst = m->ncases * NC;
  Topo t = m->topo();
  auto vec = [&](int k) { return (T*)(ws + (size_t)k * L.vec_bytes); };
  SWork w;
  w.st = (KState*)(ws + L.state_off);
  w.part = (double*)(ws + L.part_off);
  w.ticket = (unsigned*)(ws + L.ticket_off);
  w.bcase = m->seg_case;
  w.cb0 = m->seg_cb0;
  w.cs = m->seg_cs;
  w.maxit = o->max_iter > 0 ? o->max_iter : 1000;
  w.tol_rel = o->tol_rel;
  w.tol_abs = o->tol_abs;
  int* flag = (int*)(ws + L.flag_off);
  const int jac = o->precond != DIFVM_PRECOND_NONE;
  const int chunk = o->check_every > 0 ? o->check_every : 8;
  DIFVM_CUDA(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned) * m->ncases, st));
  T* rD = vec(L.n_vec - 1);
  int host_flag = 1;
  auto poll = [&]() -> difvm_status {
    k_sg_any_active<<<1, 256, 0, st>>>(nst, w.st, flag);
    DIFVM_TRY(check_launch("sg_any_active"));
    DIFVM_CUDA(cudaMemcpyAsync(&host_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DIFVM_CUDA(cudaStreamSynchronize(st));
    return DIFVM_OK;
  };
  const bool graph = stream_capturing(st);
  int* counter = flag + 1;   // loop counter under a graph
  auto run = [&](auto&& iter) -> difvm_status {
    if (graph) {
      DIFVM_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
      WhileLoop Lw;
      DIFVM_TRY(while_open(st, Lw));
      for (int k = 0; k < kGraphUnroll; ++k) iter(Lw.side);
      k_loop_cond<<<1, 32, 0, Lw.side>>>(done_flags(w.st), kStateInts, nst, counter,
                                         w.maxit / kGraphUnroll + 2, Lw.h);
      difvm_status e = check_launch("loop_cond");
      DIFVM_TRY(while_close(Lw));
      return e;
    }
    for (int it = 0; it < w.maxit;) {
      const int n = std::min(chunk, w.maxit - it);
      for (int k = 0; k < n; ++k) iter(st);
      DIFVM_TRY(check_error("sg_iter"));
      it += n;
      DIFVM_TRY(poll());
      if (!host_flag) break;
    }
    return DIFVM_OK;
  };
  if (o->method == DIFVM_PCG) {
    T *r = vec(0), *p = vec(NC), *q = vec(2 * NC);
    k_sg_pcg_init<T, NC><<<G, kKB, 0, st>>>(t, A, jac, b, x, r, p, rD, w);
    DIFVM_TRY(check_launch("sg_pcg_init"));
    k_sg_zero_rhs<T, NC><<<G, kKB, 0, st>>>(nc, x, w);
    DIFVM_TRY(check_launch("sg_zero_rhs"));
    DIFVM_TRY(run([&](cudaStream_t s) {
      k_sg_pcg_spmv<T, NC, MW><<<G, kKB, 0, s>>>(t, A, p, q, w);
      k_sg_pcg_update<T, NC><<<G, kKB, 0, s>>>(nc, p, q, rD, x, r, w);
      k_sg_pcg_pupdate<T, NC><<<G, kKB, 0, s>>>(nc, r, rD, p, w);
      count_launch(); count_launch(); count_launch();
    }));
  } else if (o->method == DIFVM_BICGSTAB) {
    T *r = vec(0), *rh = vec(NC), *p = vec(2 * NC), *v = vec(3 * NC), *s_ = vec(4 * NC),
      *tv = vec(5 * NC), *y = vec(6 * NC), *z = vec(7 * NC);
    k_sg_bicg_init<T, NC><<<G, kKB, 0, st>>>(t, A, jac, b, x, r, rh, p, v, rD, w);
    DIFVM_TRY(check_launch("sg_bicg_init"));
    k_sg_zero_rhs<T, NC><<<G, kKB, 0, st>>>(nc, x, w);
    DIFVM_TRY(check_launch("sg_zero_rhs"));
    DIFVM_TRY(run([&](cudaStream_t s) {
      k_sg_bicg_p<T, NC><<<G, kKB, 0, s>>>(nc, r, v, p, w);
      k_sg_bicg_scale<T, NC><<<G, kKB, 0, s>>>(nc, p, rD, y, w, 0);
      k_sg_bicg_spmv1<T, NC, MW><<<G, kKB, 0, s>>>(t, A, rh, y, v, w);
      k_sg_bicg_s<T, NC><<<G, kKB, 0, s>>>(nc, r, v, s_, w);
      k_sg_bicg_sfinish<T, NC><<<G, kKB, 0, s>>>(nc, y, x, w);
      k_sg_bicg_scale<T, NC><<<G, kKB, 0, s>>>(nc, s_, rD, z, w, 1);
      k_sg_bicg_spmv2<T, NC, MW><<<G, kKB, 0, s>>>(t, A, z, s_, tv, w);
      k_sg_bicg_update<T, NC><<<G, kKB, 0, s>>>(nc, y, z, s_, tv, rh, x, r, w);
      for (int q = 0; q < 8; ++q) count_launch();
    }));
  } else {
    return set_error(DIFVM_EINVAL, "unknown Krylov method %d", o->method);
  }
  if (info) {
    k_sg_write_info<<<blocks_for(nst, 128), 128, 0, st>>>(nst, w.st, info);
    DIFVM_TRY(check_launch("sg_write_info"));
  }
  if (graph) return DIFVM_OK;   // outcome in info_dev
  // worst status over all cases and components
  std::vector<KState> hs(nst);
  DIFVM_CUDA(cudaMemcpyAsync(hs.data(), w.st, sizeof(KState) * nst, cudaMemcpyDeviceToHost, st));
  DIFVM_CUDA(cudaStreamSynchronize(st));
  int worst = DIFVM_OK;
  for (const KState& s : hs) worst = std::max(worst, s.status);
  return (difvm_status)worst;
}

template <typename T>
static difvm_status solve_t(difvm_mesh_t m, const difvm_solve_opts* o, const void* D, const void* L,
                            const void* U, const void* b, void* x, int ncomp, void* ws,
                            size_t wsbytes, difvm_solve_info* info, cudaStream_t st) {
  if (o->precond == DIFVM_PRECOND_AMG || o->precond == DIFVM_PRECOND_AMG_REUSE) {
    if (o->method != DIFVM_PCG || ncomp != 1 || U)
      return set_error(DIFVM_EINVAL, "the multigrid preconditioner serves single-RHS CG on a "
                                     "symmetric matrix");
    return amg_solve<T>(m, o, (const T*)D, (const T*)L, (const T*)b, (T*)x, ws, wsbytes, info, st);
  }
  const bool dilu = o->precond == DIFVM_PRECOND_DIC && o->method == DIFVM_BICGSTAB;
  if (o->precond == DIFVM_PRECOND_DIC) {
    if (m->seg || (o->method == DIFVM_PCG && (ncomp != 1 || U)))
      return set_error(DIFVM_EINVAL, "the incomplete factorisation serves single-RHS CG on a symmetric "
                                     "matrix (DIC) or BiCGStab (DILU), on a single (not batched) mesh");
    if (!dilu) return dic_solve<T>(m, o, (const T*)D, (const T*)L, (const T*)b, (T*)x, ws, wsbytes, info, st);
  }
  WsLayout Ly = layout(m, sizeof(T), o->method, ncomp);
  const size_t need = Ly.total + (dilu ? ilu_extra_bytes(m, sizeof(T)) : 0);
  if (!ws || wsbytes < need)
    return set_error(DIFVM_EINVAL, "workspace of %zu bytes < %zu needed", wsbytes, need);
  char* extra = dilu ? (char*)ws + Ly.total : nullptr;
  T* val = (T*)((char*)ws + Ly.val_off);
  DIFVM_TRY(fill_ell<T>(m, (const T*)L, (const T*)U, val, st));
  Mat<T> A{(const T*)D, m->ell(), val};
  KState hs[3];
  const int mw = maxw_bucket(m);
  if (m->seg) {
#define DIFVM_SOLVE(NC, MW) solve_sg<T, NC, MW>(m, o, A, (const T*)b, (T*)x, (char*)ws, Ly, info, st)
    switch (ncomp * 16 + mw) {
      case 16 + 4: return DIFVM_SOLVE(1, 4);
      case 16 + 8: return DIFVM_SOLVE(1, 8);
      case 16 + 0: return DIFVM_SOLVE(1, 0);
      case 32 + 4: return DIFVM_SOLVE(2, 4);
      case 32 + 8: return DIFVM_SOLVE(2, 8);
      case 32 + 0: return DIFVM_SOLVE(2, 0);
      case 48 + 4: return DIFVM_SOLVE(3, 4);
      case 48 + 8: return DIFVM_SOLVE(3, 8);
      case 48 + 0: return DIFVM_SOLVE(3, 0);
    }
#undef DIFVM_SOLVE
    return set_error(DIFVM_EINVAL, "ncomp must be 1..3");
  }
#define DIFVM_SOLVE(NC, MW) solve_nc<T, NC, MW>(m, o, A, (const T*)b, (T*)x, (char*)ws, Ly, info, st, hs, \
                                               (const T*)L, (const T*)(U ? U : L), extra)
  switch (ncomp * 16 + mw) {
    case 16 + 4: return DIFVM_SOLVE(1, 4);
    case 16 + 8: return DIFVM_SOLVE(1, 8);
    case 16 + 0: return DIFVM_SOLVE(1, 0);
    case 32 + 4: return DIFVM_SOLVE(2, 4);
    case 32 + 8: return DIFVM_SOLVE(2, 8);
    case 32 + 0: return DIFVM_SOLVE(2, 0);
    case 48 + 4: return DIFVM_SOLVE(3, 4);
    case 48 + 8: return DIFVM_SOLVE(3, 8);
    case 48 + 0: return DIFVM_SOLVE(3, 0);
  }
#undef DIFVM_SOLVE
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

extern "C" size_t difvm_krylov_opts_workspace_bytes(difvm_mesh_t m, difvm_prec prec,
                                                    const difvm_solve_opts* o, int ncomp) {
  if (!m || !o || ncomp < 1 || ncomp > 3) return 0;
  const bool refine = prec == DIFVM_F32 && o->refine_max > 0;
  if (o->precond == DIFVM_PRECOND_AMG || o->precond == DIFVM_PRECOND_AMG_REUSE) {
    if (o->method != DIFVM_PCG || ncomp != 1 || (m->seg && refine)) return 0;
    return amg_workspace_bytes(m, refine ? 4 : (prec == DIFVM_F64 ? 8 : 4));
  }
  if (o->precond == DIFVM_PRECOND_DIC) {
    if (m->seg || refine) return 0;
    if (o->method == DIFVM_PCG) return ncomp == 1 ? dic_workspace_bytes(m, prec == DIFVM_F64 ? 8 : 4) : 0;
    dic_workspace_bytes(m, 4);   // builds the dependency levels
    const size_t e = prec == DIFVM_F64 ? 8 : 4;
    return difvm_krylov_workspace_bytes(m, prec, o->method, ncomp) + ilu_extra_bytes(m, e);
  }
  const size_t plain = difvm_krylov_workspace_bytes(m, prec, o->method, ncomp);
  return refine ? std::max(plain, difvm_krylov_refine_workspace_bytes(m, o->method, ncomp)) : plain;
}

extern "C" size_t difvm_krylov_refine_workspace_bytes(difvm_mesh_t m, int method, int ncomp) {
  if (!m || ncomp != 1 || method != DIFVM_PCG) return 0;
  return rr_bytes(m, nullptr, nullptr, nullptr, nullptr);
}

extern "C" difvm_status difvm_krylov_solve_refine(difvm_mesh_t m, const difvm_solve_opts* o,
                                                  const float* D, const float* L, const float* U,
                                                  const double* b64, double* x64, int ncomp, void* ws,
                                                  size_t wsbytes, difvm_solve_info* info, void* stream) {
  DIFVM_TRY(check_solve(m, DIFVM_F32, o, ncomp, D, L));
  if (m->seg) return set_error(DIFVM_EINVAL, "difvm_krylov_solve_refine: not available on batched meshes");
  if (o->precond == DIFVM_PRECOND_AMG || o->precond == DIFVM_PRECOND_AMG_REUSE) {
    if (o->method != DIFVM_PCG || ncomp != 1 || U)
      return set_error(DIFVM_EINVAL, "the multigrid preconditioner serves single-RHS CG on a symmetric matrix");
    if (!b64 || !x64) return set_error(DIFVM_EINVAL, "null vector");
    return amg_refine(m, o, D, L, b64, x64, ws, wsbytes, info, (cudaStream_t)stream);
  }
  if (ncomp != 1 || o->method != DIFVM_PCG)
    return set_error(DIFVM_EINVAL, "the mixed-precision solve is single-RHS PCG");
  if (U) return set_error(DIFVM_EINVAL, "the mixed-precision PCG needs a symmetric matrix (upper = NULL)");
  if (!b64 || !x64 || !ws) return set_error(DIFVM_EINVAL, "null vector or workspace");
  cudaStream_t st = (cudaStream_t)stream;
  switch (maxw_bucket(m)) {
    case 4: return rr_pcg<4>(m, o, D, L, b64, x64, (char*)ws, wsbytes, info, st);
    case 8: return rr_pcg<8>(m, o, D, L, b64, x64, (char*)ws, wsbytes, info, st);
    default: return rr_pcg<0>(m, o, D, L, b64, x64, (char*)ws, wsbytes, info, st);
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
