// PISO step with the RCR Windkessel outlet (Sec. 2.4.2, 2.6.3), device-resident.
//
// One step:  Windkessel (Q from the current face flux, exact / FE / BE update,
// p_out imposed on the outlet patch)  ->  momentum predictor (backward Euler,
// implicit upwind convection with the current flux, implicit orthogonal and
// explicit over-relaxed non-orthogonal diffusion; BiCGStab on the three
// components at once)  ->  n_corr pressure correctors (HbyA, face flux
// phiHbyA, weighted graph Laplacian of Eq. pressure_poisson with face weight
// (V/D)_f c_f, PCG, Rhie-Chow flux correction, velocity correction of
// Eq. velocity_correction).
//
// Face coefficients that two cells share are written once by a face kernel
// (L/U of the momentum matrix, phiHbyA, a_f, the non-orthogonal flux); cell
// kernels then reduce them over the cell-CSR rows in ascending face order.
#include <math.h>

#include <algorithm>

#include "difvm_internal.cuh"

struct difvm_piso {
  difvm_mesh* m = nullptr;
  difvm_prec prec = DIFVM_F64;
  difvm_piso_opts o{};
  bool mixed = false;
  int has_fixed_p = 0;
  size_t elt = 8;
  void *gradp = nullptr, *gradU = nullptr, *D = nullptr, *Lo = nullptr, *Up = nullptr, *b = nullptr;
  void *rhs = nullptr, *rAU = nullptr, *HbyA = nullptr, *Dp = nullptr, *Lp = nullptr, *bp = nullptr;
  void *phiHbyA = nullptr, *af = nullptr, *nonorth = nullptr;
  void* wsU = nullptr;
  size_t wsU_bytes = 0;
  void* wsp = nullptr;
  size_t wsp_bytes = 0;
  double *p64 = nullptr, *b64 = nullptr;
  difvm_solve_info* sinfo = nullptr;  // [3 + 4] device
  std::vector<void*> allocs;
};

namespace difvm {

constexpr int kPB = 256;

// ------------------------------------------------------------- Windkessel
__device__ __forceinline__ void wk_step(int scheme, double Rp, double C, double Rd, double Q,
                                        double dt, double& pc, double& po) {
  if (scheme == DIFVM_WK_EXACT) {
    const double e = exp(-dt / (Rd * C));
    pc = pc * e + Rd * Q * (1.0 - e);
  } else if (scheme == DIFVM_WK_FE) {
    pc = pc + dt * (Q - pc / Rd) / C;
  } else {
    pc = (pc + dt * Q / C) / (1.0 + dt / (Rd * C));
  }
  po = pc + Rp * Q;
}

__global__ void k_windkessel(int n, int scheme, const double* Rp, const double* C, const double* Rd,
                             const double* Q, double dt, double* pc, double* po) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  double p = pc[o], out;
  wk_step(scheme, Rp[o], C[o], Rd[o], Q[o], dt, p, out);
  pc[o] = p;
  if (po) po[o] = out;
}

// Adjoint of one RCR step (closed-form derivatives of the three updates).
__global__ void k_windkessel_bwd(int n, int scheme, const double* Rp, const double* C,
                                 const double* Rd, const double* Q, double dt, const double* pc_in,
                                 const double* pcb, const double* pob, double* pc_in_bar,
                                 double* Qb, double* Rpb, double* Cb, double* Rdb) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const double rp = Rp[o], c = C[o], rd = Rd[o], q = Q[o], p0 = pc_in[o];
  const double pob_ = pob ? pob[o] : 0.0;
  const double g = (pcb ? pcb[o] : 0.0) + pob_;
  double dp0, dq, drd, dc;
  if (scheme == DIFVM_WK_EXACT) {
    const double e = exp(-dt / (rd * c));
    dp0 = e;
    dq = rd * (1.0 - e);
    const double de = p0 - rd * q;                 // d pc_out / d e
    drd = de * e * dt / (rd * rd * c) + q * (1.0 - e);
    dc = de * e * dt / (rd * c * c);
  } else if (scheme == DIFVM_WK_FE) {
    dp0 = 1.0 - dt / (rd * c);
    dq = dt / c;
    drd = dt * p0 / (rd * rd * c);
    dc = -dt * (q - p0 / rd) / (c * c);
  } else {
    const double M = 1.0 + dt / (rd * c), N = p0 + dt * q / c;
    dp0 = 1.0 / M;
    dq = dt / (c * M);
    drd = N * dt / (M * M * rd * rd * c);
    dc = -dt * q / (c * c * M) + N * dt / (M * M * rd * c * c);
  }
  if (pc_in_bar) pc_in_bar[o] = g * dp0;
  if (Qb) Qb[o] += g * dq + pob_ * rp;
  if (Rpb) Rpb[o] += pob_ * q;
  if (Cb) Cb[o] += g * dc;
  if (Rdb) Rdb[o] += g * drd;
}

// One block per outlet: Q = sum of the patch's face flux (fixed order), RCR
// step on wk = (Rp, C, Rd, p_c), p_out written to every face of the patch.
template <typename T>
__global__ void __launch_bounds__(kPB) k_piso_windkessel(int ni, const int* pstart, const int* psize,
                                                         int scheme, double dt, const T* phi,
                                                         T* pb, double* wk, double* Qout,
                                                         double* pout) {
  const int o = blockIdx.x;
  const int s = pstart[o], z = psize[o];
  double acc = 0.0;
  for (int k = threadIdx.x; k < z; k += blockDim.x) acc += (double)phi[s + k];
  __shared__ double sm[kPB / 32];
  __shared__ double po_sh;
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double Q = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) Q += sm[k];
    double pc = wk[4 * o + 3], po;
    wk_step(scheme, wk[4 * o], wk[4 * o + 1], wk[4 * o + 2], Q, dt, pc, po);
    wk[4 * o + 3] = pc;
    Qout[o] = Q;
    pout[o] = po;
    po_sh = po;
  }
  __syncthreads();
  const T po = (T)po_sh;
  for (int k = threadIdx.x; k < z; k += blockDim.x) pb[s + k - ni] = po;
}

// Limited explicit non-orthogonal correction: capped at psi/(1-psi) times the
// magnitude of the face's orthogonal part; psi outside (0,1) means unlimited.
template <typename T>
__device__ __forceinline__ T limit_corr(T corr, T orth, T psi) {
  if (!(psi > T(0) && psi < T(1))) return corr;
  const T cap = psi / (T(1) - psi) * fabs(orth);
  return fabs(corr) > cap ? (corr > T(0) ? cap : -cap) : corr;
}

// -------------------------------------------------------------- momentum
// internal faces: Up = min(m,0) - nu c (row O, col N), Lo = -max(m,0) - nu c (row N, col O)
template <typename T>
__global__ void k_mom_faces(int ni, Geo<T> g, T nu, const T* phi, T* Lo, T* Up) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= ni) return;
  const T m = phi[f];
  const T a = nu * ld4(g.ck + f).x;
  Up[f] = fmin(m, T(0)) - a;
  Lo[f] = -fmax(m, T(0)) - a;
}

// cells: D = V/dt + sum over faces; b = V/dt U^n + sigma nu (gradU)_f.k + boundary;
// rhs = b - V grad p
template <typename T, bool NONORTH>
__global__ void __launch_bounds__(kPB) k_mom_cells(Topo t, Geo<T> g, T nu, T rdt, T psi, const T* phi,
                                                   const T* U, const T* Ub, const T* gradU,
                                                   const T* gradp, T* D, T* b, T* rhs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc, nb = t.nb;
  const T V = g.V[i];
  T d = V * rdt;
  T bc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) bc[c] = V * rdt * U[c * nc + i];
  T gi[3][3];
  if (NONORTH)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) gi[c][k] = gradU[(c * 3 + k) * nc + i];
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e];
    const int f = ent >> 1;
    const T m = phi[f];
    const V4<T> ck = ld4(g.ck + f);
    const T a = nu * ck.x;
    if (f < t.ni) {
      const bool nside = ent & 1;
      d += (nside ? fmax(-m, T(0)) : fmax(m, T(0))) + a;
      if (NONORTH) {
        const int2 on = t.on[f];
        const int j = nside ? on.x : on.y;
        const T w = ld4(g.Sw + f).w;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T gf[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const T gj = gradU[(c * 3 + k) * nc + j];
            const T gO = nside ? gj : gi[c][k], gN = nside ? gi[c][k] : gj;
            gf[k] = w * gO + (T(1) - w) * gN;
          }
          const T uj = U[c * nc + j], ui = U[c * nc + i];
          const T orth = ck.x * (nside ? ui - uj : uj - ui);
          const T corr = nu * limit_corr(gf[0] * ck.y + gf[1] * ck.z + gf[2] * ck.w, orth, psi);
          bc[c] += nside ? -corr : corr;
        }
      }
    } else {
      const int bb = f - t.ni;
      const int kind = face_kind(t, bb, DIFVM_BC_VELOCITY);
      if (kind == DIFVM_FACE_FIXED) {
        d += a;
#pragma unroll
        for (int c = 0; c < 3; ++c) bc[c] += (a - m) * Ub[c * nb + bb];
      } else if (kind == DIFVM_FACE_ZEROGRAD) {
        d += m;
      }
    }
  }
  D[i] = d;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    b[c * nc + i] = bc[c];
    rhs[c * nc + i] = bc[c] - V * gradp[c * nc + i];
  }
}

// HbyA = (b - sum offdiag U)/D,  rAU = V/D   (Eq. Ap_H)
template <typename T>
__global__ void __launch_bounds__(kPB) k_HbyA(Topo t, Geo<T> g, const T* D, const T* Lo,
                                              const T* Up, const T* b, const T* U, T* HbyA, T* rAU) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc;
  T h[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) h[c] = b[c * nc + i];
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e];
    const int f = ent >> 1;
    if (f >= t.ni) break;
    const int2 on = t.on[f];
    const bool nside = ent & 1;
    const int j = nside ? on.x : on.y;
    const T a = nside ? Lo[f] : Up[f];
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] -= a * U[c * nc + j];
  }
  const T di = D[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) HbyA[c * nc + i] = h[c] / di;
  rAU[i] = g.V[i] / di;
}

// ---------------------------------------------------------------- pressure
// per face: phiHbyA, a_f = rAU_f c_f, nonorth_f = rAU_f (grad p)_f . k_f, Lp = -a_f
template <typename T, bool NONORTH>
__global__ void k_p_faces(Topo t, Geo<T> g, T psi, const T* HbyA, const T* rAU, const T* Ub,
                          const T* gradp, const T* p, T* phiHbyA, T* af, T* nonorth, T* Lp) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nf) return;
  const int nc = t.nc, nb = t.nb;
  const V4<T> s = ld4(g.Sw + f);
  const V4<T> ck = ld4(g.ck + f);
  if (f < t.ni) {
    const int2 on = t.on[f];
    const int O = on.x, N = on.y;
    const T w = s.w;
    T hf[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) hf[c] = w * HbyA[c * nc + O] + (T(1) - w) * HbyA[c * nc + N];
    phiHbyA[f] = hf[0] * s.x + hf[1] * s.y + hf[2] * s.z;
    const T rf = w * rAU[O] + (T(1) - w) * rAU[N];
    const T a = rf * ck.x;
    af[f] = a;
    Lp[f] = -a;
    T no = T(0);
    if (NONORTH) {
      T gf[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) gf[k] = w * gradp[k * nc + O] + (T(1) - w) * gradp[k * nc + N];
      no = rf * limit_corr(gf[0] * ck.y + gf[1] * ck.z + gf[2] * ck.w, ck.x * (p[N] - p[O]), psi);
    }
    nonorth[f] = no;
  } else {
    const int bb = f - t.ni;
    const int O = t.bown[bb];
    const int ku = face_kind(t, bb, DIFVM_BC_VELOCITY);
    const int kp = face_kind(t, bb, DIFVM_BC_PRESSURE);
    T ph = T(0), a = T(0);
    if (ku == DIFVM_FACE_FIXED) {
      ph = Ub[bb] * s.x + Ub[nb + bb] * s.y + Ub[2 * nb + bb] * s.z;
    } else if (ku == DIFVM_FACE_ZEROGRAD) {
      ph = HbyA[O] * s.x + HbyA[nc + O] * s.y + HbyA[2 * nc + O] * s.z;
    }
    if (ku != DIFVM_FACE_EMPTY && kp == DIFVM_FACE_FIXED) a = rAU[O] * ck.x;
    phiHbyA[f] = ph;
    af[f] = a;
  }
}

// per cell: Dp = sum a_f, bp = sum sigma(-phiHbyA + nonorth) + sum_fixed a_f p_b; pinned cell
template <typename T>
__global__ void __launch_bounds__(kPB) k_p_cells(Topo t, const T* phiHbyA, const T* af,
                                                 const T* nonorth, const T* pb, int pin, T* Dp,
                                                 T* bp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  T d = T(0), r = T(0);
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e];
    const int f = ent >> 1;
    if (f < t.ni) {
      const T q = -phiHbyA[f] + nonorth[f];
      d += af[f];
      r += (ent & 1) ? -q : q;
    } else {
      const int bb = f - t.ni;
      r += -phiHbyA[f];
      if (face_kind(t, bb, DIFVM_BC_PRESSURE) == DIFVM_FACE_FIXED &&
          face_kind(t, bb, DIFVM_BC_VELOCITY) != DIFVM_FACE_EMPTY) {
        d += af[f];
        r += af[f] * pb[bb];
      }
    }
  }
  if (i == pin) d += d;  // p_ref = 0 at the pinned cell (all-Neumann pressure)
  Dp[i] = d;
  bp[i] = r;
}

// Rhie-Chow flux correction: phi = phiHbyA - a_f dp - nonorth
template <typename T>
__global__ void k_flux_correct(Topo t, const T* phiHbyA, const T* af, const T* nonorth,
                               const T* p, const T* pb, T* phi) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nf) return;
  if (f < t.ni) {
    const int2 on = t.on[f];
    phi[f] = phiHbyA[f] - af[f] * (p[on.y] - p[on.x]) - nonorth[f];
  } else {
    const int bb = f - t.ni;
    if (face_kind(t, bb, DIFVM_BC_PRESSURE) == DIFVM_FACE_FIXED &&
        face_kind(t, bb, DIFVM_BC_VELOCITY) != DIFVM_FACE_EMPTY)
      phi[f] = phiHbyA[f] - af[f] * (pb[bb] - p[t.bown[bb]]);
    else
      phi[f] = phiHbyA[f];
  }
}

// U = HbyA - rAU grad p
template <typename T>
__global__ void k_U_correct(int nc, const T* HbyA, const T* rAU, const T* gradp, T* U) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const T r = rAU[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) U[c * nc + i] = HbyA[c * nc + i] - r * gradp[c * nc + i];
}

// phi_f = U_f . S_f (linear), boundary U_b.S / U_O.S / 0
template <typename T>
__global__ void k_flux_from_U(Topo t, Geo<T> g, const T* U, const T* Ub, T* phi) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nf) return;
  const int nc = t.nc, nb = t.nb;
  const V4<T> s = ld4(g.Sw + f);
  T u[3];
  if (f < t.ni) {
    const int2 on = t.on[f];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = s.w * U[c * nc + on.x] + (T(1) - s.w) * U[c * nc + on.y];
  } else {
    const int bb = f - t.ni;
    const int kind = face_kind(t, bb, DIFVM_BC_VELOCITY);
    if (kind == DIFVM_FACE_EMPTY) { phi[f] = T(0); return; }
    const int O = t.bown[bb];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = kind == DIFVM_FACE_FIXED ? Ub[c * nb + bb] : U[c * nc + O];
  }
  phi[f] = u[0] * s.x + u[1] * s.y + u[2] * s.z;
}

template <typename T> __global__ void k_to64(int n, const T* a, double* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
template <typename T> __global__ void k_from64(int n, const double* a, T* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

__global__ void k_piso_info(const difvm_solve_info* si, int ncorr, int status, int n_out,
                            const double* Q, const double* po, difvm_piso_info* out) {
  if (threadIdx.x != 0) return;
  difvm_piso_info r;
  for (int c = 0; c < 3; ++c) r.itU[c] = si[c].iters;
  for (int k = 0; k < 4; ++k) r.itp[k] = k < ncorr ? si[3 + k].iters : 0;
  int st = status;
  for (int c = 0; c < 3 + (ncorr < 4 ? ncorr : 4); ++c) st = st > si[c].status ? st : si[c].status;
  r.status = st;
  r.pad = 0;
  for (int k = 0; k < 16; ++k) {
    r.Q[k] = k < n_out ? Q[k] : 0.0;
    r.p_out[k] = k < n_out ? po[k] : 0.0;
  }
  *out = r;
}

// ---------------------------------------------------------------- driver
template <typename T>
static difvm_status piso_step_t(difvm_piso* h, T* U, T* p, T* phi, const T* Ub, T* pb, double* wk,
                                difvm_piso_info* info, cudaStream_t st) {
  difvm_mesh* m = h->m;
  const int nc = m->nc, ni = m->ni, nf = m->nf;
  const difvm_piso_opts& o = h->o;
  Topo t = m->topo();
  Geo<T> g = geo<T>(m);
  const unsigned Bc = blocks_for(nc, kPB), Bf = blocks_for(nf, kPB), Bi = blocks_for(std::max(ni, 1), kPB);
  T *gradp = (T*)h->gradp, *gradU = (T*)h->gradU, *D = (T*)h->D, *Lo = (T*)h->Lo, *Up = (T*)h->Up;
  T *b = (T*)h->b, *rhs = (T*)h->rhs, *rAU = (T*)h->rAU, *HbyA = (T*)h->HbyA, *Dp = (T*)h->Dp;
  T *Lp = (T*)h->Lp, *bp = (T*)h->bp, *phiH = (T*)h->phiHbyA, *af = (T*)h->af;
  T* no = (T*)h->nonorth;
  // scratch for Windkessel outputs: inside the solve-info buffer tail
  double* Qd = (double*)(h->sinfo + 8);
  double* pod = Qd + 16;
  int worst = DIFVM_OK;
  // 1. Windkessel outlets
  if (o.n_out > 0) {
    if (!wk) return set_error(DIFVM_EINVAL, "Windkessel outlets need the wk state array");
    // patch starts/sizes of the outlets live in a small device table after Qd/pod
    int* tab = (int*)(pod + 16);
    k_piso_windkessel<T><<<o.n_out, kPB, 0, st>>>(ni, tab, tab + 16, o.wk_scheme, o.dt, phi, pb, wk,
                                                    Qd, pod);
    DIFVM_TRY(check_launch("piso_windkessel"));
  }
  // 2. momentum predictor
  DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_PRESSURE, p, pb, 1, gradp, st));
  const bool no_U = (o.nonorth & DIFVM_NONORTH_MOMENTUM) != 0;
  const bool no_p = (o.nonorth & DIFVM_NONORTH_PRESSURE) != 0;
  if (no_U) DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_VELOCITY, U, Ub, 3, gradU, st));
  if (ni > 0) {
    k_mom_faces<T><<<Bi, kPB, 0, st>>>(ni, g, (T)o.nu, phi, Lo, Up);
    DIFVM_TRY(check_launch("mom_faces"));
  }
  const T psi = (T)o.nonorth_limit;
  if (no_U)
    k_mom_cells<T, true><<<Bc, kPB, 0, st>>>(t, g, (T)o.nu, (T)(1.0 / o.dt), psi, phi, U, Ub, gradU, gradp, D, b, rhs);
  else
    k_mom_cells<T, false><<<Bc, kPB, 0, st>>>(t, g, (T)o.nu, (T)(1.0 / o.dt), psi, phi, U, Ub, gradU, gradp, D, b, rhs);
  DIFVM_TRY(check_launch("mom_cells"));
  {
    difvm_prec pr = sizeof(T) == 8 ? DIFVM_F64 : DIFVM_F32;
    difvm_status s = difvm_krylov_solve(m, pr, &o.solve_U, D, Lo, Up, rhs, U, 3, h->wsU, h->wsU_bytes,
                                        h->sinfo, st);
    if (s == DIFVM_EINVAL || s == DIFVM_ECUDA) return s;
    worst = std::max(worst, (int)s);
  }
  // 3. pressure correctors
  const int pin = h->has_fixed_p ? -1 : o.pref_cell;
  for (int corr = 0; corr < o.n_corr; ++corr) {
    k_HbyA<T><<<Bc, kPB, 0, st>>>(t, g, D, Lo, Up, b, U, HbyA, rAU);
    DIFVM_TRY(check_launch("HbyA"));
    if (no_p) {
      DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_PRESSURE, p, pb, 1, gradp, st));
      k_p_faces<T, true><<<Bf, kPB, 0, st>>>(t, g, psi, HbyA, rAU, Ub, gradp, p, phiH, af, no, Lp);
    } else {
      k_p_faces<T, false><<<Bf, kPB, 0, st>>>(t, g, psi, HbyA, rAU, Ub, gradp, p, phiH, af, no, Lp);
    }
    DIFVM_TRY(check_launch("p_faces"));
    k_p_cells<T><<<Bc, kPB, 0, st>>>(t, phiH, af, no, pb, pin, Dp, bp);
    DIFVM_TRY(check_launch("p_cells"));
    difvm_solve_info* si = h->sinfo + 3 + std::min(corr, 3);
    difvm_status s;
    if (h->mixed) {
      k_to64<T><<<Bc, kPB, 0, st>>>(nc, bp, h->b64);
      k_to64<T><<<Bc, kPB, 0, st>>>(nc, p, h->p64);
      DIFVM_TRY(check_launch("to64"));
      count_launch();
      s = difvm_krylov_solve_refine(m, &o.solve_p, (const float*)Dp, (const float*)Lp, nullptr,
                                    h->b64, h->p64, 1, h->wsp, h->wsp_bytes, si, st);
      k_from64<T><<<Bc, kPB, 0, st>>>(nc, h->p64, p);
      DIFVM_TRY(check_launch("from64"));
    } else {
      difvm_prec pr = sizeof(T) == 8 ? DIFVM_F64 : DIFVM_F32;
      s = difvm_krylov_solve(m, pr, &o.solve_p, Dp, Lp, nullptr, bp, p, 1, h->wsp, h->wsp_bytes, si, st);
    }
    if (s == DIFVM_EINVAL || s == DIFVM_ECUDA) return s;
    worst = std::max(worst, (int)s);
    k_flux_correct<T><<<Bf, kPB, 0, st>>>(t, phiH, af, no, p, pb, phi);
    DIFVM_TRY(check_launch("flux_correct"));
    DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_PRESSURE, p, pb, 1, gradp, st));
    k_U_correct<T><<<Bc, kPB, 0, st>>>(nc, HbyA, rAU, gradp, U);
    DIFVM_TRY(check_launch("U_correct"));
  }
  if (info) {
    k_piso_info<<<1, 32, 0, st>>>(h->sinfo, o.n_corr, DIFVM_OK, o.n_out, Qd, pod, info);
    DIFVM_TRY(check_launch("piso_info"));
  }
  return (difvm_status)worst;
}

}  // namespace difvm

using namespace difvm;

extern "C" difvm_status difvm_windkessel_update(int n, int scheme, const double* Rp, const double* C,
                                                const double* Rd, const double* Q, double dt,
                                                double* pc, double* po, void* stream) {
  if (n < 0 || (n > 0 && (!Rp || !C || !Rd || !Q || !pc)))
    return set_error(DIFVM_EINVAL, "bad Windkessel arguments");
  if (scheme < DIFVM_WK_EXACT || scheme > DIFVM_WK_BE)
    return set_error(DIFVM_EINVAL, "bad Windkessel scheme %d", scheme);
  if (n == 0) return DIFVM_OK;
  k_windkessel<<<blocks_for(n, 128), 128, 0, (cudaStream_t)stream>>>(n, scheme, Rp, C, Rd, Q, dt, pc, po);
  return check_launch("windkessel");
}

extern "C" difvm_status difvm_windkessel_update_bwd(int n, int scheme, const double* Rp,
                                                    const double* C, const double* Rd,
                                                    const double* Q, double dt, const double* pc_in,
                                                    const double* pcb, const double* pob,
                                                    double* pc_in_bar, double* Qb, double* Rpb,
                                                    double* Cb, double* Rdb, void* stream) {
  if (n < 0 || (n > 0 && (!Rp || !C || !Rd || !Q || !pc_in)))
    return set_error(DIFVM_EINVAL, "bad Windkessel arguments");
  if (scheme < DIFVM_WK_EXACT || scheme > DIFVM_WK_BE)
    return set_error(DIFVM_EINVAL, "bad Windkessel scheme %d", scheme);
  if (n == 0) return DIFVM_OK;
  k_windkessel_bwd<<<blocks_for(n, 128), 128, 0, (cudaStream_t)stream>>>(
      n, scheme, Rp, C, Rd, Q, dt, pc_in, pcb, pob, pc_in_bar, Qb, Rpb, Cb, Rdb);
  return check_launch("windkessel_bwd");
}

extern "C" difvm_status difvm_flux_from_U(difvm_mesh_t m, difvm_prec prec, const void* U,
                                          const void* Ub, void* phi, void* stream) {
  DIFVM_TRY(check_mesh(m));
  DIFVM_TRY(check_prec(prec));
  if (!U || !phi) return set_error(DIFVM_EINVAL, "null field");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == DIFVM_F64)
    k_flux_from_U<double><<<blocks_for(m->nf, kPB), kPB, 0, st>>>(m->topo(), m->geo64(),
                                                                  (const double*)U, (const double*)Ub, (double*)phi);
  else
    k_flux_from_U<float><<<blocks_for(m->nf, kPB), kPB, 0, st>>>(m->topo(), m->geo32(),
                                                                 (const float*)U, (const float*)Ub, (float*)phi);
  return check_launch("flux_from_U");
}

extern "C" void difvm_piso_destroy(difvm_piso_t h) {
  if (!h) return;
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

extern "C" difvm_status difvm_piso_create(difvm_mesh_t m, difvm_prec prec, const difvm_piso_opts* o,
                                          difvm_piso_t* out) {
  DIFVM_TRY(check_mesh(m));
  DIFVM_TRY(check_prec(prec));
  if (!o || !out) return set_error(DIFVM_EINVAL, "null argument");
  *out = nullptr;
  if (!(o->dt > 0) || !(o->nu >= 0)) return set_error(DIFVM_EINVAL, "need dt > 0 and nu >= 0");
  if (o->n_corr < 1 || o->n_corr > 8) return set_error(DIFVM_EINVAL, "n_corr must be 1..8");
  if (o->n_out < 0 || o->n_out > 16) return set_error(DIFVM_EINVAL, "n_out must be 0..16");
  if (o->solve_U.method != DIFVM_BICGSTAB && o->solve_U.method != DIFVM_PCG)
    return set_error(DIFVM_EINVAL, "bad momentum solver");
  if (o->solve_p.method != DIFVM_PCG && o->solve_p.method != DIFVM_BICGSTAB)
    return set_error(DIFVM_EINVAL, "bad pressure solver");
  for (int k = 0; k < o->n_out; ++k) {
    int p = o->wk_patch[k];
    if (p < 0 || p >= m->npatch || m->patch_type[p] != DIFVM_PATCH_OUTLET)
      return set_error(DIFVM_EINVAL, "Windkessel patch %d is not an OUTLET patch", p);
  }
  difvm_piso* h = new (std::nothrow) difvm_piso();
  if (!h) return set_error(DIFVM_ENOMEM, "host allocation failed");
  h->m = m;
  h->prec = prec;
  h->o = *o;
  h->mixed = prec == DIFVM_F32 && o->solve_p.refine_max > 0;
  h->elt = prec == DIFVM_F64 ? 8 : 4;
  for (int p = 0; p < m->npatch; ++p) h->has_fixed_p |= m->patch_type[p] == DIFVM_PATCH_OUTLET;
  if (!h->has_fixed_p && (o->pref_cell < 0 || o->pref_cell >= m->nc)) {
    delete h;
    return set_error(DIFVM_EINVAL, "pref_cell %d out of range (no patch fixes p)", o->pref_cell);
  }
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    h->allocs.push_back(*p);
    return true;
  };
  const size_t e = h->elt, nc = m->nc, ni = std::max(m->ni, 1), nf = m->nf;
  bool ok = alloc(&h->gradp, 3 * nc * e) && alloc(&h->gradU, 9 * nc * e) && alloc(&h->D, nc * e) &&
            alloc(&h->Lo, ni * e) && alloc(&h->Up, ni * e) && alloc(&h->b, 3 * nc * e) &&
            alloc(&h->rhs, 3 * nc * e) && alloc(&h->rAU, nc * e) && alloc(&h->HbyA, 3 * nc * e) &&
            alloc(&h->Dp, nc * e) && alloc(&h->Lp, ni * e) && alloc(&h->bp, nc * e) &&
            alloc(&h->phiHbyA, nf * e) && alloc(&h->af, nf * e) && alloc(&h->nonorth, ni * e);
  h->wsU_bytes = difvm_krylov_workspace_bytes(m, prec, o->solve_U.method, 3);
  ok = ok && alloc(&h->wsU, h->wsU_bytes);
  if (h->mixed) {
    h->wsp_bytes = difvm_krylov_refine_workspace_bytes(m, o->solve_p.method, 1);
    ok = ok && alloc((void**)&h->p64, nc * 8) && alloc((void**)&h->b64, nc * 8);
  } else {
    h->wsp_bytes = difvm_krylov_workspace_bytes(m, prec, o->solve_p.method, 1);
  }
  ok = ok && alloc(&h->wsp, h->wsp_bytes);
  // solve infos [8] + Q[16] + p_out[16] + outlet table (start[16], size[16])
  ok = ok && alloc((void**)&h->sinfo, 8 * sizeof(difvm_solve_info) + 32 * sizeof(double) + 32 * sizeof(int));
  if (!ok) {
    difvm_piso_destroy(h);
    return set_error(DIFVM_ENOMEM, "device allocation for the PISO workspace failed");
  }
  int tab[32] = {0};
  for (int k = 0; k < o->n_out; ++k) {
    tab[k] = m->patch_start[o->wk_patch[k]];
    tab[16 + k] = m->patch_size[o->wk_patch[k]];
  }
  double* Qd = (double*)(h->sinfo + 8);
  if (cudaMemcpy(Qd + 32, tab, sizeof tab, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(h->sinfo, 0, 8 * sizeof(difvm_solve_info) + 32 * sizeof(double)) != cudaSuccess) {
    difvm_piso_destroy(h);
    return set_error(DIFVM_ECUDA, "PISO table upload failed");
  }
  *out = h;
  return DIFVM_OK;
}

extern "C" difvm_status difvm_piso_step(difvm_piso_t h, void* U, void* p, void* phi, const void* Ub,
                                        void* pb, double* wk, difvm_piso_info* info, void* stream) {
  if (!h) return set_error(DIFVM_EINVAL, "null PISO handle");
  if (!U || !p || !phi) return set_error(DIFVM_EINVAL, "null state field");
  cudaStream_t st = (cudaStream_t)stream;
  if (h->prec == DIFVM_F64)
    return piso_step_t<double>(h, (double*)U, (double*)p, (double*)phi, (const double*)Ub,
                               (double*)pb, wk, info, st);
  return piso_step_t<float>(h, (float*)U, (float*)p, (float*)phi, (const float*)Ub, (float*)pb, wk,
                            info, st);
}
