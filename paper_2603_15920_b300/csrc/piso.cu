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
  int nk = 1;                      // cases (solve-info slots per solve)
  int pin = -1;                    // pinned cell of a single-case mesh
  unsigned char* pinflag = nullptr;  // batched mesh: 1 on each case's pinned cell
  size_t elt = 8;
  void *gradp = nullptr, *gradU = nullptr, *D = nullptr, *Lo = nullptr, *Up = nullptr, *b = nullptr;
  void *rhs = nullptr, *rAU = nullptr, *HbyA = nullptr, *Dp = nullptr, *Lp = nullptr, *bp = nullptr;
  void *phiHbyA = nullptr, *af = nullptr, *nonorth = nullptr;
  void* sou_d = nullptr;           // second-order upwind: V4<T> x_f - x_O [ni], then x_f - x_N [ni]
  // multigrid pressure solves: the operators of corrector 0 are built on a side
  // stream while the momentum predictor is solved (the pressure matrix needs only
  // V/D); rAU_e is that stream's copy of V/D
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void* rAU_e = nullptr;
  void* wsU = nullptr;
  size_t wsU_bytes = 0;
  void* wsp = nullptr;
  size_t wsp_bytes = 0;
  double *p64 = nullptr, *b64 = nullptr;
  // solve infos: momentum [3 nk] (case-major), then 4 pressure slots of [nk];
  // followed by Q[16], p_out[16] (double) and the outlet table (int start[16], size[16])
  difvm_solve_info* sinfo = nullptr;
  std::vector<void*> allocs;
  // adjoint workspace, allocated by the first difvm_piso_step_bwd
  bool adj_ready = false;
  void *a_HAb = nullptr, *a_gpb = nullptr, *a_gpn = nullptr, *a_rAUb = nullptr, *a_Db = nullptr;
  void *a_bb = nullptr, *a_Lob = nullptr, *a_Upb = nullptr, *a_lam = nullptr, *a_lamU = nullptr;
  void *a_phiHb = nullptr, *a_rfb = nullptr, *a_lk = nullptr, *a_ld = nullptr, *a_phio = nullptr;
  void *a_pbb = nullptr, *a_gUb = nullptr, *a_lkU = nullptr, *a_ldU = nullptr, *a_gp2 = nullptr;
  void* a_lsU = nullptr;           // second-order upwind: per face and component, t_bar m
  double *a_nuf = nullptr, *a_part = nullptr;
  // starting guesses of the adjoint pressure solves, one per corrector (FP64 on
  // mixed-precision handles): the previous reverse step's solutions
  void* a_lamw = nullptr;
  // CUDA-graph form of the step: one instantiated graph per argument set
  struct GraphEntry {
    const void* key[7];
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
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

// Partial derivatives of the new p_c of one RCR step with respect to the old
// p_c, Q, R_d and C (closed forms of the three updates).
__device__ __forceinline__ void wk_partials(int scheme, double C, double Rd, double Q, double dt,
                                            double p0, double& dp0, double& dq, double& drd,
                                            double& dc) {
  if (scheme == DIFVM_WK_EXACT) {
    const double e = exp(-dt / (Rd * C));
    dp0 = e;
    dq = Rd * (1.0 - e);
    const double de = p0 - Rd * Q;                 // d pc_out / d e
    drd = de * e * dt / (Rd * Rd * C) + Q * (1.0 - e);
    dc = de * e * dt / (Rd * C * C);
  } else if (scheme == DIFVM_WK_FE) {
    dp0 = 1.0 - dt / (Rd * C);
    dq = dt / C;
    drd = dt * p0 / (Rd * Rd * C);
    dc = -dt * (Q - p0 / Rd) / (C * C);
  } else {
    const double M = 1.0 + dt / (Rd * C), N = p0 + dt * Q / C;
    dp0 = 1.0 / M;
    dq = dt / (C * M);
    drd = N * dt / (M * M * Rd * Rd * C);
    dc = -dt * Q / (C * C * M) + N * dt / (M * M * Rd * C * C);
  }
}

// Adjoint of one RCR step (closed-form derivatives of the three updates).
__global__ void k_windkessel_bwd(int n, int scheme, const double* Rp, const double* C,
                                 const double* Rd, const double* Q, double dt, const double* pc_in,
                                 const double* pcb, const double* pob, double* pc_in_bar,
                                 double* Qb, double* Rpb, double* Cb, double* Rdb) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const double rp = Rp[o], q = Q[o];
  const double pob_ = pob ? pob[o] : 0.0;
  const double g = (pcb ? pcb[o] : 0.0) + pob_;
  double dp0, dq, drd, dc;
  wk_partials(scheme, C[o], Rd[o], q, dt, pc_in[o], dp0, dq, drd, dc);
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

// x_f - x_O and x_f - x_N of every internal face (second-order upwind reconstruction)
template <typename T>
__global__ void k_sou_d(int ni, const int2* on, const double* Cf, const double* C, V4<T>* d) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= ni) return;
  const int O = on[f].x, N = on[f].y;
  d[f] = V4<T>{(T)(Cf[3 * f] - C[3 * O]), (T)(Cf[3 * f + 1] - C[3 * O + 1]), (T)(Cf[3 * f + 2] - C[3 * O + 2]), T(0)};
  d[ni + f] = V4<T>{(T)(Cf[3 * f] - C[3 * N]), (T)(Cf[3 * f + 1] - C[3 * N + 1]),
                    (T)(Cf[3 * f + 2] - C[3 * N + 2]), T(0)};
}

// cells: D = V/dt + sum over faces; b = V/dt U^n + sigma nu (gradU)_f.k + boundary;
// rhs = b - V grad p.  SOU: second-order upwind by deferred correction (Eqs.
// deferred_correction, sou): each internal face moves t_f = m (gradU)_C . (x_f - x_C)
// of its upwind cell C (the owner when m >= 0) out of the owner's row into the
// neighbour's: b_O -= t_f, b_N += t_f.
template <typename T, bool NONORTH, bool SOU>
__global__ void __launch_bounds__(kPB) k_mom_cells(Topo t, Geo<T> g, T nu, T rdt, T psi, const T* phi,
                                                   const T* U, const T* Ub, const T* gradU,
                                                   const V4<T>* sd, const T* gradp, T* D, T* b, T* rhs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc, nb = t.nb;
  const T V = g.V[i];
  T d = V * rdt;
  T bc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) bc[c] = V * rdt * U[c * nc + i];
  T gi[3][3];
  if (NONORTH || SOU)
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
      if (NONORTH || SOU) {
        const int2 on = t.on[f];
        const int j = nside ? on.x : on.y;
        const bool upO = m >= T(0);             // the owner is the upwind cell
        const bool up_self = upO != nside;      // this cell is the upwind cell
        T gj[3][3];
        if (NONORTH || !up_self)
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < 3; ++k) gj[c][k] = gradU[(c * 3 + k) * nc + j];
        if (NONORTH) {
          const T w = ld4(g.Sw + f).w;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            T gf[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const T gO = nside ? gj[c][k] : gi[c][k], gN = nside ? gi[c][k] : gj[c][k];
              gf[k] = w * gO + (T(1) - w) * gN;
            }
            const T uj = U[c * nc + j], ui = U[c * nc + i];
            const T orth = ck.x * (nside ? ui - uj : uj - ui);
            const T corr = nu * limit_corr(gf[0] * ck.y + gf[1] * ck.z + gf[2] * ck.w, orth, psi);
            bc[c] += nside ? -corr : corr;
          }
        }
        if (SOU) {
          const V4<T> dc = ld4(sd + (upO ? f : t.ni + f));
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const T* gC = up_self ? gi[c] : gj[c];
            const T tf = m * (gC[0] * dc.x + gC[1] * dc.y + gC[2] * dc.z);
            bc[c] += nside ? tf : -tf;
          }
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

// Crank-Nicolson form of the momentum rows: with the backward-Euler rows
// D = V/dt + D_cd, Lo/Up and b = V/dt U^n + b_cd, average the spatial operator
// over the two time levels: D <- V/dt + D_cd/2, b and rhs -= (A_cd U^n)/2 (the
// off-diagonals are halved afterwards by k_cn_faces, so they are read whole here).
template <typename T>
__global__ void __launch_bounds__(kPB) k_cn_cells(Topo t, Geo<T> g, T rdt, const T* Lo, const T* Up,
                                                  const T* U, T* D, T* b, T* rhs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc;
  const T Vdt = g.V[i] * rdt, Dcd = D[i] - Vdt;
  T a[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) a[c] = Dcd * U[c * nc + i];
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e];
    const int f = ent >> 1;
    if (f >= t.ni) break;
    const int2 on = t.on[f];
    const bool nside = ent & 1;
    const T coef = nside ? Lo[f] : Up[f];   // row N holds Lo_f U_O, row O holds Up_f U_N
    const int j = nside ? on.x : on.y;
#pragma unroll
    for (int c = 0; c < 3; ++c) a[c] += coef * U[c * nc + j];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    b[c * nc + i] -= T(0.5) * a[c];
    rhs[c * nc + i] -= T(0.5) * a[c];
  }
  D[i] = Vdt + T(0.5) * Dcd;
}
template <typename T>
__global__ void k_cn_faces(int ni, T* Lo, T* Up) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= ni) return;
  Lo[f] *= T(0.5);
  Up[f] *= T(0.5);
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
                                                 const T* nonorth, const T* pb, int pin,
                                                 const unsigned char* pinflag, T* Dp,
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
  // p_ref = 0 at the pinned cell (all-Neumann pressure)
  if (pinflag ? pinflag[i] != 0 : i == pin) d += d;
  Dp[i] = d;
  bp[i] = r;
}

// The pressure matrix alone (the same arithmetic as k_HbyA's rAU, k_p_faces' a_f,
// Lp and k_p_cells' Dp, so the values are identical): rAU = V/D, a_f, Lp = -a_f
template <typename T>
__global__ void k_p_rau(int nc, Geo<T> g, const T* D, T* rAU) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  rAU[i] = g.V[i] / D[i];
}
template <typename T>
__global__ void k_p_matrix(Topo t, Geo<T> g, const T* rAU, T* af, T* Lp) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nf) return;
  const V4<T> ck = ld4(g.ck + f);
  if (f < t.ni) {
    const int2 on = t.on[f];
    const T w = ld4(g.Sw + f).w;
    const T rf = w * rAU[on.x] + (T(1) - w) * rAU[on.y];
    const T a = rf * ck.x;
    af[f] = a;
    Lp[f] = -a;
  } else {
    const int bb = f - t.ni;
    const int ku = face_kind(t, bb, DIFVM_BC_VELOCITY);
    const int kp = face_kind(t, bb, DIFVM_BC_PRESSURE);
    af[f] = (ku != DIFVM_FACE_EMPTY && kp == DIFVM_FACE_FIXED) ? rAU[t.bown[bb]] * ck.x : T(0);
  }
}
template <typename T>
__global__ void __launch_bounds__(kPB) k_p_diag(Topo t, const T* af, int pin, const unsigned char* pinflag,
                                                T* Dp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  T d = T(0);
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int f = t.cent[e] >> 1;
    if (f < t.ni) {
      d += af[f];
    } else {
      const int bb = f - t.ni;
      if (face_kind(t, bb, DIFVM_BC_PRESSURE) == DIFVM_FACE_FIXED &&
          face_kind(t, bb, DIFVM_BC_VELOCITY) != DIFVM_FACE_EMPTY)
        d += af[f];
    }
  }
  if (pinflag ? pinflag[i] != 0 : i == pin) d += d;
  Dp[i] = d;
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

// Step record: per solve the largest iteration count over the cases, the
// worst status over all solves and cases, and the outlet values.
__global__ void k_piso_info(const difvm_solve_info* si, int nk, int ncorr, int status, int n_out,
                            const double* Q, const double* po, difvm_piso_info* out) {
  if (threadIdx.x != 0) return;
  difvm_piso_info r;
  int st = status;
  for (int c = 0; c < 3; ++c) {
    int it = 0;
    for (int k = 0; k < nk; ++k) {
      it = max(it, si[k * 3 + c].iters);
      st = max(st, si[k * 3 + c].status);
    }
    r.itU[c] = it;
  }
  for (int q = 0; q < 4; ++q) {
    int it = 0;
    if (q < ncorr)
      for (int k = 0; k < nk; ++k) {
        it = max(it, si[(3 + q) * nk + k].iters);
        st = max(st, si[(3 + q) * nk + k].status);
      }
    r.itp[q] = it;
  }
  r.status = st;
  r.pad = 0;
  for (int k = 0; k < 16; ++k) {
    r.Q[k] = k < n_out ? Q[k] : 0.0;
    r.p_out[k] = k < n_out ? po[k] : 0.0;
  }
  *out = r;
}

// ---------------------------------------------------------------- adjoint
// Reverse sweep of one PISO step (Sec. 2.5, Eqs. vjp, implicit_diff).  Face
// kernels compute each face's adjoint message once; cell kernels gather those
// messages over the cell-CSR rows in ascending face order, so every sum has a
// fixed order (no atomics, bitwise reproducible).  Non-smooth switches (upwind
// max(m, 0), the limiter) take the derivative of the branch the forward step
// took.

// Derivative of limit_corr(corr, orth, psi): returns d/dcorr, writes d/dorth.
template <typename T>
__device__ __forceinline__ T limit_corr_d(T corr, T orth, T psi, T& dorth) {
  dorth = T(0);
  if (!(psi > T(0) && psi < T(1))) return T(1);
  const T r = psi / (T(1) - psi);
  if (fabs(corr) > r * fabs(orth)) {
    const T so = orth > T(0) ? T(1) : (orth < T(0) ? T(-1) : T(0));
    dorth = (corr > T(0) ? r : -r) * so;
    return T(0);
  }
  return T(1);
}

// U_{s+1} = HbyA_s - rAU grad p_{s+1}:  HbyA_bar = U_bar, rAU_bar -= U_bar . grad p,
// (grad p_{s+1})_bar = gpn - rAU U_bar   (gpn: that gradient's use in the next corrector)
template <typename T>
__global__ void k_adj_Ucorr(int nc, const T* Ub_, const T* gradp, const T* rAU, const T* gpn,
                            T* HAb, T* rAUb, T* gpb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const T r = rAU[i];
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T u = Ub_[c * nc + i];
    HAb[c * nc + i] = u;
    acc += u * gradp[c * nc + i];
    gpb[c * nc + i] = gpn[c * nc + i] - r * u;
  }
  rAUb[i] -= acc;
}

// Rhie-Chow flux of the last corrector: p_bar_i += sum sigma a_f phi_bar_f; fixed-p
// boundary faces also move -a_f phi_bar_f to p_b.
template <typename T>
__global__ void __launch_bounds__(kPB) k_adj_flux_cells(Topo t, const T* af, const T* phio,
                                                        T* pbar, T* pbb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  T acc = T(0);
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e];
    const int f = ent >> 1;
    const T g = af[f] * phio[f];
    if (f < t.ni) {
      acc += (ent & 1) ? -g : g;
    } else {
      const int bb = f - t.ni;
      if (face_kind(t, bb, DIFVM_BC_PRESSURE) == DIFVM_FACE_FIXED &&
          face_kind(t, bb, DIFVM_BC_VELOCITY) != DIFVM_FACE_EMPTY) {
        acc += g;
        pbb[bb] -= g;
      }
    }
  }
  pbar[i] += acc;
}

// Pressure solve and assembly of corrector s, per face.  lam = A_p^{-1} p_bar_{s+1};
// coefficient adjoints Dp_bar_i = -lam_i p_i (times 2 at the pinned cell),
// Lp_bar_f = -(lam_O p_N + lam_N p_O) are folded into a_f_bar; bp_bar = lam gives
// phiHbyA_bar and nonorth_bar.  Then k_p_faces backwards: phiHb (the face's
// phiHbyA adjoint), rfb (adjoint of the interpolated rAU_f, or of rAU_O on a
// fixed-p boundary face), lk / ld (limited non-orthogonal term: weight of the
// interpolated grad p_s . k_f, and of p_s,N - p_s,O).
template <typename T, bool NONORTH, bool LAST>
__global__ void k_adj_pfaces(Topo t, Geo<T> g, T psi, int pin, const unsigned char* pinflag,
                             const T* lam, const T* pn,
                             const T* pk, const T* gk, const T* rAU, const T* af, const T* pb,
                             const T* phio, T* phiHb, T* rfb, T* lk, T* ld, T* pbb, T* Ubb) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nf) return;
  const int nc = t.nc, nb = t.nb;
  const V4<T> ck = ld4(g.ck + f);
  if (f < t.ni) {
    const int2 on = t.on[f];
    const int O = on.x, N = on.y;
    const T lO = lam[O], lN = lam[N], pO = pn[O], pN = pn[N];
    const T mO = (pinflag ? pinflag[O] != 0 : O == pin) ? T(2) : T(1);
    const T mN = (pinflag ? pinflag[N] != 0 : N == pin) ? T(2) : T(1);
    T afb = lO * pN + lN * pO - lO * pO * mO - lN * pN * mN;
    const T qb = lO - lN;
    T phb = -qb, nob = qb;
    if (LAST) {
      const T gg = phio[f];
      phb += gg;
      afb -= gg * (pN - pO);
      nob -= gg;
    }
    const T w = ld4(g.Sw + f).w;
    T r = afb * ck.x;
    if (NONORTH) {
      const T rf = w * rAU[O] + (T(1) - w) * rAU[N];
      T gf[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) gf[k] = w * gk[k * nc + O] + (T(1) - w) * gk[k * nc + N];
      const T corr = gf[0] * ck.y + gf[1] * ck.z + gf[2] * ck.w;
      const T orth = ck.x * (pk[N] - pk[O]);
      r += nob * limit_corr(corr, orth, psi);
      T dorth;
      const T dcorr = limit_corr_d(corr, orth, psi, dorth);
      const T lb = nob * rf;
      lk[f] = lb * dcorr;
      ld[f] = lb * dorth * ck.x;
    }
    phiHb[f] = phb;
    rfb[f] = r;
  } else {
    const int bb = f - t.ni;
    const int O = t.bown[bb];
    const int ku = face_kind(t, bb, DIFVM_BC_VELOCITY);
    if (ku == DIFVM_FACE_EMPTY) {
      phiHb[f] = T(0);
      rfb[f] = T(0);
      return;
    }
    const T lO = lam[O];
    T phb = -lO;
    if (LAST) phb += phio[f];
    T r = T(0);
    if (face_kind(t, bb, DIFVM_BC_PRESSURE) == DIFVM_FACE_FIXED) {
      const T pO = pn[O], mO = (pinflag ? pinflag[O] != 0 : O == pin) ? T(2) : T(1);
      T afb = lO * pb[bb] - lO * pO * mO;
      if (LAST) afb -= phio[f] * (pb[bb] - pO);
      pbb[bb] += lO * af[f];
      r = afb * ck.x;
    }
    if (ku == DIFVM_FACE_FIXED && Ubb) {
      const V4<T> s = ld4(g.Sw + f);
      Ubb[bb] += phb * s.x;
      Ubb[nb + bb] += phb * s.y;
      Ubb[2 * nb + bb] += phb * s.z;
    }
    phiHb[f] = phb;
    rfb[f] = r;
  }
}

// Gather of k_adj_pfaces: HbyA_bar and rAU_bar of corrector s, the adjoint of
// grad p_s from its non-orthogonal use (overwrites gpn), limiter terms into p_bar_s.
template <typename T, bool NONORTH>
__global__ void __launch_bounds__(kPB) k_adj_pcells(Topo t, Geo<T> g, const T* phiHb,
                                                    const T* rfb, const T* lk, const T* ld, T* HAb,
                                                    T* rAUb, T* gpn, T* pbar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc;
  T h[3], gacc[3] = {T(0), T(0), T(0)}, r = T(0), pacc = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) h[c] = HAb[c * nc + i];
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e];
    const int f = ent >> 1;
    const V4<T> s = ld4(g.Sw + f);
    const T ph = phiHb[f];
    if (f < t.ni) {
      const bool nside = ent & 1;
      const T wi = nside ? T(1) - s.w : s.w;
      h[0] += wi * ph * s.x;
      h[1] += wi * ph * s.y;
      h[2] += wi * ph * s.z;
      r += wi * rfb[f];
      if (NONORTH) {
        const V4<T> ck = ld4(g.ck + f);
        const T l = wi * lk[f];
        gacc[0] += l * ck.y;
        gacc[1] += l * ck.z;
        gacc[2] += l * ck.w;
        pacc += nside ? ld[f] : -ld[f];
      }
    } else {
      const int bb = f - t.ni;
      const int ku = face_kind(t, bb, DIFVM_BC_VELOCITY);
      if (ku == DIFVM_FACE_EMPTY) continue;
      if (ku == DIFVM_FACE_ZEROGRAD) {
        h[0] += ph * s.x;
        h[1] += ph * s.y;
        h[2] += ph * s.z;
      }
      r += rfb[f];
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) HAb[c * nc + i] = h[c];
  rAUb[i] += r;
  if (NONORTH) {
#pragma unroll
    for (int c = 0; c < 3; ++c) gpn[c * nc + i] = gacc[c];
    pbar[i] += pacc;
  }
}

// HbyA_s = (b - N U_s)/D backwards: D_bar -= h_bar . HbyA, b_bar += h_bar,
// U_bar_s = -N^T h_bar (overwritten), h_bar = HbyA_bar / D.
template <typename T>
__global__ void __launch_bounds__(kPB) k_adj_HbyA(Topo t, const T* D, const T* Lo, const T* Up,
                                                  const T* b, const T* Us, const T* HAb, T* Db,
                                                  T* bb, T* Ubar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc;
  T h[3], u[3] = {T(0), T(0), T(0)};
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
    const T a = nside ? Lo[f] : Up[f];     // row i, column j
    const T aT = nside ? Up[f] : Lo[f];    // row j, column i
    const T rDj = T(1) / D[j];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h[c] -= a * Us[c * nc + j];
      u[c] -= aT * (HAb[c * nc + j] * rDj);
    }
  }
  const T di = D[i];
  T dacc = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T hb = HAb[c * nc + i] / di;
    dacc += hb * (h[c] / di);
    bb[c * nc + i] += hb;
    Ubar[c * nc + i] = u[c];
  }
  Db[i] -= dacc;
}

// Off-diagonal coefficient adjoints of the HbyA products: Up_bar_f -= h_bar_O . U_s,N,
// Lo_bar_f -= h_bar_N . U_s,O.
template <typename T>
__global__ void k_adj_LU(int ni, int nc, const int2* on, const T* D, const T* HAb, const T* Us,
                         T* Lob, T* Upb) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= ni) return;
  const int2 o = on[f];
  const T rO = T(1) / D[o.x], rN = T(1) / D[o.y];
  T su = T(0), sl = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    su += HAb[c * nc + o.x] * rO * Us[c * nc + o.y];
    sl += HAb[c * nc + o.y] * rN * Us[c * nc + o.x];
  }
  Upb[f] -= su;
  Lob[f] -= sl;
}

// Momentum predictor backwards, per cell: lamU = A^{-T} U_bar_0;  D_bar gets the
// solve term and rAU = V/D; b_bar += lamU; (grad p^n)_bar -= V lamU; then
// U_bar^n = V/dt b_bar (overwrites U_bar).
template <typename T>
__global__ void k_adj_mom_cells(int nc, Geo<T> g, T rdt, const T* D, const T* lamU,
                                const T* Ustar, const T* rAUb, T* Db, T* bb, T* gpn, T* Ubar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const T V = g.V[i], di = D[i];
  T d = Db[i] - rAUb[i] * V / (di * di);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T l = lamU[c * nc + i];
    d -= l * Ustar[c * nc + i];
    const T bv = bb[c * nc + i] + l;
    bb[c * nc + i] = bv;
    gpn[c * nc + i] -= V * l;
    Ubar[c * nc + i] = V * rdt * bv;
  }
  Db[i] = d;
}

// Crank-Nicolson rows backwards, per cell (D, Lo, Up hold the halved rows; the
// backward-Euler coefficients are D_cd = 2 (D - V/dt), 2 Lo, 2 Up):
//   D_bar <- D_bar/2 - sum_c b_bar U^n / 2,  U^n_bar -= (A_cd^T b_bar)/2.
template <typename T>
__global__ void __launch_bounds__(kPB) k_adj_cn_cells(Topo t, Geo<T> g, T rdt, const T* D, const T* Lo,
                                                      const T* Up, const T* U0, const T* bb, T* Db,
                                                      T* Ubar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc;
  const T Dcd = T(2) * (D[i] - g.V[i] * rdt);
  T s = T(0), a[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T bi = bb[c * nc + i];
    s += bi * U0[c * nc + i];
    a[c] = Dcd * bi;
  }
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e];
    const int f = ent >> 1;
    if (f >= t.ni) break;
    const int2 on = t.on[f];
    const bool nside = ent & 1;
    // U_i enters row N through Lo_f when i is the owner, row O through Up_f when i is the neighbour
    const T coef = T(2) * (nside ? Up[f] : Lo[f]);
    const int j = nside ? on.x : on.y;
#pragma unroll
    for (int c = 0; c < 3; ++c) a[c] += coef * bb[c * nc + j];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) Ubar[c * nc + i] -= T(0.5) * a[c];
  Db[i] = T(0.5) * Db[i] - T(0.5) * s;
}

// Momentum assembly backwards, per face: the face flux adjoint (upwind switch),
// the viscosity adjoint contribution (FP64, reduced later in a fixed order), the
// limited non-orthogonal correction (lkU / ldU per component), U_b_bar.
template <typename T, bool NONORTH, bool SOU>
__global__ void k_adj_mom_faces(Topo t, Geo<T> g, T nu, T psi, const T* phi0, const T* Db,
                                const T* bb, const T* Lob, const T* Upb, const T* lamU,
                                const T* Ustar, const T* U0, const T* gradU, const T* Ub, T* phib,
                                double* nuf, T* lkU, T* ldU, const V4<T>* sd, T* lsU, T* Ubb, int cn) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nf) return;
  const int nc = t.nc, nb = t.nb, ni = t.ni;
  const T m = phi0[f];
  const V4<T> ck = ld4(g.ck + f);
  if (f < ni) {
    const int2 on = t.on[f];
    const int O = on.x, N = on.y;
    T upt = Upb[f], lot = Lob[f];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      upt -= lamU[c * nc + O] * Ustar[c * nc + N];
      lot -= lamU[c * nc + N] * Ustar[c * nc + O];
    }
    if (cn) {   // Crank-Nicolson rows: halved coefficients and -A_cd U^n / 2 in b
      T su = T(0), sl = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        su += bb[c * nc + O] * U0[c * nc + N];
        sl += bb[c * nc + N] * U0[c * nc + O];
      }
      upt = T(0.5) * upt - T(0.5) * su;
      lot = T(0.5) * lot - T(0.5) * sl;
    }
    const T dO = Db[O], dN = Db[N];
    const bool hp = m > T(0), hn = m < T(0);
    phib[f] = (hp ? dO - lot : T(0)) + (hn ? upt - dN : T(0));
    double nv = (double)(ck.x * (dO + dN - upt - lot));
    if (NONORTH) {
      const T w = ld4(g.Sw + f).w;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T gf[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
          gf[k] = w * gradU[(c * 3 + k) * nc + O] + (T(1) - w) * gradU[(c * 3 + k) * nc + N];
        const T corr = gf[0] * ck.y + gf[1] * ck.z + gf[2] * ck.w;
        const T orth = ck.x * (U0[c * nc + N] - U0[c * nc + O]);
        const T cb = bb[c * nc + O] - bb[c * nc + N];
        nv += (double)(cb * limit_corr(corr, orth, psi));
        T dorth;
        const T dcorr = limit_corr_d(corr, orth, psi, dorth);
        const T lb = nu * cb;
        lkU[c * ni + f] = lb * dcorr;
        ldU[c * ni + f] = lb * dorth * ck.x;
      }
    }
    if (SOU) {   // t_f = m (gradU)_C . d_Cf enters b_O with -1 and b_N with +1
      const bool upO = m >= T(0);
      const int Cu = upO ? O : N;
      const V4<T> dc = ld4(sd + (upO ? f : ni + f));
      T mb = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T tb = bb[c * nc + N] - bb[c * nc + O];
        mb += tb * (gradU[(c * 3) * nc + Cu] * dc.x + gradU[(c * 3 + 1) * nc + Cu] * dc.y +
                    gradU[(c * 3 + 2) * nc + Cu] * dc.z);
        lsU[c * ni + f] = tb * m;
      }
      phib[f] += mb;
    }
    nuf[f] = nv;
  } else {
    const int b = f - ni;
    const int O = t.bown[b];
    const int kind = face_kind(t, b, DIFVM_BC_VELOCITY);
    if (kind == DIFVM_FACE_FIXED) {
      const T a = nu * ck.x;
      T s = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T bo = bb[c * nc + O];
        s += bo * Ub[c * nb + b];
        if (Ubb) Ubb[c * nb + b] += (a - m) * bo;
      }
      phib[f] = -s;
      nuf[f] = (double)(ck.x * (Db[O] + s));
    } else {
      phib[f] = kind == DIFVM_FACE_ZEROGRAD ? Db[O] : T(0);
      nuf[f] = 0.0;
    }
  }
}

// Gather of the momentum non-orthogonal terms: (grad U^n)_bar (overwritten) and
// the limiter's U^n_bar terms; SOU: the upwind cell's share t_bar m (x_f - x_C).
template <typename T, bool NONORTH, bool SOU>
__global__ void __launch_bounds__(kPB) k_adj_mom_cells2(Topo t, Geo<T> g, const T* lkU,
                                                        const T* ldU, const T* phi0, const V4<T>* sd,
                                                        const T* lsU, T* gUb, T* Ubar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc, ni = t.ni;
  T ga[3][3], ua[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ua[c] = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) ga[c][k] = T(0);
  }
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e];
    const int f = ent >> 1;
    if (f >= ni) break;
    const bool nside = ent & 1;
    if (NONORTH) {
      const T w = ld4(g.Sw + f).w;
      const T wi = nside ? T(1) - w : w;
      const V4<T> ck = ld4(g.ck + f);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T l = wi * lkU[c * ni + f];
        ga[c][0] += l * ck.y;
        ga[c][1] += l * ck.z;
        ga[c][2] += l * ck.w;
        const T d = ldU[c * ni + f];
        ua[c] += nside ? d : -d;
      }
    }
    if (SOU && ((phi0[f] >= T(0)) != nside)) {   // this cell is the face's upwind cell
      const V4<T> dc = ld4(sd + (nside ? ni + f : f));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T l = lsU[c * ni + f];
        ga[c][0] += l * dc.x;
        ga[c][1] += l * dc.y;
        ga[c][2] += l * dc.z;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int k = 0; k < 3; ++k) gUb[(c * 3 + k) * nc + i] = ga[c][k];
    Ubar[c * nc + i] += ua[c];
  }
}

// Fixed-order FP64 sum: kRedBlocks blocks stride the array, one block adds the
// partial sums in block order and accumulates into *out.
constexpr int kRedBlocks = 296;
__global__ void __launch_bounds__(kPB) k_sum_partial(int n, const double* a, double* part) {
  double s = 0.0;
  for (int i = blockIdx.x * kPB + threadIdx.x; i < n; i += kRedBlocks * kPB) s += a[i];
  __shared__ double sm[kPB];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int h = kPB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void k_sum_final(const double* part, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < kRedBlocks; ++k) s += part[k];
  *out += s;
}

template <typename T>
__global__ void k_axpy1(int n, const T* a, T* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] += a[i];
}

// Windkessel backwards, one block per outlet: p_out_bar = sum of the patch's p_b
// adjoint (the patch's input p_b is overwritten, so its adjoint is zero), RCR
// step derivatives, then Q_bar is added to every face flux of the patch.
template <typename T>
__global__ void __launch_bounds__(kPB) k_adj_windkessel(int ni, const int* pstart, const int* psize,
                                                        int scheme, double dt, const double* wk,
                                                        const double* pc_in, const double* Q,
                                                        T* pbb, T* phib, double* wkb,
                                                        double* Qbar, double* pobar) {
  const int o = blockIdx.x;
  const int s = pstart[o], z = psize[o];
  double acc = 0.0;
  for (int k = threadIdx.x; k < z; k += blockDim.x) {
    acc += (double)pbb[s + k - ni];
    pbb[s + k - ni] = T(0);
  }
  __shared__ double sm[kPB / 32];
  __shared__ double qb_sh;
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double pob = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) pob += sm[k];
    const double Rp = wk[4 * o], C = wk[4 * o + 1], Rd = wk[4 * o + 2], q = Q[o];
    double dp0, dq, drd, dc;
    wk_partials(scheme, C, Rd, q, dt, pc_in[o], dp0, dq, drd, dc);
    const double G = wkb[4 * o + 3] + pob;
    const double qb = G * dq + pob * Rp;
    wkb[4 * o] += pob * q;
    wkb[4 * o + 1] += G * dc;
    wkb[4 * o + 2] += G * drd;
    wkb[4 * o + 3] = G * dp0;
    Qbar[o] = qb;
    pobar[o] = pob;
    qb_sh = qb;
  }
  __syncthreads();
  const T qb = (T)qb_sh;
  for (int k = threadIdx.x; k < z; k += blockDim.x) phib[s + k] += qb;
}

// p_c before the step, for the tape
__global__ void k_tape_wk_in(int n_out, const double* wk, double* pc_in) {
  int o = threadIdx.x;
  if (o < n_out) pc_in[o] = wk[4 * o + 3];
}

// ---------------------------------------------------------------- driver
static inline bool amg_opts(const difvm_solve_opts& o) {
  return o.precond == DIFVM_PRECOND_AMG || o.precond == DIFVM_PRECOND_AMG_REUSE;
}

// Tape of one recorded step (byte offsets, each section 256-byte aligned):
// U^n [3][nc], U_s [n_corr+1][3][nc] (U_0 = predicted velocity, U_s after
// corrector s), p_s [n_corr+1][nc] (p_0 = p^n), phi^n [nf], p_b after the
// Windkessel update [nb], then FP64 p_c before the step [16] and Q [16].
struct TapeLayout {
  size_t U0, Us, ps, phi, pb, wk, bytes;
};
static TapeLayout tape_layout(const difvm_piso* h) {
  const difvm_mesh* m = h->m;
  const size_t e = h->elt, nc = m->nc, K = h->o.n_corr;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  TapeLayout L;
  size_t off = 0;
  L.U0 = off; off = al(off + 3 * nc * e);
  L.Us = off; off = al(off + 3 * nc * e * (K + 1));
  L.ps = off; off = al(off + nc * e * (K + 1));
  L.phi = off; off = al(off + (size_t)m->nf * e);
  L.pb = off; off = al(off + (size_t)std::max(m->nb, 1) * e);
  L.wk = off; off = al(off + 32 * sizeof(double));
  L.bytes = off;
  return L;
}

// the Crank-Nicolson transform of the assembled backward-Euler rows (U = U^n)
template <typename T>
static difvm_status momentum_cn(difvm_piso* h, const T* U, cudaStream_t st) {
  const difvm_mesh* m = h->m;
  k_cn_cells<T><<<blocks_for(m->nc, kPB), kPB, 0, st>>>(m->topo(), geo<T>(m), (T)(1.0 / h->o.dt),
                                                        (const T*)h->Lo, (const T*)h->Up, U, (T*)h->D,
                                                        (T*)h->b, (T*)h->rhs);
  DIFVM_TRY(check_launch("cn_cells"));
  if (m->ni > 0) {
    k_cn_faces<T><<<blocks_for(m->ni, kPB), kPB, 0, st>>>(m->ni, (T*)h->Lo, (T*)h->Up);
    DIFVM_TRY(check_launch("cn_faces"));
  }
  return DIFVM_OK;
}

template <typename T, typename... A>
static void launch_mom_cells(bool no_U, bool sou, unsigned Bc, cudaStream_t st, A... a) {
  if (no_U && sou) k_mom_cells<T, true, true><<<Bc, kPB, 0, st>>>(a...);
  else if (no_U) k_mom_cells<T, true, false><<<Bc, kPB, 0, st>>>(a...);
  else if (sou) k_mom_cells<T, false, true><<<Bc, kPB, 0, st>>>(a...);
  else k_mom_cells<T, false, false><<<Bc, kPB, 0, st>>>(a...);
}

template <typename T>
static difvm_status piso_step_t(difvm_piso* h, T* U, T* p, T* phi, const T* Ub, T* pb, double* wk,
                                difvm_piso_info* info, unsigned char* tape, cudaStream_t st) {
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
  double* Qd = (double*)(h->sinfo + 7 * h->nk + 1);
  double* pod = Qd + 16;
  int worst = DIFVM_OK;
  TapeLayout TL{};
  const size_t v3 = 3 * (size_t)nc * sizeof(T), v1 = (size_t)nc * sizeof(T);
  if (o.n_out > 0 && !wk) return set_error(DIFVM_EINVAL, "Windkessel outlets need the wk state array");
  if (tape) {
    TL = tape_layout(h);
    DIFVM_CUDA(cudaMemcpyAsync(tape + TL.U0, U, v3, cudaMemcpyDeviceToDevice, st));
    DIFVM_CUDA(cudaMemcpyAsync(tape + TL.ps, p, v1, cudaMemcpyDeviceToDevice, st));
    DIFVM_CUDA(cudaMemcpyAsync(tape + TL.phi, phi, (size_t)nf * sizeof(T), cudaMemcpyDeviceToDevice, st));
    if (o.n_out > 0) {
      k_tape_wk_in<<<1, 32, 0, st>>>(o.n_out, wk, (double*)(tape + TL.wk));
      DIFVM_TRY(check_launch("tape_wk_in"));
    }
  }
  // 1. Windkessel outlets
  phase_mark(DIFVM_PHASE_WINDKESSEL, st);
  if (o.n_out > 0) {
    if (!wk) return set_error(DIFVM_EINVAL, "Windkessel outlets need the wk state array");
    // patch starts/sizes of the outlets live in a small device table after Qd/pod
    int* tab = (int*)(pod + 16);
    k_piso_windkessel<T><<<o.n_out, kPB, 0, st>>>(ni, tab, tab + 16, o.wk_scheme, o.dt, phi, pb, wk,
                                                    Qd, pod);
    DIFVM_TRY(check_launch("piso_windkessel"));
  }
  if (tape) {
    const size_t nbb = (size_t)m->nb * sizeof(T);
    if (pb && nbb)
      DIFVM_CUDA(cudaMemcpyAsync(tape + TL.pb, pb, nbb, cudaMemcpyDeviceToDevice, st));
    else if (nbb)
      DIFVM_CUDA(cudaMemsetAsync(tape + TL.pb, 0, nbb, st));
    if (o.n_out > 0)
      DIFVM_CUDA(cudaMemcpyAsync(tape + TL.wk + 16 * sizeof(double), Qd, o.n_out * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
  }
  // 2. momentum predictor
  phase_mark(DIFVM_PHASE_MOMENTUM_ASSEMBLY, st);
  DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_PRESSURE, p, pb, 1, gradp, st));
  const bool no_U = (o.nonorth & DIFVM_NONORTH_MOMENTUM) != 0;
  const bool no_p = (o.nonorth & DIFVM_NONORTH_PRESSURE) != 0;
  const bool sou = o.conv == DIFVM_CONV_SOU;
  if (no_U || sou) DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_VELOCITY, U, Ub, 3, gradU, st));
  if (ni > 0) {
    k_mom_faces<T><<<Bi, kPB, 0, st>>>(ni, g, (T)o.nu, phi, Lo, Up);
    DIFVM_TRY(check_launch("mom_faces"));
  }
  const T psi = (T)o.nonorth_limit;
  launch_mom_cells<T>(no_U, sou, Bc, st, t, g, (T)o.nu, (T)(1.0 / o.dt), psi, phi, U, Ub, gradU,
                      (const V4<T>*)h->sou_d, gradp, D, b, rhs);
  DIFVM_TRY(check_launch("mom_cells"));
  if (o.time_scheme == DIFVM_TIME_CN) DIFVM_TRY(momentum_cn<T>(h, U, st));
  // multigrid pressure solves: build corrector 0's operators beside the momentum solve
  const bool prebuilt = h->side != nullptr;
  if (prebuilt) {
    DIFVM_CUDA(cudaEventRecord(h->ev_fork, st));
    DIFVM_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    T* rAUe = (T*)h->rAU_e;
    k_p_rau<T><<<Bc, kPB, 0, h->side>>>(nc, g, D, rAUe);
    k_p_matrix<T><<<Bf, kPB, 0, h->side>>>(t, g, rAUe, af, Lp);
    k_p_diag<T><<<Bc, kPB, 0, h->side>>>(t, af, h->pin, h->pinflag, Dp);
    DIFVM_TRY(check_launch("p_matrix"));
    count_launch(); count_launch();
    DIFVM_TRY(amg_prebuild(m, h->mixed ? 4 : sizeof(T), Dp, Lp, h->wsp, h->wsp_bytes, h->side));
    DIFVM_CUDA(cudaEventRecord(h->ev_join, h->side));
  }
  phase_mark(DIFVM_PHASE_MOMENTUM_SOLVE, st);
  {
    difvm_prec pr = sizeof(T) == 8 ? DIFVM_F64 : DIFVM_F32;
    difvm_status s = difvm_krylov_solve(m, pr, &o.solve_U, D, Lo, Up, rhs, U, 3, h->wsU, h->wsU_bytes,
                                        h->sinfo, st);
    if (s == DIFVM_EINVAL || s == DIFVM_ECUDA) return s;
    worst = std::max(worst, (int)s);
  }
  if (tape) DIFVM_CUDA(cudaMemcpyAsync(tape + TL.Us, U, v3, cudaMemcpyDeviceToDevice, st));
  if (prebuilt) DIFVM_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
  // 3. pressure correctors
  for (int corr = 0; corr < o.n_corr; ++corr) {
    phase_mark(DIFVM_PHASE_PRESSURE_ASSEMBLY, st);
    k_HbyA<T><<<Bc, kPB, 0, st>>>(t, g, D, Lo, Up, b, U, HbyA, rAU);
    DIFVM_TRY(check_launch("HbyA"));
    if (no_p) {
      DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_PRESSURE, p, pb, 1, gradp, st));
      k_p_faces<T, true><<<Bf, kPB, 0, st>>>(t, g, psi, HbyA, rAU, Ub, gradp, p, phiH, af, no, Lp);
    } else {
      k_p_faces<T, false><<<Bf, kPB, 0, st>>>(t, g, psi, HbyA, rAU, Ub, gradp, p, phiH, af, no, Lp);
    }
    DIFVM_TRY(check_launch("p_faces"));
    k_p_cells<T><<<Bc, kPB, 0, st>>>(t, phiH, af, no, pb, h->pin, h->pinflag, Dp, bp);
    DIFVM_TRY(check_launch("p_cells"));
    difvm_solve_info* si = h->sinfo + (3 + std::min(corr, 3)) * h->nk;
    // the pressure matrix depends only on V/D: correctors after the first reuse the
    // multigrid operators the first one built
    difvm_solve_opts sp = o.solve_p;
    if ((corr > 0 || prebuilt) && amg_opts(sp)) sp.precond = DIFVM_PRECOND_AMG_REUSE;
    phase_mark(DIFVM_PHASE_PRESSURE_SOLVE, st);
    difvm_status s;
    if (h->mixed) {
      k_to64<T><<<Bc, kPB, 0, st>>>(nc, bp, h->b64);
      k_to64<T><<<Bc, kPB, 0, st>>>(nc, p, h->p64);
      DIFVM_TRY(check_launch("to64"));
      count_launch();
      s = difvm_krylov_solve_refine(m, &sp, (const float*)Dp, (const float*)Lp, nullptr,
                                    h->b64, h->p64, 1, h->wsp, h->wsp_bytes, si, st);
      k_from64<T><<<Bc, kPB, 0, st>>>(nc, h->p64, p);
      DIFVM_TRY(check_launch("from64"));
    } else {
      difvm_prec pr = sizeof(T) == 8 ? DIFVM_F64 : DIFVM_F32;
      s = difvm_krylov_solve(m, pr, &sp, Dp, Lp, nullptr, bp, p, 1, h->wsp, h->wsp_bytes, si, st);
    }
    if (s == DIFVM_EINVAL || s == DIFVM_ECUDA) return s;
    worst = std::max(worst, (int)s);
    phase_mark(DIFVM_PHASE_CORRECTION, st);
    k_flux_correct<T><<<Bf, kPB, 0, st>>>(t, phiH, af, no, p, pb, phi);
    DIFVM_TRY(check_launch("flux_correct"));
    DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_PRESSURE, p, pb, 1, gradp, st));
    k_U_correct<T><<<Bc, kPB, 0, st>>>(nc, HbyA, rAU, gradp, U);
    DIFVM_TRY(check_launch("U_correct"));
    if (tape) {
      DIFVM_CUDA(cudaMemcpyAsync(tape + TL.Us + (corr + 1) * v3, U, v3, cudaMemcpyDeviceToDevice, st));
      DIFVM_CUDA(cudaMemcpyAsync(tape + TL.ps + (corr + 1) * v1, p, v1, cudaMemcpyDeviceToDevice, st));
    }
  }
  if (info) {
    k_piso_info<<<1, 32, 0, st>>>(h->sinfo, h->nk, o.n_corr, DIFVM_OK, o.n_out, Qd, pod, info);
    DIFVM_TRY(check_launch("piso_info"));
  }
  phase_mark(-1, st);
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
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
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
  if (o->conv != DIFVM_CONV_UPWIND && o->conv != DIFVM_CONV_SOU)
    return set_error(DIFVM_EINVAL, "unknown convection scheme %d", o->conv);
  if (o->time_scheme != DIFVM_TIME_BE && o->time_scheme != DIFVM_TIME_CN)
    return set_error(DIFVM_EINVAL, "unknown time scheme %d", o->time_scheme);
  if (o->solve_U.method != DIFVM_BICGSTAB && o->solve_U.method != DIFVM_PCG)
    return set_error(DIFVM_EINVAL, "bad momentum solver");
  if (o->solve_p.method != DIFVM_PCG && o->solve_p.method != DIFVM_BICGSTAB)
    return set_error(DIFVM_EINVAL, "bad pressure solver");
  if (amg_opts(o->solve_U))
    return set_error(DIFVM_EINVAL, "the multigrid preconditioner serves the pressure CG only");
  if (amg_opts(o->solve_p) && o->solve_p.method != DIFVM_PCG)
    return set_error(DIFVM_EINVAL, "the multigrid preconditioner needs CG");
  if (o->solve_U.precond == DIFVM_PRECOND_DIC &&
      (o->solve_U.method != DIFVM_BICGSTAB || m->seg || (prec == DIFVM_F32 && o->solve_U.refine_max > 0)))
    return set_error(DIFVM_EINVAL, "the incomplete LU preconditioner of the momentum solve needs BiCGStab "
                                   "on a single (not batched) mesh");
  if (o->solve_p.precond == DIFVM_PRECOND_DIC &&
      (o->solve_p.method != DIFVM_PCG || m->seg || (prec == DIFVM_F32 && o->solve_p.refine_max > 0)))
    return set_error(DIFVM_EINVAL, "the incomplete-Cholesky preconditioner needs CG without refinement on a "
                                   "single (not batched) mesh");
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
  h->nk = m->seg ? m->ncases : 1;
  if (h->mixed && m->seg) {
    delete h;
    return set_error(DIFVM_EINVAL, "FP64 refinement of the pressure solve is not available on batched "
                                   "meshes (use FP32 with FP64 dots, refine_max = 0, or FP64)");
  }
  // which cases have a fixed-pressure face (their pressure needs no pin)
  std::vector<char> fixed(h->nk, 0);
  for (int p = 0; p < m->npatch; ++p) {
    if (m->patch_type[p] != DIFVM_PATCH_OUTLET) continue;
    for (int f = m->patch_start[p]; f < m->patch_start[p] + m->patch_size[p]; ++f) {
      const int own = m->bown_host[f - m->ni];
      const int k = (int)(std::upper_bound(m->case_start.begin(), m->case_start.end(), own) -
                          m->case_start.begin()) - 1;
      fixed[m->seg ? k : 0] = 1;
    }
  }
  std::vector<unsigned char> pf;
  for (int k = 0; k < h->nk; ++k) {
    if (fixed[k]) continue;
    const int n0 = m->seg ? m->case_start[k] : 0, n1 = m->seg ? m->case_start[k + 1] : m->nc;
    if (o->pref_cell < 0 || o->pref_cell >= n1 - n0) {
      delete h;
      return set_error(DIFVM_EINVAL, "pref_cell %d out of range of case %d (no face fixes p there)",
                       o->pref_cell, k);
    }
    if (m->seg) {
      if (pf.empty()) pf.assign(m->nc, 0);
      pf[n0 + o->pref_cell] = 1;
    } else {
      h->pin = o->pref_cell;
    }
  }
  h->has_fixed_p = fixed[0];
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
            alloc(&h->phiHbyA, nf * e) && alloc(&h->af, nf * e) && alloc(&h->nonorth, ni * e) &&
            (o->conv != DIFVM_CONV_SOU || alloc(&h->sou_d, 2 * ni * (e == 8 ? sizeof(V4<double>) : sizeof(V4<float>))));
  h->wsU_bytes = difvm_krylov_opts_workspace_bytes(m, prec, &o->solve_U, 3);
  ok = ok && h->wsU_bytes > 0 && alloc(&h->wsU, h->wsU_bytes);
  h->wsp_bytes = difvm_krylov_opts_workspace_bytes(m, prec, &o->solve_p, 1);
  if (h->mixed) ok = ok && alloc((void**)&h->p64, nc * 8) && alloc((void**)&h->b64, nc * 8);
  ok = ok && h->wsp_bytes > 0 && alloc(&h->wsp, h->wsp_bytes);
  // solve infos [7 nk + 1] + Q[16] + p_out[16] + outlet table (start[16], size[16])
  const size_t ninfo = 7 * (size_t)h->nk + 1;
  ok = ok && alloc((void**)&h->sinfo, ninfo * sizeof(difvm_solve_info) + 32 * sizeof(double) + 32 * sizeof(int));
  if (!pf.empty()) ok = ok && alloc((void**)&h->pinflag, m->nc);
  if (!ok) {
    difvm_piso_destroy(h);
    return set_error(DIFVM_ENOMEM, "device allocation for the PISO workspace failed");
  }
  int tab[32] = {0};
  for (int k = 0; k < o->n_out; ++k) {
    tab[k] = m->patch_start[o->wk_patch[k]];
    tab[16 + k] = m->patch_size[o->wk_patch[k]];
  }
  if (amg_opts(o->solve_p) && !m->seg) {
    if (!alloc(&h->rAU_e, nc * e) ||
        cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      difvm_piso_destroy(h);
      return set_error(DIFVM_ECUDA, "side stream for the multigrid setup could not be created");
    }
  }
  if (o->conv == DIFVM_CONV_SOU && m->ni > 0) {
    if (e == 8)
      k_sou_d<double><<<blocks_for(m->ni, kPB), kPB>>>(m->ni, m->on, m->Cf64, m->C64, (V4<double>*)h->sou_d);
    else
      k_sou_d<float><<<blocks_for(m->ni, kPB), kPB>>>(m->ni, m->on, m->Cf64, m->C64, (V4<float>*)h->sou_d);
    if (check_launch("sou_d") != DIFVM_OK || cudaDeviceSynchronize() != cudaSuccess) {
      difvm_piso_destroy(h);
      return set_error(DIFVM_ECUDA, "second-order upwind setup failed");
    }
  }
  double* Qd = (double*)(h->sinfo + ninfo);
  if (cudaMemcpy(Qd + 32, tab, sizeof tab, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(h->sinfo, 0, ninfo * sizeof(difvm_solve_info) + 32 * sizeof(double)) != cudaSuccess ||
      (!pf.empty() && cudaMemcpy(h->pinflag, pf.data(), pf.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
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
                               (double*)pb, wk, info, nullptr, st);
  return piso_step_t<float>(h, (float*)U, (float*)p, (float*)phi, (const float*)Ub, (float*)pb, wk,
                            info, nullptr, st);
}

// ---------------------------------------------------------------- adjoint driver
static difvm_status adj_alloc(difvm_piso* h) {
  if (h->adj_ready) return DIFVM_OK;
  const difvm_mesh* m = h->m;
  const size_t e = h->elt, nc = m->nc, ni = std::max(m->ni, 1), nf = m->nf;
  const size_t nb = std::max(m->nb, 1);
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) return false;
    h->allocs.push_back(*p);
    return true;
  };
  bool ok = alloc(&h->a_HAb, 3 * nc * e) && alloc(&h->a_gpb, 3 * nc * e) &&
            alloc(&h->a_gpn, 3 * nc * e) && alloc(&h->a_rAUb, nc * e) && alloc(&h->a_Db, nc * e) &&
            alloc(&h->a_bb, 3 * nc * e) && alloc(&h->a_Lob, ni * e) && alloc(&h->a_Upb, ni * e) &&
            alloc(&h->a_lam, nc * e) && alloc(&h->a_lamU, 3 * nc * e) &&
            alloc(&h->a_phiHb, nf * e) && alloc(&h->a_rfb, nf * e) && alloc(&h->a_lk, ni * e) &&
            alloc(&h->a_ld, ni * e) && alloc(&h->a_phio, nf * e) && alloc(&h->a_pbb, nb * e) &&
            alloc(&h->a_gUb, 9 * nc * e) && alloc(&h->a_lkU, 3 * ni * e) &&
            alloc(&h->a_ldU, 3 * ni * e) && alloc(&h->a_gp2, 3 * nc * e) &&
            (h->o.conv != DIFVM_CONV_SOU || alloc(&h->a_lsU, 3 * ni * e)) &&
            alloc((void**)&h->a_nuf, nf * sizeof(double)) &&
            alloc((void**)&h->a_part, kRedBlocks * sizeof(double)) &&
            alloc(&h->a_lamw, (size_t)h->o.n_corr * nc * (h->mixed ? 8 : e));
  if (!ok) return set_error(DIFVM_ENOMEM, "device allocation for the PISO adjoint workspace failed");
  DIFVM_CUDA(cudaMemset(h->a_lamw, 0, (size_t)h->o.n_corr * nc * (h->mixed ? 8 : e)));
  DIFVM_CUDA(cudaMemset(h->a_lamU, 0, 3 * nc * e));
  h->adj_ready = true;
  return DIFVM_OK;
}

// lam = A_p^{-1} rhs with the forward step's pressure matrix and solver
// settings (the matrix is symmetric, so A^{-T} = A^{-1}).  The solve starts
// from corrector s's solution of the previous call, like the forward step
// starts from p^n; *lam points at the result.
template <typename T>
static difvm_status adj_psolve(difvm_piso* h, const T* rhs, int s, T* scratch, T** lam,
                               difvm_solve_info* si, cudaStream_t st) {
  difvm_mesh* m = h->m;
  const int nc = m->nc;
  const unsigned Bc = blocks_for(nc, kPB);
  // the reverse sweep recomputed the step's pressure matrix: its first adjoint
  // solve (the last corrector's) builds the multigrid operators, the others reuse them
  difvm_solve_opts sp = h->o.solve_p;
  if (s < h->o.n_corr - 1 && amg_opts(sp)) sp.precond = DIFVM_PRECOND_AMG_REUSE;
  if (h->mixed) {
    double* x = (double*)h->a_lamw + (size_t)s * nc;
    k_to64<T><<<Bc, kPB, 0, st>>>(nc, rhs, h->b64);
    DIFVM_TRY(check_launch("to64"));
    difvm_status r = difvm_krylov_solve_refine(m, &sp, (const float*)h->Dp,
                                               (const float*)h->Lp, nullptr, h->b64, x, 1, h->wsp,
                                               h->wsp_bytes, si, st);
    if (r == DIFVM_EINVAL || r == DIFVM_ECUDA) return r;
    k_from64<T><<<Bc, kPB, 0, st>>>(nc, x, scratch);
    DIFVM_TRY(check_launch("from64"));
    *lam = scratch;
    return r;
  }
  T* x = (T*)h->a_lamw + (size_t)s * nc;
  difvm_prec pr = sizeof(T) == 8 ? DIFVM_F64 : DIFVM_F32;
  *lam = x;
  return difvm_krylov_solve(m, pr, &sp, h->Dp, h->Lp, nullptr, rhs, x, 1, h->wsp,
                            h->wsp_bytes, si, st);
}

template <typename T>
static difvm_status piso_step_bwd_t(difvm_piso* h, const unsigned char* tape, const T* Ub,
                                    const double* wk, T* Ubar, T* pbar, T* phibar, T* pbbar,
                                    double* wkbar, T* Ubbar, double* nubar, difvm_piso_info* info,
                                    cudaStream_t st) {
  difvm_mesh* m = h->m;
  const int nc = m->nc, ni = m->ni, nf = m->nf, nb = m->nb, K = h->o.n_corr;
  const difvm_piso_opts& o = h->o;
  Topo t = m->topo();
  Geo<T> g = geo<T>(m);
  const unsigned Bc = blocks_for(nc, kPB), Bf = blocks_for(nf, kPB), Bi = blocks_for(std::max(ni, 1), kPB);
  const TapeLayout TL = tape_layout(h);
  const size_t v3 = 3 * (size_t)nc, v1 = nc;
  const T* U0 = (const T*)(tape + TL.U0);
  const T* Us = (const T*)(tape + TL.Us);
  const T* ps = (const T*)(tape + TL.ps);
  const T* phi0 = (const T*)(tape + TL.phi);
  const T* pb1 = (const T*)(tape + TL.pb);
  const double* pc_in = (const double*)(tape + TL.wk);
  const double* Qrec = pc_in + 16;
  T *gradp = (T*)h->gradp, *gradU = (T*)h->gradU, *D = (T*)h->D, *Lo = (T*)h->Lo, *Up = (T*)h->Up;
  T *b = (T*)h->b, *rhs = (T*)h->rhs, *rAU = (T*)h->rAU, *HbyA = (T*)h->HbyA, *Dp = (T*)h->Dp;
  T *Lp = (T*)h->Lp, *bp = (T*)h->bp, *phiH = (T*)h->phiHbyA, *af = (T*)h->af;
  T* no = (T*)h->nonorth;
  T *HAb = (T*)h->a_HAb, *gpb = (T*)h->a_gpb, *gpn = (T*)h->a_gpn, *rAUb = (T*)h->a_rAUb;
  T *Db = (T*)h->a_Db, *bb = (T*)h->a_bb, *Lob = (T*)h->a_Lob, *Upb = (T*)h->a_Upb;
  T *lam_scratch = (T*)h->a_lam, *lamU = (T*)h->a_lamU, *phiHb = (T*)h->a_phiHb, *rfb = (T*)h->a_rfb;
  T *lk = (T*)h->a_lk, *ld = (T*)h->a_ld, *phio = (T*)h->a_phio, *pbb = (T*)h->a_pbb;
  T *gUb = (T*)h->a_gUb, *lkU = (T*)h->a_lkU, *ldU = (T*)h->a_ldU, *gp2 = (T*)h->a_gp2;
  const bool no_U = (o.nonorth & DIFVM_NONORTH_MOMENTUM) != 0;
  const bool no_p = (o.nonorth & DIFVM_NONORTH_PRESSURE) != 0;
  const T psi = (T)o.nonorth_limit;
  const difvm_prec pr = sizeof(T) == 8 ? DIFVM_F64 : DIFVM_F32;
  double* Qb = (double*)(h->sinfo + 7 * h->nk + 1);
  double* pob = Qb + 16;
  int worst = DIFVM_OK;

  // recompute the forward step's matrices from the tape
  DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_PRESSURE, ps, pb1, 1, gradp, st));
  const bool sou = o.conv == DIFVM_CONV_SOU;
  const V4<T>* sd = (const V4<T>*)h->sou_d;
  if (no_U || sou) DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_VELOCITY, U0, Ub, 3, gradU, st));
  if (ni > 0) {
    k_mom_faces<T><<<Bi, kPB, 0, st>>>(ni, g, (T)o.nu, phi0, Lo, Up);
    DIFVM_TRY(check_launch("mom_faces"));
  }
  launch_mom_cells<T>(no_U, sou, Bc, st, t, g, (T)o.nu, (T)(1.0 / o.dt), psi, phi0, U0, Ub, gradU, sd,
                      gradp, D, b, rhs);
  DIFVM_TRY(check_launch("mom_cells"));
  if (o.time_scheme == DIFVM_TIME_CN) DIFVM_TRY(momentum_cn<T>(h, U0, st));
  k_HbyA<T><<<Bc, kPB, 0, st>>>(t, g, D, Lo, Up, b, Us, HbyA, rAU);
  DIFVM_TRY(check_launch("HbyA"));
  k_p_faces<T, false><<<Bf, kPB, 0, st>>>(t, g, psi, HbyA, rAU, Ub, gradp, ps, phiH, af, no, Lp);
  DIFVM_TRY(check_launch("p_faces"));
  k_p_cells<T><<<Bc, kPB, 0, st>>>(t, phiH, af, no, pb1, h->pin, h->pinflag, Dp, bp);
  DIFVM_TRY(check_launch("p_cells"));

  // adjoint state
  DIFVM_CUDA(cudaMemcpyAsync(phio, phibar, (size_t)nf * sizeof(T), cudaMemcpyDeviceToDevice, st));
  if (nb > 0) {
    if (pbbar)
      DIFVM_CUDA(cudaMemcpyAsync(pbb, pbbar, (size_t)nb * sizeof(T), cudaMemcpyDeviceToDevice, st));
    else
      DIFVM_CUDA(cudaMemsetAsync(pbb, 0, (size_t)nb * sizeof(T), st));
  }
  DIFVM_CUDA(cudaMemsetAsync(gpn, 0, v3 * sizeof(T), st));
  DIFVM_CUDA(cudaMemsetAsync(rAUb, 0, v1 * sizeof(T), st));
  DIFVM_CUDA(cudaMemsetAsync(Db, 0, v1 * sizeof(T), st));
  DIFVM_CUDA(cudaMemsetAsync(bb, 0, v3 * sizeof(T), st));
  DIFVM_CUDA(cudaMemsetAsync(Lob, 0, (size_t)std::max(ni, 1) * sizeof(T), st));
  DIFVM_CUDA(cudaMemsetAsync(Upb, 0, (size_t)std::max(ni, 1) * sizeof(T), st));

  // pressure correctors, last first
  for (int s = K - 1; s >= 0; --s) {
    const T* Uk = Us + s * v3;
    const T* pk = ps + s * v1;
    const T* pn = pk + v1;
    DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_PRESSURE, pn, pb1, 1, gradp, st));
    k_adj_Ucorr<T><<<Bc, kPB, 0, st>>>(nc, Ubar, gradp, rAU, gpn, HAb, rAUb, gpb);
    DIFVM_TRY(check_launch("adj_Ucorr"));
    DIFVM_TRY(difvm_grad_gauss_bwd(m, pr, DIFVM_BC_PRESSURE, gpb, 1, pbar, pbb, st));
    const bool last = s == K - 1;
    if (last) {
      k_adj_flux_cells<T><<<Bc, kPB, 0, st>>>(t, af, phio, pbar, pbb);
      DIFVM_TRY(check_launch("adj_flux_cells"));
    }
    T* lam = nullptr;
    {
      difvm_status sv = adj_psolve<T>(h, pbar, s, lam_scratch, &lam,
                                      h->sinfo + (3 + std::min(s, 3)) * h->nk, st);
      if (sv == DIFVM_EINVAL || sv == DIFVM_ECUDA) return sv;
      worst = std::max(worst, (int)sv);
    }
    DIFVM_CUDA(cudaMemsetAsync(pbar, 0, v1 * sizeof(T), st));   // now the adjoint of p_s
    if (no_p) DIFVM_TRY(grad_gauss_t<T>(m, DIFVM_BC_PRESSURE, pk, pb1, 1, gp2, st));
#define DIFVM_PF(NO, LA)                                                                          \
  k_adj_pfaces<T, NO, LA><<<Bf, kPB, 0, st>>>(t, g, psi, h->pin, h->pinflag, lam, pn, pk, gp2,  \
                                              rAU, af, pb1,                                      \
                                              phio, phiHb, rfb, lk, ld, pbb, Ubbar)
    if (no_p) { if (last) DIFVM_PF(true, true); else DIFVM_PF(true, false); }
    else { if (last) DIFVM_PF(false, true); else DIFVM_PF(false, false); }
#undef DIFVM_PF
    DIFVM_TRY(check_launch("adj_pfaces"));
    if (no_p)
      k_adj_pcells<T, true><<<Bc, kPB, 0, st>>>(t, g, phiHb, rfb, lk, ld, HAb, rAUb, gpn, pbar);
    else
      k_adj_pcells<T, false><<<Bc, kPB, 0, st>>>(t, g, phiHb, rfb, lk, ld, HAb, rAUb, gpn, pbar);
    DIFVM_TRY(check_launch("adj_pcells"));
    k_adj_HbyA<T><<<Bc, kPB, 0, st>>>(t, D, Lo, Up, b, Uk, HAb, Db, bb, Ubar);
    DIFVM_TRY(check_launch("adj_HbyA"));
    if (ni > 0) {
      k_adj_LU<T><<<Bi, kPB, 0, st>>>(ni, nc, t.on, D, HAb, Uk, Lob, Upb);
      DIFVM_TRY(check_launch("adj_LU"));
    }
  }

  // momentum predictor: lamU = A^{-T} U_bar_0 (lower and upper swapped), started
  // from the previous call's lamU
  {
    difvm_status sv = difvm_krylov_solve(m, pr, &o.solve_U, D, Up, Lo, Ubar, lamU, 3, h->wsU,
                                         h->wsU_bytes, h->sinfo, st);
    if (sv == DIFVM_EINVAL || sv == DIFVM_ECUDA) return sv;
    worst = std::max(worst, (int)sv);
  }
  k_adj_mom_cells<T><<<Bc, kPB, 0, st>>>(nc, g, (T)(1.0 / o.dt), D, lamU, Us, rAUb, Db, bb, gpn, Ubar);
  DIFVM_TRY(check_launch("adj_mom_cells"));
  const int cn = o.time_scheme == DIFVM_TIME_CN;
  if (cn) {
    k_adj_cn_cells<T><<<Bc, kPB, 0, st>>>(t, g, (T)(1.0 / o.dt), D, Lo, Up, U0, bb, Db, Ubar);
    DIFVM_TRY(check_launch("adj_cn_cells"));
  }
  DIFVM_TRY(difvm_grad_gauss_bwd(m, pr, DIFVM_BC_PRESSURE, gpn, 1, pbar, pbb, st));
  T* lsU = (T*)h->a_lsU;
#define DIFVM_AMF(NO, SO)                                                                          \
  k_adj_mom_faces<T, NO, SO><<<Bf, kPB, 0, st>>>(t, g, (T)o.nu, psi, phi0, Db, bb, Lob, Upb, lamU, Us, \
                                                 U0, gradU, Ub, phibar, h->a_nuf, lkU, ldU, sd, lsU, Ubbar, cn)
  if (no_U) { if (sou) DIFVM_AMF(true, true); else DIFVM_AMF(true, false); }
  else { if (sou) DIFVM_AMF(false, true); else DIFVM_AMF(false, false); }
#undef DIFVM_AMF
  DIFVM_TRY(check_launch("adj_mom_faces"));
  if (no_U || sou) {
    if (no_U && sou) k_adj_mom_cells2<T, true, true><<<Bc, kPB, 0, st>>>(t, g, lkU, ldU, phi0, sd, lsU, gUb, Ubar);
    else if (no_U) k_adj_mom_cells2<T, true, false><<<Bc, kPB, 0, st>>>(t, g, lkU, ldU, phi0, sd, lsU, gUb, Ubar);
    else k_adj_mom_cells2<T, false, true><<<Bc, kPB, 0, st>>>(t, g, lkU, ldU, phi0, sd, lsU, gUb, Ubar);
    DIFVM_TRY(check_launch("adj_mom_cells2"));
    DIFVM_TRY(difvm_grad_gauss_bwd(m, pr, DIFVM_BC_VELOCITY, gUb, 3, Ubar, Ubbar, st));
  }
  if (nubar) {
    k_sum_partial<<<kRedBlocks, kPB, 0, st>>>(nf, h->a_nuf, h->a_part);
    k_sum_final<<<1, 32, 0, st>>>(h->a_part, nubar);
    DIFVM_TRY(check_launch("sum_nu"));
  }
  // Windkessel outlets
  if (o.n_out > 0) {
    int* tab = (int*)(pob + 16);
    k_adj_windkessel<T><<<o.n_out, kPB, 0, st>>>(ni, tab, tab + 16, o.wk_scheme, o.dt, wk, pc_in,
                                                  Qrec, pbb, phibar, wkbar, Qb, pob);
    DIFVM_TRY(check_launch("adj_windkessel"));
  }
  if (pbbar && nb > 0)
    DIFVM_CUDA(cudaMemcpyAsync(pbbar, pbb, (size_t)nb * sizeof(T), cudaMemcpyDeviceToDevice, st));
  if (info) {
    k_piso_info<<<1, 32, 0, st>>>(h->sinfo, h->nk, K, DIFVM_OK, o.n_out, Qb, pob, info);
    DIFVM_TRY(check_launch("piso_info"));
  }
  return (difvm_status)worst;
}

extern "C" size_t difvm_piso_tape_bytes(difvm_piso_t h) { return h ? tape_layout(h).bytes : 0; }

extern "C" difvm_status difvm_piso_adjoint_reset(difvm_piso_t h, void* stream) {
  if (!h) return set_error(DIFVM_EINVAL, "null PISO handle");
  if (!h->adj_ready) return DIFVM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nc = h->m->nc;
  DIFVM_CUDA(cudaMemsetAsync(h->a_lamw, 0, (size_t)h->o.n_corr * nc * (h->mixed ? 8 : h->elt), st));
  DIFVM_CUDA(cudaMemsetAsync(h->a_lamU, 0, 3 * nc * h->elt, st));
  return DIFVM_OK;
}

extern "C" difvm_status difvm_piso_step_record(difvm_piso_t h, void* U, void* p, void* phi,
                                               const void* Ub, void* pb, double* wk,
                                               difvm_piso_info* info, void* tape,
                                               size_t tape_bytes, void* stream) {
  if (!h) return set_error(DIFVM_EINVAL, "null PISO handle");
  if (!U || !p || !phi) return set_error(DIFVM_EINVAL, "null state field");
  if (!tape) return set_error(DIFVM_EINVAL, "null tape");
  if ((uintptr_t)tape % 256 != 0) return set_error(DIFVM_EINVAL, "the tape must be 256-byte aligned");
  if (tape_bytes < tape_layout(h).bytes)
    return set_error(DIFVM_EINVAL, "tape of %zu bytes, the step needs %zu", tape_bytes,
                     tape_layout(h).bytes);
  cudaStream_t st = (cudaStream_t)stream;
  if (h->prec == DIFVM_F64)
    return piso_step_t<double>(h, (double*)U, (double*)p, (double*)phi, (const double*)Ub,
                               (double*)pb, wk, info, (unsigned char*)tape, st);
  return piso_step_t<float>(h, (float*)U, (float*)p, (float*)phi, (const float*)Ub, (float*)pb, wk,
                            info, (unsigned char*)tape, st);
}

extern "C" difvm_status difvm_piso_step_bwd(difvm_piso_t h, const void* tape, size_t tape_bytes,
                                            const void* Ub, const double* wk, void* U_bar,
                                            void* p_bar, void* phi_bar, void* p_b_bar,
                                            double* wk_bar, void* U_b_bar, double* nu_bar,
                                            difvm_piso_info* info, void* stream) {
  if (!h) return set_error(DIFVM_EINVAL, "null PISO handle");
  if (!tape || !U_bar || !p_bar || !phi_bar) return set_error(DIFVM_EINVAL, "null argument");
  if ((uintptr_t)tape % 256 != 0) return set_error(DIFVM_EINVAL, "the tape must be 256-byte aligned");
  if (tape_bytes < tape_layout(h).bytes)
    return set_error(DIFVM_EINVAL, "tape of %zu bytes, the step needs %zu", tape_bytes,
                     tape_layout(h).bytes);
  if (h->o.n_out > 0 && (!wk || !wk_bar))
    return set_error(DIFVM_EINVAL, "Windkessel outlets need wk and wk_bar");
  DIFVM_TRY(adj_alloc(h));
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned char* tp = (const unsigned char*)tape;
  if (h->prec == DIFVM_F64)
    return piso_step_bwd_t<double>(h, tp, (const double*)Ub, wk, (double*)U_bar, (double*)p_bar,
                                   (double*)phi_bar, (double*)p_b_bar, wk_bar, (double*)U_b_bar,
                                   nu_bar, info, st);
  return piso_step_bwd_t<float>(h, tp, (const float*)Ub, wk, (float*)U_bar, (float*)p_bar,
                                (float*)phi_bar, (float*)p_b_bar, wk_bar, (float*)U_b_bar, nu_bar,
                                info, st);
}

// The step as a CUDA graph: captured once per argument set on an internal
// stream (each Krylov solve becomes a device-side WHILE loop), then replayed
// with one launch on the caller's stream.  No host synchronisation.
extern "C" difvm_status difvm_piso_step_graph(difvm_piso_t h, void* U, void* p, void* phi,
                                              const void* Ub, void* pb, double* wk,
                                              difvm_piso_info* info, void* stream) {
  if (!h) return set_error(DIFVM_EINVAL, "null PISO handle");
  if (!U || !p || !phi || !info) return set_error(DIFVM_EINVAL, "null state field or info");
  if (h->o.n_out > 0 && !wk) return set_error(DIFVM_EINVAL, "Windkessel outlets need the wk state array");
  if (prof_active())
    return set_error(DIFVM_EINVAL, "per-kernel profiling is not available inside a graph");
  const void* key[7] = {U, p, phi, Ub, pb, wk, info};
  cudaGraphExec_t exec = nullptr;
  for (auto& g : h->graphs)
    if (std::equal(key, key + 7, g.key)) exec = g.exec;
  if (!exec) {
    if (!h->cap_stream) DIFVM_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = h->cap_stream;
    DIFVM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    difvm_status st = h->prec == DIFVM_F64
                          ? piso_step_t<double>(h, (double*)U, (double*)p, (double*)phi,
                                                (const double*)Ub, (double*)pb, wk, info, nullptr, cs)
                          : piso_step_t<float>(h, (float*)U, (float*)p, (float*)phi,
                                               (const float*)Ub, (float*)pb, wk, info, nullptr, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (st != DIFVM_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (st != DIFVM_OK) return st;
      return set_error(DIFVM_ECUDA, "capture of the PISO step: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
      return set_error(DIFVM_ECUDA, "instantiation of the PISO step graph: %s", cudaGetErrorString(e));
    difvm_piso::GraphEntry ge;
    std::copy(key, key + 7, ge.key);
    ge.exec = exec;
    h->graphs.push_back(ge);
  }
  DIFVM_CUDA(cudaGraphLaunch(exec, (cudaStream_t)stream));
  return DIFVM_OK;
}
