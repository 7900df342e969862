// Face operators of the message-passing form (Sec. 2.4.1) and their adjoints.
//
// Every operator is one cell-centric kernel: thread i walks the row of cell i
// (faces in ascending id; the forward operators read the half-face layout, in
// which a row's face records arrive with coalesced loads), recomputes the face message of each face
// exactly as the owner side does (same operands, same instruction order, so
// the owner and the neighbour see bitwise the same message), and accumulates
// sigma * message in registers.  This is the aggregation of Eq. aggregate as a
// deterministic segmented sum: no atomics, no stored face fluxes.  Face data
// (S_f, w_f packed in one 16/32-byte record; c_f, k_f in another) and the
// neighbour cell values are gathered through the read-only path; RCM ordering
// keeps the second visit of a face within L2 reach of the first.
#include <algorithm>
#include <utility>

#include "difvm_internal.cuh"

namespace difvm {

constexpr int kBlock = 256;

template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
// a rounded product that the compiler may not fuse into the following add, so
// that a face message is the same number on both of its cells
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// A row's half-face slots, four at a time: their words (and face ids, or the
// slot copies of the face records) arrive with coalesced loads issued before
// any is used.  The neighbour values and the boundary values are gathered in
// one second round: a boundary slot's word carries its patch category, so the
// face's kind for the requested boundary-condition class needs no load.  Slots
// are consumed in row order (ascending face id), so every sum keeps the CSR
// order.  WK > 0: every row has exactly WK slots, known at compile time (the
// uniform layout of tetrahedral meshes, WK = 4); WK = 0: the row width is read
// from the layout.
template <int WK>
__device__ __forceinline__ void hf_row_w(const Hf& H, int i, int& base, int& w) {
  if (WK > 0) {
    base = (i >> 5) * 32 * WK + (i & 31);
    w = WK;
  } else {
    hf_row(H, i, base, w);
  }
}

// first face owned by the slice of row i (compact slot words only)
__device__ __forceinline__ int hf_fbase(const Hf& H, int i) { return H.cw ? __ldg(H.fb + (i >> 5)) : 0; }

// words (and, with FID, face ids) of slots k0..k0+3 of row i; -1 past its end.
// With FID the compact words are read where the mesh has them (one 4-byte
// load per slot instead of 8; fb = hf_fbase(H, i)).
template <bool FID>
__device__ __forceinline__ void hf_words(const Hf& H, int i, int fb, int base, int k0, int w, int (&v)[4],
                                         int (&f)[4]) {
  if (FID && H.cw) {
    int q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = k0 + k < w ? __ldg(H.cw + base + 32 * (k0 + k)) : -1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (q[k] >= 0) {
        const int dj = (q[k] << 1) >> 17;           // bits 30..16, sign-extended
        v[k] = 2 * (i + dj) + (dj < 0 ? 1 : 0);
        f[k] = fb + (int)(short)(q[k] & 0xffff);
      } else {
        v[k] = q[k];
        f[k] = q[k] <= -2 ? H.ni + hf_bface(q[k]) : 0;
      }
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int slot = base + 32 * (k0 + k);
    v[k] = -1;
    f[k] = 0;
    if (k0 + k < w) {
      if (FID) {
        const int2 q = __ldg(H.nf + slot);
        v[k] = q.x;
        f[k] = max(q.y, 0);   // padding carries face id -1
      } else {
        v[k] = ldg(H.nb + slot);
      }
    }
  }
}

// boundary kind of slot word v (v <= -2) for class cls
__device__ __forceinline__ int hf_kind(int v, int cls) { return bc_kind(cls, hf_bcat(v)); }

// the NC components of the value across slot word v of row i: the other cell's
// (internal face), the boundary value (fixed boundary face) or the row's own
// value (zero-gradient boundary face; also returned for empty faces and
// padding, which no sum uses).  The source is chosen once per slot, so every
// component is one load with no per-component branch.
template <typename T, int NC>
__device__ __forceinline__ void hf_gather(int v, int cls, const T* __restrict__ phi, const T* __restrict__ phib,
                                          int nc, int nb, int i, T (&out)[NC]) {
  const T* src = phi + i;
  int str = nc;
  if (v >= 0) {
    src = phi + (v >> 1);
  } else if (v <= -2 && hf_kind(v, cls) == DIFVM_FACE_FIXED) {
    src = phib + hf_bface(v);
    str = nb;
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) out[c] = ldg(src + c * str);
}

// slot k0+k takes no part in a sum: padding, or an empty boundary face
__device__ __forceinline__ bool hf_skip(int v, int cls) {
  return v == -1 || (v <= -2 && hf_kind(v, cls) == DIFVM_FACE_EMPTY);
}

// ----------------------------------------------------------- Gauss gradient
// grad_i = (1/V_i) sum_f sigma phi_f S_f   (Eq. gauss_green).  Face records are
// read from their slot copies (coalesced, no face id), or with FIDGEO by face id
// from the face arrays (compact slot words: half the index bytes, each record
// from DRAM once).
template <typename T, int NC, int WK, int MINB, bool FIDGEO = false>
__global__ void __launch_bounds__(kBlock, MINB) k_grad_gauss(Topo t, Hf H, HfGeo<T> hg, Geo<T> g, int cls,
                                                             const T* __restrict__ phi,
                                                             const T* __restrict__ phib,
                                                             T* __restrict__ grad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc, nb = t.nb;
  T pi[NC], acc[NC][3];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    pi[c] = ldg(phi + c * nc + i);
    acc[c][0] = acc[c][1] = acc[c][2] = T(0);
  }
  const T r = ldg(g.rV + i);
  int base, w;
  hf_row_w<WK>(H, i, base, w);
  const int fb = FIDGEO ? hf_fbase(H, i) : 0;
  for (int k0 = 0; k0 < w; k0 += 4) {
    int v[4], f[4];
    hf_words<FIDGEO>(H, i, fb, base, k0, w, v, f);
    V4<T> s[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (FIDGEO)
        s[k] = v[k] != -1 ? ld4(g.Sw + f[k]) : V4<T>{T(0), T(0), T(0), T(0)};
      else
        s[k] = k0 + k < w ? ld4(hg.sw + base + 32 * (k0 + k)) : V4<T>{T(0), T(0), T(0), T(0)};
    }
    T pj[4][NC];
#pragma unroll
    for (int k = 0; k < 4; ++k) hf_gather<T, NC>(v[k], cls, phi, phib, nc, nb, i, pj[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int vk = v[k];
      if (hf_skip(vk, cls)) continue;
      const V4<T> sk = s[k];
      T pf[NC];
      T sg = T(1);
      if (vk >= 0) {
        const bool nside = vk & 1;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T pO = nside ? pj[k][c] : pi[c], pN = nside ? pi[c] : pj[k][c];
          pf[c] = sk.w * pO + (T(1) - sk.w) * pN;
        }
        if (nside) sg = T(-1);
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) pf[c] = pj[k][c];
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T qv = sg * pf[c];
        acc[c][0] += qv * sk.x;
        acc[c][1] += qv * sk.y;
        acc[c][2] += qv * sk.z;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) grad[(c * 3 + d) * nc + i] = acc[c][d] * r;
}

// Adjoint: with a_i = grad_bar_i / V_i, a face carries (a_O - a_N).S back to
// its two cells with weights w and 1-w (zero-gradient boundary faces to the
// owner, fixed boundary faces to phi_b_bar).
template <typename T, int NC>
__global__ void __launch_bounds__(kBlock) k_grad_gauss_bwd(Topo t, Geo<T> g, int cls,
                                                           const T* __restrict__ gbar,
                                                           T* __restrict__ phibar,
                                                           T* __restrict__ phibbar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc, nb = t.nb;
  T ai[NC][3], acc[NC];
  const T ri = ldg(g.rV + i);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    acc[c] = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) ai[c][d] = ldg(gbar + (c * 3 + d) * nc + i) * ri;
  }
  const int e1 = ldg(t.cptr + i + 1);
  for (int e = ldg(t.cptr + i); e < e1; ++e) {
    const int ent = ldg(t.cent + e);
    const int f = ent >> 1;
    const V4<T> s = ld4(g.Sw + f);
    if (f < t.ni) {
      const int2 on = ldg(t.on + f);
      const bool nside = ent & 1;
      const int j = nside ? on.x : on.y;
      const T rj = ldg(g.rV + j);
      const T wi = nside ? (T(1) - s.w) : s.w;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T aj[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) aj[d] = ldg(gbar + (c * 3 + d) * nc + j) * rj;
        // (a_O - a_N).S
        T dO = (ai[c][0] - aj[0]) * s.x + (ai[c][1] - aj[1]) * s.y + (ai[c][2] - aj[2]) * s.z;
        if (nside) dO = -dO;
        acc[c] += wi * dO;
      }
    } else {
      const int b = f - t.ni;
      const int kind = face_kind(t, b, cls);
      if (kind == DIFVM_FACE_EMPTY) continue;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T v = ai[c][0] * s.x + ai[c][1] * s.y + ai[c][2] * s.z;
        if (kind == DIFVM_FACE_FIXED) {
          if (phibbar) phibbar[c * nb + b] += v;
        } else {
          acc[c] += v;
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) phibar[c * nc + i] += acc[c];
}

// ------------------------------------------------------------ convection
// out_i = sum_f sigma m_f phi_f   (Eqs. conv_face_flux, upwind; tie m=0 -> owner).
// The face flux (and, for the linear scheme, w_f) is read by face id.
template <typename T, int NC, bool UPWIND, int WK>
__device__ __forceinline__ void div_row(const Topo& t, const Hf& H, const HfGeo<T>& hg, int cls,
                                        const T* __restrict__ mf, const T* __restrict__ phi,
                                        const T* __restrict__ phib, T* __restrict__ out, int i) {
  const int nc = t.nc, nb = t.nb;
  T pi[NC], acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    pi[c] = ldg(phi + c * nc + i);
    acc[c] = T(0);
  }
  int base, w;
  hf_row_w<WK>(H, i, base, w);
  const int fb = hf_fbase(H, i);
  for (int k0 = 0; k0 < w; k0 += 4) {
    int v[4], f[4];
    hf_words<true>(H, i, fb, base, k0, w, v, f);
    T mk[4], wk[4], pj[4][NC];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      mk[k] = v[k] != -1 ? ldg(mf + f[k]) : T(0);
      wk[k] = (!UPWIND && v[k] >= 0) ? ldg(hg.w + f[k]) : T(0);
      hf_gather<T, NC>(v[k], cls, phi, phib, nc, nb, i, pj[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int vk = v[k];
      if (hf_skip(vk, cls)) continue;
      // mm: the face flux out of this cell (-m on the neighbour side, exactly);
      // the message mm * phi_f is then the owner's message or its exact negation
      const bool nside = vk >= 0 && (vk & 1);
      const T mm = nside ? -mk[k] : mk[k];
      if (UPWIND) {
        // upwind value: the own cell's on outflow, the other's on inflow (a
        // boundary face always carries its boundary value); at m = 0 the
        // message is a zero either way
        const bool oth = vk < 0 || mm < T(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += mul_rn(mm, oth ? pj[k][c] : pi[c]);
      } else if (vk >= 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T pO = nside ? pj[k][c] : pi[c], pN = nside ? pi[c] : pj[k][c];
          acc[c] += mul_rn(mm, wk[k] * pO + (T(1) - wk[k]) * pN);
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += mul_rn(mm, pj[k][c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) out[c * nc + i] = acc[c];
}

template <typename T, int NC, bool UPWIND, int WK, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_div_flux(Topo t, Hf H, HfGeo<T> hg, int cls,
                                                           const T* __restrict__ mf,
                                                           const T* __restrict__ phi,
                                                           const T* __restrict__ phib,
                                                           T* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < t.nc) div_row<T, NC, UPWIND, WK>(t, H, hg, cls, mf, phi, phib, out, i);
}

// Adjoint.  delta_f = obar_O - obar_N (internal) or obar_O (boundary):
//   mbar_f += sum_c phi_f delta_f  (written by the owner side / boundary entry)
//   phi_f's operands receive m delta_f with the scheme's weights.
template <typename T, int NC, bool UPWIND>
__global__ void __launch_bounds__(kBlock) k_div_flux_bwd(Topo t, Geo<T> g, int cls,
                                                         const T* __restrict__ mf,
                                                         const T* __restrict__ phi,
                                                         const T* __restrict__ phib,
                                                         const T* __restrict__ obar,
                                                         T* __restrict__ mbar,
                                                         T* __restrict__ phibar,
                                                         T* __restrict__ phibbar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc, nb = t.nb;
  T pi[NC], oi[NC], acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    pi[c] = ldg(phi + c * nc + i);
    oi[c] = ldg(obar + c * nc + i);
    acc[c] = T(0);
  }
  const int e1 = ldg(t.cptr + i + 1);
  for (int e = ldg(t.cptr + i); e < e1; ++e) {
    const int ent = ldg(t.cent + e);
    const int f = ent >> 1;
    const T m = ldg(mf + f);
    if (f < t.ni) {
      const int2 on = ldg(t.on + f);
      const bool nside = ent & 1;
      const int j = nside ? on.x : on.y;
      T w = T(0);
      if (!UPWIND) w = ld4(g.Sw + f).w;
      T macc = T(0);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T oj = ldg(obar + c * nc + j);
        const T delta = nside ? (oj - oi[c]) : (oi[c] - oj);
        T wi;
        if (UPWIND) wi = (m >= T(0)) == !nside ? T(1) : T(0);
        else wi = nside ? (T(1) - w) : w;
        acc[c] += wi * m * delta;
        if (mbar && !nside) {
          const T pj = ldg(phi + c * nc + j);
          const T pf = UPWIND ? (m >= T(0) ? pi[c] : pj) : w * pi[c] + (T(1) - w) * pj;
          macc += pf * delta;
        }
      }
      if (mbar && !nside) mbar[f] += macc;
    } else {
      const int b = f - t.ni;
      const int kind = face_kind(t, b, cls);
      if (kind == DIFVM_FACE_EMPTY) continue;
      T macc = T(0);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T pf = kind == DIFVM_FACE_FIXED ? ldg(phib + c * nb + b) : pi[c];
        macc += pf * oi[c];
        if (kind == DIFVM_FACE_FIXED) {
          if (phibbar) phibbar[c * nb + b] += m * oi[c];
        } else {
          acc[c] += m * oi[c];
        }
      }
      if (mbar) mbar[f] += macc;
    }
  }
  if (phibar) {
#pragma unroll
    for (int c = 0; c < NC; ++c) phibar[c * nc + i] += acc[c];
  }
}

// --------------------------------------------------------------- diffusion
// out_i = sum_f sigma gamma [c_f (phi_N - phi_O) + (grad phi)_f . k_f]   (Eq. nonortho_flux).
// (c, k) and w_f are read by face id.
template <typename T, int NC, bool NONORTH, int WK, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_laplacian(Topo t, Hf H, HfGeo<T> hg, int cls, T gamma,
                                                            const T* __restrict__ phi,
                                                            const T* __restrict__ phib,
                                                            const T* __restrict__ grad,
                                                            T* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc, nb = t.nb;
  T pi[NC], acc[NC], gi[NC][3];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    pi[c] = ldg(phi + c * nc + i);
    acc[c] = T(0);
    if (NONORTH)
#pragma unroll
      for (int d = 0; d < 3; ++d) gi[c][d] = ldg(grad + (c * 3 + d) * nc + i);
  }
  int base, w;
  hf_row_w<WK>(H, i, base, w);
  const int fb = hf_fbase(H, i);
  for (int k0 = 0; k0 < w; k0 += 4) {
    int v[4], f[4];
    hf_words<true>(H, i, fb, base, k0, w, v, f);
    V4<T> ck[4];
    T wk[4], pj[4][NC];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ck[k] = v[k] != -1 ? ld4(hg.ck + f[k]) : V4<T>{T(0), T(0), T(0), T(0)};
      wk[k] = (NONORTH && v[k] >= 0) ? ldg(hg.w + f[k]) : T(0);
      hf_gather<T, NC>(v[k], cls, phi, phib, nc, nb, i, pj[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int vk = v[k];
      if (vk == -1) continue;
      const V4<T> c4 = ck[k];
      if (vk >= 0) {
        const bool nside = vk & 1;
        const int j = vk >> 1;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T pO = nside ? pj[k][c] : pi[c], pN = nside ? pi[c] : pj[k][c];
          T F = c4.x * (pN - pO);
          if (NONORTH) {
            T gk = T(0);
            const T kk[3] = {c4.y, c4.z, c4.w};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const T gj = ldg(grad + (c * 3 + d) * nc + j);
              const T gO = nside ? gj : gi[c][d], gN = nside ? gi[c][d] : gj;
              gk += (wk[k] * gO + (T(1) - wk[k]) * gN) * kk[d];
            }
            F += gk;
          }
          F *= gamma;
          acc[c] += nside ? -F : F;
        }
      } else {
        if (hf_kind(vk, cls) != DIFVM_FACE_FIXED) continue;
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += gamma * (c4.x * (pj[k][c] - pi[c]));
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) out[c * nc + i] = acc[c];
}

// Adjoint: delta_f = obar_O - obar_N;  phi_N += gamma c delta, phi_O -= gamma c delta,
// grad_O += gamma w k delta, grad_N += gamma (1-w) k delta; fixed boundary: phi_b += gamma c obar_O.
template <typename T, int NC>
__global__ void __launch_bounds__(kBlock) k_laplacian_bwd(Topo t, Geo<T> g, int cls, T gamma,
                                                          const T* __restrict__ obar,
                                                          T* __restrict__ phibar,
                                                          T* __restrict__ phibbar,
                                                          T* __restrict__ gradbar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc, nb = t.nb;
  T oi[NC], acc[NC], gacc[NC][3];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    oi[c] = ldg(obar + c * nc + i);
    acc[c] = T(0);
    gacc[c][0] = gacc[c][1] = gacc[c][2] = T(0);
  }
  const int e1 = ldg(t.cptr + i + 1);
  for (int e = ldg(t.cptr + i); e < e1; ++e) {
    const int ent = ldg(t.cent + e);
    const int f = ent >> 1;
    const V4<T> ck = ld4(g.ck + f);
    if (f < t.ni) {
      const int2 on = ldg(t.on + f);
      const bool nside = ent & 1;
      const int j = nside ? on.x : on.y;
      const T w = ld4(g.Sw + f).w;
      const T wi = nside ? (T(1) - w) : w;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T oj = ldg(obar + c * nc + j);
        const T delta = gamma * (nside ? (oj - oi[c]) : (oi[c] - oj));
        acc[c] += nside ? ck.x * delta : -ck.x * delta;
        gacc[c][0] += wi * ck.y * delta;
        gacc[c][1] += wi * ck.z * delta;
        gacc[c][2] += wi * ck.w * delta;
      }
    } else {
      const int b = f - t.ni;
      if (face_kind(t, b, cls) != DIFVM_FACE_FIXED) continue;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T v = gamma * ck.x * oi[c];
        acc[c] -= v;
        if (phibbar) phibbar[c * nb + b] += v;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (phibar) phibar[c * nc + i] += acc[c];
    if (gradbar)
#pragma unroll
      for (int d = 0; d < 3; ++d) gradbar[(c * 3 + d) * nc + i] += gacc[c][d];
  }
}

// ---------------------------------------------------------------- LDU apply
// y_i = D_i x_i + sum_{O(f)=i} U_f x_N + sum_{N(f)=i} L_f x_O   (Eq. Ap_H)
template <typename T, int NC, int WK, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_ldu_apply(Topo t, Hf H, const T* __restrict__ D,
                                                            const T* __restrict__ L,
                                                            const T* __restrict__ U,
                                                            const T* __restrict__ x,
                                                            T* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.nc) return;
  const int nc = t.nc;
  const T d = ldg(D + i);
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = d * ldg(x + c * nc + i);
  int base, w;
  hf_row_w<WK>(H, i, base, w);
  const int fb = hf_fbase(H, i);
  for (int k0 = 0; k0 < w; k0 += 4) {
    int v[4], fk[4];
    hf_words<true>(H, i, fb, base, k0, w, v, fk);
    T ak[4], xk[4][NC];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ak[k] = v[k] >= 0 ? ((v[k] & 1) ? ldg(L + fk[k]) : ldg(U + fk[k])) : T(0);
#pragma unroll
      for (int c = 0; c < NC; ++c) xk[k][c] = v[k] >= 0 ? ldg(x + c * nc + (v[k] >> 1)) : T(0);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (v[k] < 0) continue;   // boundary faces and padding carry no off-diagonal entry
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] += ak[k] * xk[k][c];
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) y[c * nc + i] = acc[c];
}

// Coefficient adjoints of y = A x: Dbar_i += sum_c ybar_i x_i,
// Lbar_f += sum_c ybar_N x_O, Ubar_f += sum_c ybar_O x_N (SYM: both into Lbar).
template <typename T, int NC, bool SYM>
__global__ void k_ldu_coeff_bwd(Topo t, const T* __restrict__ x, const T* __restrict__ ybar,
                                T* __restrict__ Dbar, T* __restrict__ Lbar, T* __restrict__ Ubar) {
  const int nc = t.nc;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < t.ni) {
    const int2 on = ldg(t.on + k);
    T lb = T(0), ub = T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      lb += ldg(ybar + c * nc + on.y) * ldg(x + c * nc + on.x);
      ub += ldg(ybar + c * nc + on.x) * ldg(x + c * nc + on.y);
    }
    if (SYM) {
      if (Lbar) Lbar[k] += lb + ub;
    } else {
      if (Lbar) Lbar[k] += lb;
      if (Ubar) Ubar[k] += ub;
    }
  }
  if (Dbar && k < nc) {
    T db = T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) db += ldg(ybar + c * nc + k) * ldg(x + c * nc + k);
    Dbar[k] += db;
  }
}

template <typename T> __global__ void k_axpy_inplace(int n, const T* __restrict__ a, T* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] += a[i];
}

// ---------------------------------------------------------------- dispatch
#define DIFVM_NC_SWITCH(nc, ...)                      \
  switch (nc) {                                       \
    case 1: { constexpr int NCc = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int NCc = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int NCc = 3; __VA_ARGS__; } break; \
    default: return set_error(DIFVM_EINVAL, "ncomp must be 1..3 (got %d)", nc); \
  }

static difvm_status check_common(difvm_mesh_t m, difvm_prec prec, int ncomp) {
  DIFVM_TRY(check_mesh(m));
  DIFVM_TRY(check_prec(prec));
  if (ncomp < 1 || ncomp > 3) return set_error(DIFVM_EINVAL, "ncomp must be 1..3 (got %d)", ncomp);
  return DIFVM_OK;
}

static difvm_status check_cls(int cls) {
  if (cls < 0 || cls > 3) return set_error(DIFVM_EINVAL, "bad bc class %d", cls);
  return DIFVM_OK;
}

// Face records by slot (the Sw copies of the half-face layout: coalesced, no
// face-id load; the Gauss gradient) or by face id from the face arrays (each
// record read from DRAM once, its second visit an L2 hit within the RCM
// bandwidth; the kernels that load the face id anyway).  Chosen per kernel by
// measurement on the 1.6M-cell Kuhn mesh.
template <typename T> static HfGeo<T> fgeo(const difvm_mesh* m) {
  const Geo<T> g = geo<T>(m);
  return HfGeo<T>{g.Sw, g.ck, hfgeo<T>(m).w};
}

// ------------------------------------------------------------- autotuning
// The F32 kernels of the uniform tetrahedral layout (four slots per row) come
// in launch variants that differ in the register budget the compiler must meet:
// variant 0 lets it choose (one block per SM guaranteed), 1 and 2 force six and
// eight resident 256-thread blocks per SM (the Gauss gradient's variant 1 reads
// its geometry by face id instead).  More resident warps hide more of the
// gather latency but may spill; which variant wins depends on the operator,
// the component count and the mesh.  So the first call of each (operator,
// components, scheme) on a mesh times every variant on that call's own
// arguments (a forward operator only writes its output, so running it again
// changes nothing) and the mesh keeps the fastest, the default unless another
// is at least 2% faster; later calls launch it.  A
// first call under stream capture (no timing possible) launches the default
// variant without recording a choice.  difvm_mesh_autotune switches timing off
// (every call then launches the default) or clears the kept choices.
constexpr int kVariants = 3;
enum { kOpGrad = 1, kOpDiv = 2, kOpLap = 3, kOpLdu = 4 };
static uint32_t tune_key(int op, int extra, int nc) { return (uint32_t)(op << 8 | extra << 4 | nc); }

static int tuned_variant(const difvm_mesh* m, uint32_t key) {
  for (const auto& kv : m->tuned)
    if (kv.first == key) return kv.second;
  return -1;
}

template <typename F>
static difvm_status tuned_launch(difvm_mesh* m, uint32_t key, int dflt, cudaStream_t s, F&& launch) {
  int var = tuned_variant(m, key);
  if (var < 0 && m->autotune && !stream_capturing(s)) {
    constexpr int kReps = 5;
    cudaEvent_t ev[kVariants][2];
    for (int v = 0; v < kVariants; ++v)
      for (int e = 0; e < 2; ++e) DIFVM_CUDA(cudaEventCreate(&ev[v][e]));
    difvm_status st = DIFVM_OK;
    for (int v = 0; v < kVariants && st == DIFVM_OK; ++v) {
      launch(v);                       // first launch of the variant: not timed
      cudaEventRecord(ev[v][0], s);
      for (int r = 0; r < kReps; ++r) launch(v);
      cudaEventRecord(ev[v][1], s);
      st = check_error("autotune");
    }
    // the default stays unless another variant is at least 2% faster (the
    // timing of a few launches varies by about that much)
    float t[kVariants] = {};
    for (int v = 0; v < kVariants && st == DIFVM_OK; ++v)
      if (cudaEventSynchronize(ev[v][1]) != cudaSuccess ||
          cudaEventElapsedTime(&t[v], ev[v][0], ev[v][1]) != cudaSuccess)
        st = set_error(DIFVM_ECUDA, "autotune timing failed");
    if (st == DIFVM_OK) {
      var = dflt;
      for (int v = 0; v < kVariants; ++v)
        if (t[v] < 0.98f * t[var]) var = v;
    }
    for (int v = 0; v < kVariants; ++v)
      for (int e = 0; e < 2; ++e) cudaEventDestroy(ev[v][e]);
    DIFVM_TRY(st);
    m->tuned.emplace_back(key, var);
  }
  launch(var < 0 ? dflt : var);
  return DIFVM_OK;
}

template <typename T>
difvm_status grad_gauss_t(difvm_mesh_t m, int cls, const void* phi, const void* phib,
                          int ncomp, void* grad, cudaStream_t s) {
  const unsigned B = blocks_for(m->nc, kBlock);
  const auto args = [&](auto k) {
    k<<<B, kBlock, 0, s>>>(m->topo(), m->hf(), hfgeo<T>(m), geo<T>(m), cls, (const T*)phi, (const T*)phib,
                           (T*)grad);
  };
  if (sizeof(T) == 4 && m->hf_w == 4) {
    DIFVM_NC_SWITCH(ncomp, DIFVM_TRY(tuned_launch(m, tune_key(kOpGrad, 0, NCc), 0, s, [&](int var) {
      switch (var) {
        case 0: args(k_grad_gauss<T, NCc, 4, 1>); break;
        case 1: args(k_grad_gauss<T, NCc, 4, 1, true>); break;
        default: args(k_grad_gauss<T, NCc, 4, 8>); break;
      }
    })));
  } else if (m->hf_w == 4) {
    DIFVM_NC_SWITCH(ncomp, args(k_grad_gauss<T, NCc, 4, 1>));
  } else {
    DIFVM_NC_SWITCH(ncomp, args(k_grad_gauss<T, NCc, 0, 1>));
  }
  return check_launch("grad_gauss");
}
template difvm_status grad_gauss_t<float>(difvm_mesh_t, int, const void*, const void*, int, void*,
                                          cudaStream_t);
template difvm_status grad_gauss_t<double>(difvm_mesh_t, int, const void*, const void*, int, void*,
                                           cudaStream_t);

template <typename T>
static difvm_status grad_gauss_bwd_t(difvm_mesh_t m, int cls, const void* gbar, int ncomp,
                                     void* phibar, void* phibbar, cudaStream_t s) {
  DIFVM_NC_SWITCH(ncomp, k_grad_gauss_bwd<T, NCc><<<blocks_for(m->nc, kBlock), kBlock, 0, s>>>(
                             m->topo(), geo<T>(m), cls, (const T*)gbar, (T*)phibar, (T*)phibbar));
  return check_launch("grad_gauss_bwd");
}

template <typename T, bool UPWIND>
static difvm_status div_flux_s(difvm_mesh_t m, int cls, const void* mf, const void* phi, const void* phib,
                               int ncomp, void* out, cudaStream_t s) {
  const unsigned B = blocks_for(m->nc, kBlock);
  const auto args = [&](auto k) {
    k<<<B, kBlock, 0, s>>>(m->topo(), m->hf(), fgeo<T>(m), cls, (const T*)mf, (const T*)phi, (const T*)phib,
                           (T*)out);
  };
  if (sizeof(T) == 4 && m->hf_w == 4) {
    DIFVM_NC_SWITCH(ncomp, DIFVM_TRY(tuned_launch(m, tune_key(kOpDiv, UPWIND, NCc), UPWIND ? 1 : 0, s,
                                                  [&](int var) {
      switch (var) {
        case 0: args(k_div_flux<T, NCc, UPWIND, 4, 1>); break;
        case 1: args(k_div_flux<T, NCc, UPWIND, 4, 6>); break;
        default: args(k_div_flux<T, NCc, UPWIND, 4, 8>); break;
      }
    })));
  } else if (m->hf_w == 4) {
    DIFVM_NC_SWITCH(ncomp, args(k_div_flux<T, NCc, UPWIND, 4, 1>));
  } else {
    DIFVM_NC_SWITCH(ncomp, args(k_div_flux<T, NCc, UPWIND, 0, 1>));
  }
  return check_launch("div_flux");
}
template <typename T>
static difvm_status div_flux_t(difvm_mesh_t m, int scheme, int cls, const void* mf,
                               const void* phi, const void* phib, int ncomp, void* out,
                               cudaStream_t s) {
  return scheme == DIFVM_DIV_UPWIND ? div_flux_s<T, true>(m, cls, mf, phi, phib, ncomp, out, s)
                                    : div_flux_s<T, false>(m, cls, mf, phi, phib, ncomp, out, s);
}

template <typename T>
static difvm_status div_flux_bwd_t(difvm_mesh_t m, int scheme, int cls, const void* mf,
                                   const void* phi, const void* phib, int ncomp, const void* obar,
                                   void* mbar, void* phibar, void* phibbar, cudaStream_t s) {
  if (scheme == DIFVM_DIV_UPWIND) {
    DIFVM_NC_SWITCH(ncomp, k_div_flux_bwd<T, NCc, true><<<blocks_for(m->nc, kBlock), kBlock, 0, s>>>(
                               m->topo(), geo<T>(m), cls, (const T*)mf, (const T*)phi,
                               (const T*)phib, (const T*)obar, (T*)mbar, (T*)phibar, (T*)phibbar));
  } else {
    DIFVM_NC_SWITCH(ncomp, k_div_flux_bwd<T, NCc, false><<<blocks_for(m->nc, kBlock), kBlock, 0, s>>>(
                               m->topo(), geo<T>(m), cls, (const T*)mf, (const T*)phi,
                               (const T*)phib, (const T*)obar, (T*)mbar, (T*)phibar, (T*)phibbar));
  }
  return check_launch("div_flux_bwd");
}

template <typename T, bool NONORTH>
static difvm_status laplacian_s(difvm_mesh_t m, int cls, double gamma, const void* phi, const void* phib,
                                const void* grad, int ncomp, void* out, cudaStream_t s) {
  const unsigned B = blocks_for(m->nc, kBlock);
  const auto args = [&](auto k) {
    k<<<B, kBlock, 0, s>>>(m->topo(), m->hf(), fgeo<T>(m), cls, (T)gamma, (const T*)phi, (const T*)phib,
                           (const T*)grad, (T*)out);
  };
  if (sizeof(T) == 4 && m->hf_w == 4) {
    DIFVM_NC_SWITCH(ncomp, DIFVM_TRY(tuned_launch(m, tune_key(kOpLap, NONORTH, NCc), 0, s, [&](int var) {
      switch (var) {
        case 0: args(k_laplacian<T, NCc, NONORTH, 4, 1>); break;
        case 1: args(k_laplacian<T, NCc, NONORTH, 4, 6>); break;
        default: args(k_laplacian<T, NCc, NONORTH, 4, 8>); break;
      }
    })));
  } else if (m->hf_w == 4) {
    DIFVM_NC_SWITCH(ncomp, args(k_laplacian<T, NCc, NONORTH, 4, 1>));
  } else {
    DIFVM_NC_SWITCH(ncomp, args(k_laplacian<T, NCc, NONORTH, 0, 1>));
  }
  return check_launch("laplacian");
}
template <typename T>
static difvm_status laplacian_t(difvm_mesh_t m, int cls, double gamma, const void* phi,
                                const void* phib, const void* grad, int ncomp, void* out,
                                cudaStream_t s) {
  return grad ? laplacian_s<T, true>(m, cls, gamma, phi, phib, grad, ncomp, out, s)
              : laplacian_s<T, false>(m, cls, gamma, phi, phib, nullptr, ncomp, out, s);
}

template <typename T>
static difvm_status laplacian_bwd_t(difvm_mesh_t m, int cls, double gamma, const void* obar,
                                    int ncomp, void* phibar, void* phibbar, void* gradbar,
                                    cudaStream_t s) {
  DIFVM_NC_SWITCH(ncomp, k_laplacian_bwd<T, NCc><<<blocks_for(m->nc, kBlock), kBlock, 0, s>>>(
                             m->topo(), geo<T>(m), cls, (T)gamma, (const T*)obar, (T*)phibar,
                             (T*)phibbar, (T*)gradbar));
  return check_launch("laplacian_bwd");
}

template <typename T>
difvm_status ldu_apply_t(difvm_mesh_t m, const void* D, const void* L, const void* U,
                         const void* x, int ncomp, int transpose, void* y, cudaStream_t s) {
  const T* Lp = (const T*)L;
  const T* Up = U ? (const T*)U : Lp;
  if (transpose) std::swap(Lp, Up);
  const unsigned B = blocks_for(m->nc, kBlock);
  const auto args = [&](auto k) { k<<<B, kBlock, 0, s>>>(m->topo(), m->hf(), (const T*)D, Lp, Up, (const T*)x, (T*)y); };
  if (sizeof(T) == 4 && m->hf_w == 4) {
    DIFVM_NC_SWITCH(ncomp, DIFVM_TRY(tuned_launch(m, tune_key(kOpLdu, 0, NCc), 0, s, [&](int var) {
      switch (var) {
        case 0: args(k_ldu_apply<T, NCc, 4, 1>); break;
        case 1: args(k_ldu_apply<T, NCc, 4, 6>); break;
        default: args(k_ldu_apply<T, NCc, 4, 8>); break;
      }
    })));
  } else if (m->hf_w == 4) {
    DIFVM_NC_SWITCH(ncomp, args(k_ldu_apply<T, NCc, 4, 1>));
  } else {
    DIFVM_NC_SWITCH(ncomp, args(k_ldu_apply<T, NCc, 0, 1>));
  }
  return check_launch("ldu_apply");
}
template difvm_status ldu_apply_t<float>(difvm_mesh_t, const void*, const void*, const void*,
                                         const void*, int, int, void*, cudaStream_t);
template difvm_status ldu_apply_t<double>(difvm_mesh_t, const void*, const void*, const void*,
                                          const void*, int, int, void*, cudaStream_t);

template <typename T>
static difvm_status ldu_apply_bwd_t(difvm_mesh_t m, const void* D, const void* L, const void* U,
                                    const void* x, const void* ybar, int ncomp, void* xbar,
                                    void* Dbar, void* Lbar, void* Ubar, void* tmp, cudaStream_t s) {
  if (xbar) {
    DIFVM_TRY(ldu_apply_t<T>(m, D, L, U, ybar, ncomp, 1, tmp, s));
    k_axpy_inplace<T><<<blocks_for((int64_t)ncomp * m->nc, kBlock), kBlock, 0, s>>>(
        ncomp * m->nc, (const T*)tmp, (T*)xbar);
    DIFVM_TRY(check_launch("axpy"));
  }
  if (Dbar || Lbar || Ubar) {
    int n = std::max(m->ni, m->nc);
    if (U) {
      DIFVM_NC_SWITCH(ncomp, k_ldu_coeff_bwd<T, NCc, false><<<blocks_for(n, kBlock), kBlock, 0, s>>>(
                                 m->topo(), (const T*)x, (const T*)ybar, (T*)Dbar, (T*)Lbar, (T*)Ubar));
    } else {
      DIFVM_NC_SWITCH(ncomp, k_ldu_coeff_bwd<T, NCc, true><<<blocks_for(n, kBlock), kBlock, 0, s>>>(
                                 m->topo(), (const T*)x, (const T*)ybar, (T*)Dbar, (T*)Lbar, nullptr));
    }
    DIFVM_TRY(check_launch("ldu_coeff_bwd"));
  }
  return DIFVM_OK;
}

}  // namespace difvm

using namespace difvm;

#define DIFVM_PREC_DISPATCH(prec, fn, ...)                      \
  ((prec) == DIFVM_F64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

extern "C" difvm_status difvm_grad_gauss(difvm_mesh_t m, difvm_prec prec, int cls, const void* phi,
                                         const void* phib, int ncomp, void* grad, void* stream) {
  DIFVM_TRY(check_common(m, prec, ncomp));
  DIFVM_TRY(check_cls(cls));
  if (!phi || !grad) return set_error(DIFVM_EINVAL, "null field");
  return DIFVM_PREC_DISPATCH(prec, grad_gauss_t, m, cls, phi, phib, ncomp, grad, (cudaStream_t)stream);
}

extern "C" difvm_status difvm_grad_gauss_bwd(difvm_mesh_t m, difvm_prec prec, int cls,
                                             const void* gbar, int ncomp, void* phibar,
                                             void* phibbar, void* stream) {
  DIFVM_TRY(check_common(m, prec, ncomp));
  DIFVM_TRY(check_cls(cls));
  if (!gbar || !phibar) return set_error(DIFVM_EINVAL, "null field");
  return DIFVM_PREC_DISPATCH(prec, grad_gauss_bwd_t, m, cls, gbar, ncomp, phibar, phibbar,
                             (cudaStream_t)stream);
}

extern "C" difvm_status difvm_div_flux(difvm_mesh_t m, difvm_prec prec, int scheme, int cls,
                                       const void* mf, const void* phi, const void* phib, int ncomp,
                                       void* out, void* stream) {
  DIFVM_TRY(check_common(m, prec, ncomp));
  DIFVM_TRY(check_cls(cls));
  if (scheme != DIFVM_DIV_UPWIND && scheme != DIFVM_DIV_LINEAR)
    return set_error(DIFVM_EINVAL, "bad scheme %d", scheme);
  if (!mf || !phi || !out) return set_error(DIFVM_EINVAL, "null field");
  return DIFVM_PREC_DISPATCH(prec, div_flux_t, m, scheme, cls, mf, phi, phib, ncomp, out,
                             (cudaStream_t)stream);
}

extern "C" difvm_status difvm_div_flux_bwd(difvm_mesh_t m, difvm_prec prec, int scheme, int cls,
                                           const void* mf, const void* phi, const void* phib,
                                           int ncomp, const void* obar, void* mbar, void* phibar,
                                           void* phibbar, void* stream) {
  DIFVM_TRY(check_common(m, prec, ncomp));
  DIFVM_TRY(check_cls(cls));
  if (scheme != DIFVM_DIV_UPWIND && scheme != DIFVM_DIV_LINEAR)
    return set_error(DIFVM_EINVAL, "bad scheme %d", scheme);
  if (!mf || !phi || !obar) return set_error(DIFVM_EINVAL, "null field");
  return DIFVM_PREC_DISPATCH(prec, div_flux_bwd_t, m, scheme, cls, mf, phi, phib, ncomp, obar,
                             mbar, phibar, phibbar, (cudaStream_t)stream);
}

extern "C" difvm_status difvm_laplacian(difvm_mesh_t m, difvm_prec prec, int cls, double gamma,
                                        const void* phi, const void* phib, const void* grad,
                                        int ncomp, void* out, void* stream) {
  DIFVM_TRY(check_common(m, prec, ncomp));
  DIFVM_TRY(check_cls(cls));
  if (!phi || !out) return set_error(DIFVM_EINVAL, "null field");
  return DIFVM_PREC_DISPATCH(prec, laplacian_t, m, cls, gamma, phi, phib, grad, ncomp, out,
                             (cudaStream_t)stream);
}

extern "C" difvm_status difvm_laplacian_bwd(difvm_mesh_t m, difvm_prec prec, int cls, double gamma,
                                            const void* obar, int ncomp, void* phibar,
                                            void* phibbar, void* gradbar, void* stream) {
  DIFVM_TRY(check_common(m, prec, ncomp));
  DIFVM_TRY(check_cls(cls));
  if (!obar) return set_error(DIFVM_EINVAL, "null field");
  return DIFVM_PREC_DISPATCH(prec, laplacian_bwd_t, m, cls, gamma, obar, ncomp, phibar, phibbar,
                             gradbar, (cudaStream_t)stream);
}

extern "C" difvm_status difvm_laplacian_apply(difvm_mesh_t m, difvm_prec prec, const void* D,
                                              const void* L, const void* U, const void* x,
                                              int ncomp, int transpose, void* y, void* stream) {
  DIFVM_TRY(check_common(m, prec, ncomp));
  if (!D || (!L && m->ni > 0) || !x || !y) return set_error(DIFVM_EINVAL, "null field");
  if (x == y) return set_error(DIFVM_EINVAL, "x and y must not alias");
  return DIFVM_PREC_DISPATCH(prec, ldu_apply_t, m, D, L, U, x, ncomp, transpose, y,
                             (cudaStream_t)stream);
}

extern "C" difvm_status difvm_laplacian_apply_bwd(difvm_mesh_t m, difvm_prec prec, const void* D,
                                                  const void* L, const void* U, const void* x,
                                                  const void* ybar, int ncomp, void* xbar,
                                                  void* Dbar, void* Lbar, void* Ubar, void* tmp,
                                                  void* stream) {
  DIFVM_TRY(check_common(m, prec, ncomp));
  if (!D || (!L && m->ni > 0) || !x || !ybar) return set_error(DIFVM_EINVAL, "null field");
  if (xbar && !tmp) return set_error(DIFVM_EINVAL, "x_bar needs a [ncomp][nc] scratch buffer");
  return DIFVM_PREC_DISPATCH(prec, ldu_apply_bwd_t, m, D, L, U, x, ybar, ncomp, xbar, Dbar, Lbar,
                             Ubar, tmp, (cudaStream_t)stream);
}

extern "C" difvm_status difvm_mesh_autotune(difvm_mesh_t m, int mode) {
  DIFVM_TRY(check_mesh(m));
  if (mode < 0 || mode > 2) return set_error(DIFVM_EINVAL, "autotune mode must be 0, 1 or 2 (got %d)", mode);
  if (mode == 2) m->tuned.clear();
  m->autotune = mode != 0;
  amg_retune(m, mode);
  return DIFVM_OK;
}

extern "C" difvm_status difvm_mesh_tuning(difvm_mesh_t m, uint32_t* keys, int32_t* variants, int cap,
                                          int32_t* count) {
  DIFVM_TRY(check_mesh(m));
  if (!count || cap < 0 || (cap > 0 && (!keys || !variants))) return set_error(DIFVM_EINVAL, "bad output arrays");
  const int n = (int)m->tuned.size();
  for (int k = 0; k < n && k < cap; ++k) {
    keys[k] = m->tuned[k].first;
    variants[k] = m->tuned[k].second;
  }
  *count = n;
  return DIFVM_OK;
}
