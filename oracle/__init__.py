"""CPU oracle of the DiFVM face-operator / PISO path -- TEST INFRASTRUCTURE.

A plain, slow FP64 implementation written from the paper (arxiv 2603.15920,
Sec. 2.3-2.6) in ``difvm_oracle.c`` and loaded here through ctypes.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library: the two meet
only in the seeded inputs of ``paper_2603_15920_b300.meshgen``, which this
package does not import either (callers pass plain numpy arrays).

Every function works in the mesh's own (input) numbering, component-major
fields ``[ncomp, nc]``, boundary values ``[ncomp, nb]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "difvm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BC_FIXED, BC_ZEROGRAD, BC_EMPTY = 0, 1, 2
PT_WALL, PT_INLET, PT_OUTLET, PT_EMPTY = 0, 1, 2, 3
DIV_UPWIND, DIV_LINEAR = 0, 1
WK_EXACT, WK_FE, WK_BE = 0, 1, 2
# split of S_f = Delta_f + k_f in Eq. nonortho_flux
NONORTH_OVERRELAXED, NONORTH_MINIMUM, NONORTH_ORTHOGONAL, NONORTH_NONE = 0, 1, 2, 3
# momentum convection: upwind, or second-order upwind by deferred correction (Eqs. deferred_correction, sou)
CONV_UPWIND, CONV_SOU = 0, 1
# momentum time scheme: backward Euler or Crank-Nicolson
TIME_BE, TIME_CN = 0, 1


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def _compile(out, extra):
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -ffp-contract=off, no FMA contraction), and
    its multi-core build (the same source with -fopenmp) used only by the
    all-cores CPU baseline."""
    if force:
        for f in (_LIB, _LIB_OMP):
            if os.path.exists(f):
                os.remove(f)
    _compile(_LIB_OMP, ["-fopenmp"])
    return _compile(_LIB, [])


_lib = None
_use_omp = False


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB_OMP if _use_omp else _LIB)
    return _lib


def use_multicore(on: bool = True):
    """Switch every following oracle call to the multi-core build (True) or
    back to the single-thread oracle (False).  Returns the thread count."""
    global _lib, _use_omp
    if on != _use_omp:
        _use_omp, _lib = on, None
    return threads()


def threads() -> int:
    """Threads the selected build runs on (1 for the single-thread oracle)."""
    return int(lib().om_threads())


def set_threads(n: int) -> int:
    """Thread count of the multi-core build (no effect on the single-thread one)."""
    lib().om_set_threads(int(n))
    return threads()


class _Mesh(C.Structure):
    _fields_ = [("nc", C.c_int), ("nint", C.c_int), ("nf", C.c_int), ("npatch", C.c_int),
                ("owner", C.c_void_p), ("neighbour", C.c_void_p),
                ("Sf", C.c_void_p), ("Cf", C.c_void_p), ("V", C.c_void_p), ("C", C.c_void_p),
                ("patch_start", C.c_void_p), ("patch_size", C.c_void_p),
                ("patch_type", C.c_void_p), ("nonorth", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("res0", C.c_double), ("res", C.c_double),
                ("bnorm", C.c_double), ("status", C.c_int)]


class _PisoOpts(C.Structure):
    _fields_ = [("nu", C.c_double), ("dt", C.c_double), ("ncorr", C.c_int), ("nonorth", C.c_int),
                ("tolU", C.c_double), ("tolp", C.c_double), ("tol_abs", C.c_double),
                ("maxitU", C.c_int), ("maxitp", C.c_int), ("pref_cell", C.c_int),
                ("wk_scheme", C.c_int), ("n_out", C.c_int), ("wk_patch", C.c_void_p),
                ("Rp", C.c_void_p), ("Cw", C.c_void_p), ("Rd", C.c_void_p), ("psi", C.c_double),
                ("conv", C.c_int), ("time", C.c_int)]


class _PisoInfo(C.Structure):
    _fields_ = [("itU", C.c_int * 3), ("itp", C.c_int * 4), ("status", C.c_int),
                ("Q", C.c_double * 8), ("po", C.c_double * 8)]


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OMesh:
    """Holds the oracle's view of a mesh (plain arrays, input numbering)."""

    def __init__(self, n_cells, n_internal, owner, neighbour, Sf, Cf, V, Cc,
                 patch_start, patch_size, patch_type, nonorth=0):
        self.keep = [_i32(owner), _i32(neighbour), _f64(Sf), _f64(Cf), _f64(V), _f64(Cc),
                     _i32(patch_start), _i32(patch_size), _i32(patch_type)]
        o, n, S, X, Vv, Cv, ps, pz, pt = self.keep
        self.nc, self.nint, self.nf = int(n_cells), int(n_internal), int(o.shape[0])
        self.nb = self.nf - self.nint
        self.npatch = int(ps.shape[0])
        self.patch_start, self.patch_size, self.patch_type = ps, pz, pt
        self.nonorth = int(nonorth)
        self.s = _Mesh(self.nc, self.nint, self.nf, self.npatch, _p(o), _p(n), _p(S), _p(X),
                       _p(Vv), _p(Cv), _p(ps), _p(pz), _p(pt), self.nonorth)

    @classmethod
    def from_mesh(cls, m, nonorth=0):
        """nonorth: the split of S_f in Eq. nonortho_flux, NONORTH_OVERRELAXED (the
        paper's default), NONORTH_MINIMUM, NONORTH_ORTHOGONAL or NONORTH_NONE."""
        return cls(m.n_cells, m.n_internal, m.owner, m.neighbour, m.Sf, m.Cf, m.V, m.C,
                   m.patch_start, m.patch_size, m.patch_type, nonorth)

    def ref(self):
        return C.byref(self.s)

    def bc_U(self):
        return np.array([BC_EMPTY if t == PT_EMPTY else (BC_ZEROGRAD if t == PT_OUTLET else BC_FIXED)
                         for t in self.patch_type], np.int32)

    def bc_p(self):
        return np.array([BC_EMPTY if t == PT_EMPTY else (BC_FIXED if t == PT_OUTLET else BC_ZEROGRAD)
                         for t in self.patch_type], np.int32)


def face_coeffs(m: OMesh):
    w = np.zeros(m.nint + 1); c = np.zeros(m.nf + 1); k = np.zeros(3 * (m.nint + 1))
    lib().om_face_coeffs(m.ref(), _p(w), _p(c), _p(k))
    return w[:m.nint], c[:m.nf], k[:3 * m.nint].reshape(m.nint, 3)


def check_geometry(m: OMesh):
    cl = C.c_double(0)
    bad = lib().om_check_geometry(m.ref(), _p(m.bc_U()), C.byref(cl))
    return int(bad), float(cl.value)


def _bcarr(bc, m):
    return _i32(np.broadcast_to(np.asarray(bc, np.int32), (m.npatch,)))


def grad_gauss(m: OMesh, bc, phi, phi_b=None):
    phi = _f64(np.atleast_2d(phi)); nq = phi.shape[0]
    pb = None if phi_b is None else _f64(np.reshape(phi_b, (nq, m.nb)))
    out = np.zeros((nq, 3, m.nc))
    lib().om_grad_gauss(m.ref(), _p(_bcarr(bc, m)), nq, _p(phi), _p(pb), _p(out))
    return out


def div_flux(m: OMesh, bc, scheme, mf, phi, phi_b=None):
    phi = _f64(np.atleast_2d(phi)); nq = phi.shape[0]
    pb = None if phi_b is None else _f64(np.reshape(phi_b, (nq, m.nb)))
    out = np.zeros((nq, m.nc))
    lib().om_div_flux(m.ref(), _p(_bcarr(bc, m)), int(scheme), nq, _p(_f64(mf)), _p(phi),
                      _p(pb), _p(out))
    return out


def laplacian(m: OMesh, bc, gamma, phi, phi_b=None, grad=None):
    phi = _f64(np.atleast_2d(phi)); nq = phi.shape[0]
    pb = None if phi_b is None else _f64(np.reshape(phi_b, (nq, m.nb)))
    g = None if grad is None else _f64(np.reshape(grad, (nq, 3, m.nc)))
    out = np.zeros((nq, m.nc))
    lib().om_laplacian(m.ref(), _p(_bcarr(bc, m)), nq, C.c_double(gamma), _p(phi), _p(pb),
                       _p(g), _p(out))
    return out


def ldu_apply(m: OMesh, D, L, U, x):
    x = _f64(np.atleast_2d(x)); nq = x.shape[0]
    y = np.zeros_like(x)
    lib().om_ldu_apply(m.ref(), nq, _p(_f64(D)), _p(_f64(L)),
                       _p(None if U is None else _f64(U)), _p(x), _p(y))
    return y


def _solve(fn, m, D, L, U, b, x0, tol_rel, tol_abs, maxit):
    x = _f64(np.zeros(m.nc) if x0 is None else np.array(x0, np.float64))
    info = _Info()
    getattr(lib(), fn)(m.ref(), _p(_f64(D)), _p(_f64(L)), _p(None if U is None else _f64(U)),
                       _p(_f64(b)), _p(x), C.c_double(tol_rel), C.c_double(tol_abs), int(maxit),
                       C.byref(info))
    return x, dict(iters=info.iters, res0=info.res0, res=info.res, bnorm=info.bnorm,
                   status=info.status)


def pcg(m, D, L, U, b, x0=None, tol_rel=1e-10, tol_abs=0.0, maxit=10000):
    return _solve("om_pcg", m, D, L, U, b, x0, tol_rel, tol_abs, maxit)


def dic_factor(m, D, L, rank):
    """The diagonal d of the DIC factorisation in the elimination order rank[i]."""
    d = np.zeros(m.nc)
    lib().om_dic_factor(m.ref(), _p(_f64(D)), _p(_f64(np.concatenate([L, [0.0]]))), _p(_i32(rank)), _p(d))
    return d


def pcg_dic(m, D, L, b, rank, x0=None, tol_rel=1e-10, tol_abs=0.0, maxit=10000):
    """CG preconditioned by diagonal incomplete Cholesky, cells eliminated in the
    order rank[i] (symmetric matrix: D, L)."""
    x = np.zeros(m.nc) if x0 is None else np.array(x0, np.float64)
    info = _Info()
    lib().om_pcg_dic(m.ref(), _p(_f64(D)), _p(_f64(np.concatenate([L, [0.0]]))), _p(_i32(rank)),
                     _p(_f64(b)), _p(x), C.c_double(tol_rel), C.c_double(tol_abs), int(maxit), C.byref(info))
    return x, dict(iters=info.iters, res0=info.res0, res=info.res, bnorm=info.bnorm, status=info.status)


def dilu_factor(m, D, L, U, rank):
    """The diagonal d of the DILU factorisation (non-symmetric L, U) in the
    elimination order rank[i]."""
    d = np.zeros(m.nc)
    lib().om_dilu_factor(m.ref(), _p(_f64(D)), _p(_f64(np.concatenate([L, [0.0]]))),
                         _p(_f64(np.concatenate([U, [0.0]]))), _p(_i32(rank)), _p(d))
    return d


def dilu_apply(m, D, L, U, rank, r):
    """z = M^-1 r with the DILU preconditioner M in the order rank[i]."""
    z = np.zeros(m.nc)
    lib().om_dilu_apply(m.ref(), _p(_f64(D)), _p(_f64(np.concatenate([L, [0.0]]))),
                        _p(_f64(np.concatenate([U, [0.0]]))), _p(_i32(rank)), _p(_f64(r)), _p(z))
    return z


def bicgstab_dilu(m, D, L, U, b, rank, x0=None, tol_rel=1e-10, tol_abs=0.0, maxit=10000):
    """BiCGStab right-preconditioned by DILU, cells eliminated in the order rank[i]."""
    x = np.zeros(m.nc) if x0 is None else np.array(x0, np.float64)
    info = _Info()
    lib().om_bicgstab_dilu(m.ref(), _p(_f64(D)), _p(_f64(np.concatenate([L, [0.0]]))),
                           _p(_f64(np.concatenate([U, [0.0]]))), _p(_i32(rank)), _p(_f64(b)), _p(x),
                           C.c_double(tol_rel), C.c_double(tol_abs), int(maxit), C.byref(info))
    return x, dict(iters=info.iters, res0=info.res0, res=info.res, bnorm=info.bnorm, status=info.status)


def bicgstab(m, D, L, U, b, x0=None, tol_rel=1e-10, tol_abs=0.0, maxit=10000):
    return _solve("om_bicgstab", m, D, L, U, b, x0, tol_rel, tol_abs, maxit)


def windkessel_update(scheme, Rp, Cw, Rd, Q, dt, pc):
    Rp, Cw, Rd, Q = (_f64(np.atleast_1d(a)) for a in (Rp, Cw, Rd, Q))
    pc = _f64(np.array(np.atleast_1d(pc), np.float64))
    po = np.zeros_like(pc)
    lib().om_windkessel_update(int(pc.shape[0]), int(scheme), _p(Rp), _p(Cw), _p(Rd), _p(Q),
                               C.c_double(dt), _p(pc), _p(po))
    return pc, po


def momentum_assemble(m: OMesh, nu, dt, mf, Uold, Ub, gradU=None, psi=1.0, gradS=None,
                      time=TIME_BE):
    """gradU: the non-orthogonal correction's velocity gradient; gradS: the
    gradient of the second-order upwind deferred correction (None: upwind);
    time: TIME_BE or TIME_CN (the Crank-Nicolson form of the rows)."""
    D = np.zeros(m.nc); Lo = np.zeros(m.nint + 1); Up = np.zeros(m.nint + 1)
    b = np.zeros((3, m.nc))
    lib().om_momentum_assemble(m.ref(), _p(m.bc_U()), C.c_double(nu), C.c_double(dt),
                               _p(_f64(mf)), _p(_f64(Uold)), _p(_f64(np.reshape(Ub, (3, m.nb)))),
                               _p(None if gradU is None else _f64(gradU)),
                               _p(None if gradS is None else _f64(gradS)), C.c_double(psi), _p(D),
                               _p(Lo), _p(Up), _p(b))
    if time == TIME_CN:
        lib().om_momentum_cn(m.ref(), C.c_double(dt), _p(_f64(Uold)), _p(D), _p(Lo), _p(Up), _p(b))
    return D, Lo[:m.nint], Up[:m.nint], b


def H_op(m: OMesh, Lo, Up, b, U):
    H = np.zeros((3, m.nc))
    lib().om_H(m.ref(), _p(_f64(Lo)), _p(_f64(Up)), _p(_f64(b)), _p(_f64(U)), _p(H))
    return H


def pressure_assemble(m: OMesh, rAU, HbyA, Ub, pb, gradp=None, plag=None, psi=1.0):
    Dp = np.zeros(m.nc); Lp = np.zeros(m.nint + 1); bp = np.zeros(m.nc)
    phiH = np.zeros(m.nf); af = np.zeros(m.nf); no = np.zeros(m.nint + 1)
    lib().om_pressure_assemble(m.ref(), _p(m.bc_U()), _p(m.bc_p()), _p(_f64(rAU)), _p(_f64(HbyA)),
                               _p(_f64(np.reshape(Ub, (3, m.nb)))), _p(_f64(pb)),
                               _p(None if gradp is None else _f64(gradp)),
                               _p(_f64(np.zeros(m.nc) if plag is None else plag)), C.c_double(psi),
                               _p(Dp), _p(Lp), _p(bp),
                               _p(phiH), _p(af), _p(no))
    return dict(Dp=Dp, Lp=Lp[:m.nint], bp=bp, phiHbyA=phiH, af=af, nonorth=no[:m.nint])


def flux_from_U(m: OMesh, U, Ub):
    phi = np.zeros(m.nf)
    lib().om_flux_from_U(m.ref(), _p(_f64(U)), _p(_f64(np.reshape(Ub, (3, m.nb)))), _p(phi))
    return phi


def piso_step(m: OMesh, U, p, phi, Ub, pb, *, nu, dt, ncorr=2, nonorth=True, tolU=1e-10,
              tolp=1e-10, tol_abs=0.0, maxitU=1000, maxitp=20000, pref_cell=0,
              wk_patch=(), Rp=(), Cw=(), Rd=(), pc=(), wk_scheme=WK_EXACT, psi=1.0, conv=CONV_UPWIND,
              time=TIME_BE):
    """One PISO step in place on copies; returns (U, p, phi, pb, pc, info).

    nonorth: True (both), False (none), or a mask: 1 momentum, 2 pressure."""
    U = _f64(np.array(U, np.float64)); p = _f64(np.array(p, np.float64))
    phi = _f64(np.array(phi, np.float64)); pb = _f64(np.array(pb, np.float64))
    Ub = _f64(np.reshape(Ub, (3, m.nb)))
    wk_patch = _i32(np.atleast_1d(np.asarray(wk_patch, np.int32)))
    Rp, Cw, Rd = (_f64(np.atleast_1d(np.asarray(a, np.float64))) for a in (Rp, Cw, Rd))
    pc = _f64(np.array(np.atleast_1d(np.asarray(pc, np.float64))))
    nonorth = 3 if nonorth is True else (0 if nonorth is False else int(nonorth))
    opts = _PisoOpts(nu, dt, ncorr, nonorth, tolU, tolp, tol_abs, maxitU, maxitp, pref_cell,
                     wk_scheme, int(wk_patch.shape[0]), _p(wk_patch), _p(Rp), _p(Cw), _p(Rd), psi, conv, time)
    info = _PisoInfo()
    lib().om_piso_step(m.ref(), C.byref(opts), _p(U), _p(p), _p(phi), _p(Ub), _p(pb), _p(pc),
                       C.byref(info))
    n_out = int(wk_patch.shape[0])
    return U, p, phi, pb, pc, dict(itU=list(info.itU), itp=list(info.itp)[:ncorr],
                                   status=info.status, Q=list(info.Q)[:n_out],
                                   po=list(info.po)[:n_out])


def piso_step_bwd(m: OMesh, U, p, phi, Ub, pb, Ubar, pbar, phibar, pbbar=None, pcbar=(), *, nu,
                  dt, ncorr=2, nonorth=True, tolU=1e-10, tolp=1e-10, tol_abs=0.0, maxitU=1000,
                  maxitp=20000, pref_cell=0, wk_patch=(), Rp=(), Cw=(), Rd=(), pc=(),
                  wk_scheme=WK_EXACT, psi=1.0, conv=CONV_UPWIND, time=TIME_BE):
    """Adjoint of ``piso_step`` at the inputs (U, p, phi, Ub, pb, pc).

    (Ubar, pbar, phibar, pbbar, pcbar) are the adjoints of the step's outputs
    (U, p, phi, pb, pc).  Returns a dict with the adjoints of the inputs
    U, p, phi, pb, pc and of the parameters Ub, nu, Rp, Cw, Rd."""
    U = _f64(np.array(U, np.float64)); p = _f64(np.array(p, np.float64))
    phi = _f64(np.array(phi, np.float64)); pb = _f64(np.array(pb, np.float64))
    Ub = _f64(np.reshape(Ub, (3, m.nb)))
    wk_patch = _i32(np.atleast_1d(np.asarray(wk_patch, np.int32)))
    n_out = int(wk_patch.shape[0])
    Rp, Cw, Rd = (_f64(np.atleast_1d(np.asarray(a, np.float64))) for a in (Rp, Cw, Rd))
    pc = _f64(np.array(np.atleast_1d(np.asarray(pc, np.float64))))
    Ub_ = _f64(np.array(np.reshape(Ubar, (3, m.nc)), np.float64))
    pb_ = _f64(np.array(pbar, np.float64))
    phib_ = _f64(np.array(phibar, np.float64))
    pbb_ = _f64(np.zeros(m.nb) if pbbar is None else np.array(pbbar, np.float64))
    pcb_ = _f64(np.zeros(n_out) if len(np.atleast_1d(pcbar)) == 0
                else np.array(np.atleast_1d(pcbar), np.float64))
    Ubbar = np.zeros((3, m.nb)); nubar = C.c_double(0.0)
    Rpb, Cb, Rdb = np.zeros(max(n_out, 1)), np.zeros(max(n_out, 1)), np.zeros(max(n_out, 1))
    nonorth = 3 if nonorth is True else (0 if nonorth is False else int(nonorth))
    opts = _PisoOpts(nu, dt, ncorr, nonorth, tolU, tolp, tol_abs, maxitU, maxitp, pref_cell,
                     wk_scheme, n_out, _p(wk_patch), _p(Rp), _p(Cw), _p(Rd), psi, conv, time)
    st = lib().om_piso_step_bwd(m.ref(), C.byref(opts), _p(U), _p(p), _p(phi), _p(Ub), _p(pb),
                                _p(pc), _p(Ub_), _p(pb_), _p(phib_), _p(pbb_), _p(pcb_),
                                _p(Ubbar), C.byref(nubar), _p(Rpb), _p(Cb), _p(Rdb))
    return dict(U=Ub_, p=pb_, phi=phib_, pb=pbb_, pc=pcb_[:n_out], Ub=Ubbar, nu=nubar.value,
                Rp=Rpb[:n_out], Cw=Cb[:n_out], Rd=Rdb[:n_out], status=st)


# ------------------------------------------------------- polyhedral geometry
def polymesh_geometry(points, face_ptr, face_pts, owner, neighbour, n_cells):
    """Geometry of a polyhedral mesh from its vertices (the static graph
    arrays of Sec. 2.4.1 for a mesh given as points and face vertex loops, the
    form of an OpenFOAM polyMesh).  Face f has vertices
    face_pts[face_ptr[f]:face_ptr[f+1]] whose right-hand normal points out of
    owner[f].  Plain definitions, exact for planar faces:
      S_f = 1/2 sum_k p_k x p_{k+1}                     (vector area of the loop)
      x_f = centroid of the polygon: a fan from p_0, triangle centroids
            weighted by their signed areas along S_f
      V_i = 1/3 sum_f x_f . S_f^out                     (divergence theorem, div x = 3)
      C_i = 1/(4 V_i) sum_f (x_f . S_f^out) x_f          (div(x_a x) = 4 x_a; x . n is
                                                         constant on a planar face)
    with S_f^out = +S_f for the owner, -S_f for the neighbour.
    Returns Sf [nf, 3], Cf [nf, 3], V [nc], C [nc, 3]."""
    P = np.asarray(points, np.float64)
    fp = np.asarray(face_ptr, np.int64)
    fv = np.asarray(face_pts, np.int64)
    nf = fp.shape[0] - 1
    Sf = np.zeros((nf, 3))
    Cf = np.zeros((nf, 3))
    for f in range(nf):
        v = P[fv[fp[f]:fp[f + 1]]]
        S = 0.5 * np.cross(v, np.roll(v, -1, axis=0)).sum(axis=0)
        n = S / np.linalg.norm(S)
        a_sum, c_sum = 0.0, np.zeros(3)
        for k in range(1, v.shape[0] - 1):
            a = 0.5 * np.dot(np.cross(v[k] - v[0], v[k + 1] - v[0]), n)
            a_sum += a
            c_sum += a * (v[0] + v[k] + v[k + 1]) / 3.0
        Sf[f], Cf[f] = S, c_sum / a_sum
    own = np.asarray(owner, np.int64)
    nei = np.asarray(neighbour, np.int64)
    ni = nei.shape[0]
    xs = np.einsum("ij,ij->i", Cf, Sf)
    vol = np.zeros(n_cells)
    mom = np.zeros((n_cells, 3))
    for f in range(nf):
        vol[own[f]] += xs[f] / 3.0
        mom[own[f]] += xs[f] * Cf[f] / 4.0
        if f < ni:
            vol[nei[f]] -= xs[f] / 3.0
            mom[nei[f]] -= xs[f] * Cf[f] / 4.0
    return Sf, Cf, vol, mom / vol[:, None]
