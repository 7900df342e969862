"""Thin ctypes binding of libdifvm.so (the C ABI of include/difvm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Function names are the C names.  Field arguments are torch CUDA
tensors in the library's internal numbering (see ``Mesh``); streams default to
torch's current stream.  If the shared library is missing or fails to load,
importing this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

# ---------------------------------------------------------------- constants
OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, EBREAKDOWN, ENONFINITE, ETIMEOUT = range(8)
F32, F64 = 0, 1
PATCH_WALL, PATCH_INLET, PATCH_OUTLET, PATCH_EMPTY = 0, 1, 2, 3
BC_VELOCITY, BC_PRESSURE, BC_ALL_FIXED, BC_ALL_ZEROGRAD = 0, 1, 2, 3
DIV_UPWIND, DIV_LINEAR = 0, 1
WK_EXACT, WK_FE, WK_BE = 0, 1, 2
PCG, BICGSTAB = 0, 1
PRECOND_NONE, PRECOND_JACOBI, PRECOND_AMG, PRECOND_AMG_REUSE, PRECOND_DIC = 0, 1, 2, 3, 4
RENUMBER_RCM, SORT_FACES = 1, 2
WIDE_INDICES = 16
# momentum convection of the PISO step: upwind, or second-order upwind by deferred correction
CONV_UPWIND, CONV_SOU = 0, 1
# momentum time scheme of the PISO step: backward Euler or Crank-Nicolson
TIME_BE, TIME_CN = 0, 1
# split of S_f in Eq. nonortho_flux (mesh flags bits 2-3)
NONORTH_OVERRELAXED, NONORTH_MINIMUM, NONORTH_ORTHOGONAL, NONORTH_NONE = 0, 4, 8, 12
NONORTH_MOMENTUM, NONORTH_PRESSURE, NONORTH_ALL = 1, 2, 3

_STATUS = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ENOTCONV: "ENOTCONV",
           EBREAKDOWN: "EBREAKDOWN", ENONFINITE: "ENONFINITE", ETIMEOUT: "ETIMEOUT"}


class DifvmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


# ------------------------------------------------------------------ structs
class MeshDesc(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_internal", C.c_int32), ("n_faces", C.c_int32),
                ("n_patches", C.c_int32), ("owner", C.c_void_p), ("neighbour", C.c_void_p),
                ("Sf", C.c_void_p), ("Cf", C.c_void_p), ("V", C.c_void_p), ("C", C.c_void_p),
                ("patch_start", C.c_void_p), ("patch_size", C.c_void_p), ("patch_type", C.c_void_p),
                ("n_cases", C.c_int32), ("case_cell_start", C.c_void_p), ("flags", C.c_uint32),
                ("device", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("method", C.c_int32), ("precond", C.c_int32), ("max_iter", C.c_int32),
                ("check_every", C.c_int32), ("tol_rel", C.c_double), ("tol_abs", C.c_double),
                ("refine_max", C.c_int32), ("inner_tol", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("refinements", C.c_int32), ("status", C.c_int32),
                ("pad", C.c_int32), ("res0", C.c_double), ("res", C.c_double), ("bnorm", C.c_double)]


class PisoOpts(C.Structure):
    _fields_ = [("nu", C.c_double), ("dt", C.c_double), ("n_corr", C.c_int32),
                ("nonorth", C.c_int32), ("solve_U", SolveOpts), ("solve_p", SolveOpts),
                ("pref_cell", C.c_int32), ("wk_scheme", C.c_int32), ("n_out", C.c_int32),
                ("wk_patch", C.c_int32 * 16), ("nonorth_limit", C.c_double), ("conv", C.c_int32),
                ("time_scheme", C.c_int32)]


class PisoInfo(C.Structure):
    _fields_ = [("itU", C.c_int32 * 3), ("itp", C.c_int32 * 4), ("status", C.c_int32),
                ("pad", C.c_int32), ("Q", C.c_double * 16), ("p_out", C.c_double * 16)]


SOLVE_INFO_NBYTES = C.sizeof(SolveInfo)
PISO_INFO_NBYTES = C.sizeof(PisoInfo)

# ------------------------------------------------------------------ library
_lib = None
_vp, _i, _d = C.c_void_p, C.c_int, C.c_double

_SIGS = {
    "difvm_mesh_create": [_vp, _vp],
    "difvm_mesh_permutation": [_vp, _vp, _vp, _vp],
    "difvm_mesh_info": [_vp, _vp],
    "difvm_mesh_layout": [_vp, _vp],
    "difvm_mesh_autotune": [_vp, _i],
    "difvm_mesh_amg_config": [_vp, _i, _i],
    "difvm_mesh_tuning": [_vp, _vp, _vp, _i, _vp],
    "difvm_grad_gauss": [_vp, _i, _i, _vp, _vp, _i, _vp, _vp],
    "difvm_grad_gauss_bwd": [_vp, _i, _i, _vp, _i, _vp, _vp, _vp],
    "difvm_div_flux": [_vp, _i, _i, _i, _vp, _vp, _vp, _i, _vp, _vp],
    "difvm_div_flux_bwd": [_vp, _i, _i, _i, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp],
    "difvm_laplacian": [_vp, _i, _i, _d, _vp, _vp, _vp, _i, _vp, _vp],
    "difvm_laplacian_bwd": [_vp, _i, _i, _d, _vp, _i, _vp, _vp, _vp, _vp],
    "difvm_laplacian_apply": [_vp, _i, _vp, _vp, _vp, _vp, _i, _i, _vp, _vp],
    "difvm_laplacian_apply_bwd": [_vp, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp],
    "difvm_krylov_workspace_bytes": [_vp, _i, _i, _i],
    "difvm_krylov_solve": [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp, C.c_size_t, _vp, _vp],
    "difvm_krylov_solve_refine": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp, C.c_size_t, _vp, _vp],
    "difvm_krylov_solve_bwd": [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp,
                               C.c_size_t, _vp, _vp],
    "difvm_windkessel_update": [_i, _i, _vp, _vp, _vp, _vp, _d, _vp, _vp, _vp],
    "difvm_windkessel_update_bwd": [_i, _i, _vp, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp, _vp, _vp,
                                    _vp, _vp, _vp],
    "difvm_krylov_refine_workspace_bytes": [_vp, _i, _i],
    "difvm_krylov_opts_workspace_bytes": [_vp, _i, _vp, _i],
    "difvm_piso_create": [_vp, _i, _vp, _vp],
    "difvm_piso_step": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "difvm_piso_step_record": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp],
    "difvm_piso_step_bwd": [_vp, _vp, C.c_size_t, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                            _vp],
    "difvm_piso_adjoint_reset": [_vp, _vp],
    "difvm_piso_step_graph": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "difvm_flux_from_U": [_vp, _i, _vp, _vp, _vp, _vp],
    "difvm_laplacian_apply_bwd_noalloc": [_vp, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp,
                                          _vp],
    "difvm_polymesh_geometry": [_i, _vp, _i, _vp, _vp, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp],
    "difvm_prof_start": [_i, _i],
    "difvm_prof_stop": [_vp, _vp],
}


def lib():
    """Load (building first if stale) the CUDA library; raises if unavailable."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or _build.stale():
            try:
                _build.build()
            except Exception as e:  # nvcc missing or failed: fail loudly
                if not os.path.exists(path):
                    raise ImportError(f"libdifvm.so is missing and could not be built: {e}") from e
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is not None:
                fn.argtypes = args
                fn.restype = C.c_int
        L.difvm_last_error.restype = C.c_char_p
        L.difvm_launch_count.restype = C.c_uint64
        L.difvm_alg_bytes.restype = C.c_uint64
        L.difvm_prof_bytes.restype = C.c_uint64
        L.difvm_mesh_destroy.argtypes = [_vp]
        L.difvm_mesh_destroy.restype = None
        for nm in ("difvm_krylov_workspace_bytes", "difvm_krylov_refine_workspace_bytes",
                   "difvm_krylov_opts_workspace_bytes"):
            if hasattr(L, nm):
                getattr(L, nm).restype = C.c_size_t
        if hasattr(L, "difvm_piso_tape_bytes"):
            L.difvm_piso_tape_bytes.argtypes = [_vp]
            L.difvm_piso_tape_bytes.restype = C.c_size_t
        if hasattr(L, "difvm_piso_destroy"):
            L.difvm_piso_destroy.argtypes = [_vp]
            L.difvm_piso_destroy.restype = None
        _lib = L
    return _lib


def _check(st):
    if st != OK:
        raise DifvmError(st, lib().difvm_last_error().decode())


def difvm_polymesh_geometry(points, face_ptr, face_pts, owner, neighbour, n_cells):
    """Face area vectors and centroids, cell volumes and centroids of a
    polyhedral mesh given by vertices and face vertex loops (host arrays, input
    numbering; see include/difvm.h).  Returns (Sf [nf,3], Cf [nf,3], V [nc], C [nc,3])."""
    P = np.ascontiguousarray(points, np.float64)
    fp = np.ascontiguousarray(face_ptr, np.int32)
    fv = np.ascontiguousarray(face_pts, np.int32)
    own = np.ascontiguousarray(owner, np.int32)
    nei = np.ascontiguousarray(neighbour, np.int32)
    nf, nc = int(fp.shape[0] - 1), int(n_cells)
    Sf, Cf = np.empty((nf, 3)), np.empty((nf, 3))
    V, Cc = np.empty(nc), np.empty((nc, 3))
    _check(lib().difvm_polymesh_geometry(int(P.shape[0]), P.ctypes.data, nf, fp.ctypes.data, fv.ctypes.data,
                                         nc, own.ctypes.data, int(nei.shape[0]), nei.ctypes.data,
                                         Sf.ctypes.data, Cf.ctypes.data, V.ctypes.data, Cc.ctypes.data))
    return Sf, Cf, V, Cc


def launch_count() -> int:
    return int(lib().difvm_launch_count())


PROF_PCG_SPMV, PROF_PCG_UPDATE, PROF_PCG_PUPDATE, PROF_AMG_RESID, PROF_AMG_POST1C = 1, 2, 3, 4, 5


PHASES = ("windkessel", "momentum_assembly", "momentum_solve", "pressure_assembly", "pressure_solve",
          "correction")


def difvm_phase_prof_start(max_marks=100000):
    _check(lib().difvm_phase_prof_start(int(max_marks)))


def difvm_phase_prof_stop():
    """Returns ({phase: summed ms}, steps) of the host-loop PISO steps since start."""
    ms, n = (C.c_double * len(PHASES))(), C.c_int64()
    _check(lib().difvm_phase_prof_stop(ms, C.byref(n)))
    return {ph: float(ms[k]) for k, ph in enumerate(PHASES)}, int(n.value)


def alg_bytes() -> int:
    """Algorithmic bytes of the Krylov and multigrid kernels launched so far."""
    return int(lib().difvm_alg_bytes())


def prof_bytes() -> int:
    """Algorithmic bytes of the launches timed since difvm_prof_start."""
    return int(lib().difvm_prof_bytes())


def difvm_prof_start(tag, max_launches=100000):
    _check(lib().difvm_prof_start(tag, max_launches))


def difvm_prof_stop():
    """Returns (summed kernel milliseconds, number of timed launches)."""
    ms, n = C.c_double(), C.c_int64()
    _check(lib().difvm_prof_stop(C.byref(ms), C.byref(n)))
    return ms.value, n.value


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_cuda and t.is_contiguous(), "fields must be contiguous CUDA tensors"
        return t.data_ptr()
    return int(t)


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _prec(t):
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


# --------------------------------------------------------------------- mesh
class Mesh:
    """A mesh uploaded to the GPU (difvm_mesh_create), with its numbering maps.

    ``m`` is any object with the attributes of ``meshgen.Mesh`` (input
    numbering).  ``to_cells``/``from_cells`` and friends move numpy or torch
    data between the input numbering and the internal (RCM + sorted) one.
    """

    def __init__(self, m, device=0, flags=RENUMBER_RCM | SORT_FACES, case_cell_start=None,
                 nonorth=NONORTH_OVERRELAXED):
        self.src = m
        flags = (flags & ~NONORTH_NONE) | nonorth
        self.device = device
        keep = [np.ascontiguousarray(a, dt) for a, dt in (
            (m.owner, np.int32), (m.neighbour, np.int32), (m.Sf, np.float64), (m.Cf, np.float64),
            (m.V, np.float64), (m.C, np.float64), (m.patch_start, np.int32),
            (m.patch_size, np.int32), (m.patch_type, np.int32))]
        cs = None if case_cell_start is None else np.ascontiguousarray(case_cell_start, np.int32)
        p = lambda a: None if a is None else a.ctypes.data
        d = MeshDesc(m.n_cells, m.n_internal, int(keep[0].shape[0]), int(keep[6].shape[0]),
                     *[p(a) for a in keep], 0 if cs is None else int(cs.shape[0] - 1), p(cs),
                     flags, device)
        h = C.c_void_p()
        with torch.cuda.device(device):
            _check(lib().difvm_mesh_create(C.byref(d), C.byref(h)))
        self.h = h
        info = (C.c_int64 * 6)()
        _check(lib().difvm_mesh_info(h, info))
        self.nc, self.ni, self.nf, self.nb, self.npatch, self.nnz = (int(v) for v in info)
        cno = np.empty(self.nc, np.int32)
        fon = np.empty(self.nf, np.int32)
        flip = np.empty(self.nf, np.int8)
        _check(lib().difvm_mesh_permutation(h, cno.ctypes.data, fon.ctypes.data, flip.ctypes.data))
        self.cell_new_of_old, self.face_old_of_new, self.face_flip = cno, fon, flip
        self.cell_old_of_new = np.empty_like(cno)
        self.cell_old_of_new[cno] = np.arange(self.nc, dtype=np.int32)
        self.face_sign = np.where(flip != 0, -1.0, 1.0)
        self.bnd_old_of_new = fon[self.ni:] - self.ni
        self.patch_start = np.asarray(m.patch_start, np.int64)
        self.patch_size = np.asarray(m.patch_size, np.int64)
        self.patch_type = np.asarray(m.patch_type, np.int64)
        # a case table makes the solvers segmented: one set of Krylov scalars per case
        self.batched = cs is not None
        self.n_cases = 1 if cs is None else int(cs.shape[0] - 1)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.difvm_mesh_destroy(h)
            self.h = None

    @property
    def handle(self):
        return self.h

    # numbering maps (numpy or torch, leading component axes allowed)
    def to_cells(self, x):
        return x[..., self.cell_old_of_new] if isinstance(x, np.ndarray) else \
            x[..., torch.as_tensor(self.cell_old_of_new, device=x.device, dtype=torch.long)]

    def from_cells(self, x):
        return x[..., self.cell_new_of_old] if isinstance(x, np.ndarray) else \
            x[..., torch.as_tensor(self.cell_new_of_old, device=x.device, dtype=torch.long)]

    def to_faces(self, f, flux=True):
        """Input-numbered face field -> internal; fluxes change sign on flipped faces."""
        y = f[..., self.face_old_of_new]
        if flux:
            y = y * (self.face_sign if isinstance(y, np.ndarray) else
                     torch.as_tensor(self.face_sign, device=y.device, dtype=y.dtype))
        return y

    def from_faces(self, f, flux=True):
        if flux:
            f = f * (self.face_sign if isinstance(f, np.ndarray) else
                     torch.as_tensor(self.face_sign, device=f.device, dtype=f.dtype))
        out = np.empty_like(f) if isinstance(f, np.ndarray) else torch.empty_like(f)
        out[..., self.face_old_of_new] = f
        return out

    def to_bnd(self, b):
        return b[..., self.bnd_old_of_new] if isinstance(b, np.ndarray) else \
            b[..., torch.as_tensor(self.bnd_old_of_new, device=b.device, dtype=torch.long)]

    def from_bnd(self, b):
        out = np.empty_like(b) if isinstance(b, np.ndarray) else torch.empty_like(b)
        out[..., self.bnd_old_of_new] = b
        return out


def difvm_mesh_autotune(mesh, mode):
    """0: face operators launch their default variant; 1: first-use timing on
    (the default); 2: forget the kept choices."""
    _check(lib().difvm_mesh_autotune(_mh(mesh), int(mode)))


def difvm_mesh_tuning(mesh):
    """The kept face-operator variants: {(operator, option, components): variant}."""
    cap = 64
    keys, var, n = (C.c_uint32 * cap)(), (C.c_int32 * cap)(), C.c_int32()
    _check(lib().difvm_mesh_tuning(_mh(mesh), keys, var, cap, C.byref(n)))
    return {(int(keys[k]) >> 8, (int(keys[k]) >> 4) & 15, int(keys[k]) & 15): int(var[k])
            for k in range(min(n.value, cap))}


def difvm_mesh_layout(mesh):
    """Index layouts in use: (compact 4-byte slot words, 16-bit ELL columns)."""
    out = (C.c_int32 * 2)()
    _check(lib().difvm_mesh_layout(_mh(mesh), out))
    return bool(out[0]), bool(out[1])


def difvm_mesh_amg_config(mesh, tail_rows=-1, tail_bps=-1):
    """Levels below tail_rows rows run as one fused cooperative kernel of
    tail_bps blocks per SM (0 rows: none; -1: the library's choice)."""
    _check(lib().difvm_mesh_amg_config(_mh(mesh), int(tail_rows), int(tail_bps)))


def _mh(mesh):
    return mesh.h if isinstance(mesh, Mesh) else mesh


# ---------------------------------------------------------------- operators
def difvm_grad_gauss(mesh, bc_class, phi, phi_b=None, grad=None, stream=None):
    """grad[ncomp,3,nc] = Gauss gradient of phi[ncomp,nc] (Eq. gauss_green)."""
    nq = phi.shape[0] if phi.dim() == 2 else 1
    if grad is None:
        grad = torch.empty((nq, 3, phi.shape[-1]), dtype=phi.dtype, device=phi.device)
    _check(lib().difvm_grad_gauss(_mh(mesh), _prec(phi), bc_class, _ptr(phi), _ptr(phi_b), nq,
                                  _ptr(grad), _stream(stream)))
    return grad


def difvm_grad_gauss_bwd(mesh, bc_class, grad_bar, phi_bar, phi_b_bar=None, stream=None):
    nq = grad_bar.shape[0]
    _check(lib().difvm_grad_gauss_bwd(_mh(mesh), _prec(grad_bar), bc_class, _ptr(grad_bar), nq,
                                      _ptr(phi_bar), _ptr(phi_b_bar), _stream(stream)))


def difvm_div_flux(mesh, scheme, bc_class, mflux, phi, phi_b=None, out=None, stream=None):
    nq = phi.shape[0] if phi.dim() == 2 else 1
    if out is None:
        out = torch.empty_like(phi)
    _check(lib().difvm_div_flux(_mh(mesh), _prec(phi), scheme, bc_class, _ptr(mflux), _ptr(phi),
                                _ptr(phi_b), nq, _ptr(out), _stream(stream)))
    return out


def difvm_div_flux_bwd(mesh, scheme, bc_class, mflux, phi, phi_b, out_bar, mflux_bar=None,
                       phi_bar=None, phi_b_bar=None, stream=None):
    nq = phi.shape[0] if phi.dim() == 2 else 1
    _check(lib().difvm_div_flux_bwd(_mh(mesh), _prec(phi), scheme, bc_class, _ptr(mflux), _ptr(phi),
                                    _ptr(phi_b), nq, _ptr(out_bar), _ptr(mflux_bar), _ptr(phi_bar),
                                    _ptr(phi_b_bar), _stream(stream)))


def difvm_laplacian(mesh, bc_class, gamma, phi, phi_b=None, grad=None, out=None, stream=None):
    nq = phi.shape[0] if phi.dim() == 2 else 1
    if out is None:
        out = torch.empty_like(phi)
    _check(lib().difvm_laplacian(_mh(mesh), _prec(phi), bc_class, float(gamma), _ptr(phi),
                                 _ptr(phi_b), _ptr(grad), nq, _ptr(out), _stream(stream)))
    return out


def difvm_laplacian_bwd(mesh, bc_class, gamma, out_bar, phi_bar=None, phi_b_bar=None,
                        grad_bar=None, stream=None):
    nq = out_bar.shape[0] if out_bar.dim() == 2 else 1
    _check(lib().difvm_laplacian_bwd(_mh(mesh), _prec(out_bar), bc_class, float(gamma),
                                     _ptr(out_bar), nq, _ptr(phi_bar), _ptr(phi_b_bar),
                                     _ptr(grad_bar), _stream(stream)))


def difvm_laplacian_apply(mesh, diag, lower, upper, x, transpose=False, y=None, stream=None):
    nq = x.shape[0] if x.dim() == 2 else 1
    if y is None:
        y = torch.empty_like(x)
    _check(lib().difvm_laplacian_apply(_mh(mesh), _prec(x), _ptr(diag), _ptr(lower), _ptr(upper),
                                       _ptr(x), nq, int(bool(transpose)), _ptr(y), _stream(stream)))
    return y


def difvm_laplacian_apply_bwd(mesh, diag, lower, upper, x, y_bar, x_bar=None, diag_bar=None,
                              lower_bar=None, upper_bar=None, stream=None):
    nq = x.shape[0] if x.dim() == 2 else 1
    tmp = torch.empty_like(x) if x_bar is not None else None
    _check(lib().difvm_laplacian_apply_bwd(_mh(mesh), _prec(x), _ptr(diag), _ptr(lower),
                                           _ptr(upper), _ptr(x), _ptr(y_bar), nq, _ptr(x_bar),
                                           _ptr(diag_bar), _ptr(lower_bar), _ptr(upper_bar),
                                           _ptr(tmp), _stream(stream)))


def difvm_laplacian_apply_bwd_noalloc(mesh, diag, lower, upper, x, y_bar, x_bar=None, diag_bar=None,
                                      lower_bar=None, upper_bar=None, stream=None):
    """Adjoint of the LDU apply with the library's built-in scratch (no allocation)."""
    nq = x.shape[0] if x.dim() == 2 else 1
    _check(lib().difvm_laplacian_apply_bwd_noalloc(_mh(mesh), _prec(x), _ptr(diag), _ptr(lower),
                                                   _ptr(upper), _ptr(x), _ptr(y_bar), nq,
                                                   _ptr(x_bar), _ptr(diag_bar), _ptr(lower_bar),
                                                   _ptr(upper_bar), _stream(stream)))


# ------------------------------------------------------------------- Krylov
def solve_opts(method=PCG, tol_rel=1e-10, tol_abs=0.0, max_iter=1000, precond=PRECOND_JACOBI,
               check_every=8, refine_max=0, inner_tol=0.0):
    return SolveOpts(method, precond, max_iter, check_every, tol_rel, tol_abs, refine_max, inner_tol)


def decode_solve_info(buf, n):
    raw = buf.cpu().numpy().tobytes()
    out = []
    for c in range(n):
        s = SolveInfo.from_buffer_copy(raw[c * SOLVE_INFO_NBYTES:(c + 1) * SOLVE_INFO_NBYTES])
        out.append(dict(iters=s.iters, refinements=s.refinements, status=s.status, res0=s.res0,
                        res=s.res, bnorm=s.bnorm))
    return out


def _info_buf(n, device):
    return torch.zeros(n * SOLVE_INFO_NBYTES, dtype=torch.uint8, device=device)


def difvm_krylov_workspace_bytes(mesh, prec, method, ncomp):
    return int(lib().difvm_krylov_workspace_bytes(_mh(mesh), prec, method, ncomp))


def difvm_krylov_solve(mesh, diag, lower, upper, b, x, opts=None, workspace=None, stream=None,
                       raise_on_fail=False, **kw):
    """Solve A x = b in place (x is the initial guess).  Returns (status, [info per comp]);
    on a batched mesh the infos are per case and component, case-major."""
    opts = opts or solve_opts(**kw)
    nq = b.shape[0] if b.dim() == 2 else 1
    prec = _prec(b)
    nbytes = int(lib().difvm_krylov_opts_workspace_bytes(_mh(mesh), prec, C.byref(opts), nq))
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=b.device)
    nk = getattr(mesh, "n_cases", 1) if getattr(mesh, "batched", False) else 1
    info = _info_buf(nk * nq, b.device)
    st = lib().difvm_krylov_solve(_mh(mesh), prec, C.byref(opts), _ptr(diag), _ptr(lower), _ptr(upper),
                                  _ptr(b), _ptr(x), nq, _ptr(workspace), workspace.numel(), _ptr(info),
                                  _stream(stream))
    if st in (EINVAL, ECUDA, ENOMEM) or (raise_on_fail and st != OK):
        _check(st)
    return st, decode_solve_info(info, nk * nq)


def difvm_krylov_solve_refine(mesh, diag32, lower32, upper32, b64, x64, opts=None, workspace=None,
                              stream=None, **kw):
    opts = opts or solve_opts(**kw)
    nq = b64.shape[0] if b64.dim() == 2 else 1
    nbytes = max(int(lib().difvm_krylov_opts_workspace_bytes(_mh(mesh), F32, C.byref(opts), nq)),
                 int(lib().difvm_krylov_refine_workspace_bytes(_mh(mesh), opts.method, nq)))
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=b64.device)
    info = _info_buf(nq, b64.device)
    st = lib().difvm_krylov_solve_refine(_mh(mesh), C.byref(opts), _ptr(diag32), _ptr(lower32),
                                         _ptr(upper32), _ptr(b64), _ptr(x64), nq, _ptr(workspace),
                                         workspace.numel(), _ptr(info), _stream(stream))
    if st in (EINVAL, ECUDA, ENOMEM):
        _check(st)
    return st, decode_solve_info(info, nq)


def difvm_krylov_solve_bwd(mesh, diag, lower, upper, x, x_bar, b_bar, diag_bar=None, lower_bar=None,
                           upper_bar=None, opts=None, workspace=None, stream=None, **kw):
    opts = opts or solve_opts(**kw)
    nq = x.shape[0] if x.dim() == 2 else 1
    prec = _prec(x)
    nbytes = int(lib().difvm_krylov_opts_workspace_bytes(_mh(mesh), prec, C.byref(opts), nq))
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    info = _info_buf(nq, x.device)
    st = lib().difvm_krylov_solve_bwd(_mh(mesh), prec, C.byref(opts), _ptr(diag), _ptr(lower),
                                      _ptr(upper), _ptr(x), _ptr(x_bar), nq, _ptr(b_bar),
                                      _ptr(diag_bar), _ptr(lower_bar), _ptr(upper_bar),
                                      _ptr(workspace), workspace.numel(), _ptr(info), _stream(stream))
    if st in (EINVAL, ECUDA, ENOMEM):
        _check(st)
    return st, decode_solve_info(info, nq)


# --------------------------------------------------------------- Windkessel
def difvm_windkessel_update(scheme, Rp, Cw, Rd, Q, dt, pc, p_out=None, stream=None):
    """One RCR step on device double tensors [n_out]; pc is updated in place."""
    n = pc.numel()
    _check(lib().difvm_windkessel_update(n, scheme, _ptr(Rp), _ptr(Cw), _ptr(Rd), _ptr(Q), float(dt),
                                         _ptr(pc), _ptr(p_out), _stream(stream)))
    return pc, p_out


def difvm_windkessel_update_bwd(scheme, Rp, Cw, Rd, Q, dt, pc_in, pc_out_bar, p_out_bar, pc_in_bar,
                                Q_bar=None, Rp_bar=None, C_bar=None, Rd_bar=None, stream=None):
    n = pc_in.numel()
    _check(lib().difvm_windkessel_update_bwd(n, scheme, _ptr(Rp), _ptr(Cw), _ptr(Rd), _ptr(Q),
                                             float(dt), _ptr(pc_in), _ptr(pc_out_bar),
                                             _ptr(p_out_bar), _ptr(pc_in_bar), _ptr(Q_bar),
                                             _ptr(Rp_bar), _ptr(C_bar), _ptr(Rd_bar), _stream(stream)))


# --------------------------------------------------------------------- PISO
def difvm_flux_from_U(mesh, U, U_b, phi=None, stream=None):
    if phi is None:
        phi = torch.empty(mesh.nf, dtype=U.dtype, device=U.device)
    _check(lib().difvm_flux_from_U(_mh(mesh), _prec(U), _ptr(U), _ptr(U_b), _ptr(phi), _stream(stream)))
    return phi


def piso_opts(nu, dt, n_corr=2, nonorth=True, solve_U=None, solve_p=None, pref_cell=0,
              wk_scheme=WK_EXACT, wk_patch=(), nonorth_limit=1.0, conv=None, time_scheme=None):
    o = PisoOpts()
    # nonorth: True = momentum and pressure corrections, False = none, or a bitmask
    mask = NONORTH_ALL if nonorth is True else (0 if nonorth is False else int(nonorth))
    o.nu, o.dt, o.n_corr, o.nonorth = float(nu), float(dt), int(n_corr), mask
    o.solve_U = solve_U or solve_opts(BICGSTAB, 1e-10, max_iter=1000)
    o.solve_p = solve_p or solve_opts(PCG, 1e-10, max_iter=20000)
    o.pref_cell, o.wk_scheme, o.n_out = int(pref_cell), int(wk_scheme), len(wk_patch)
    for k, p in enumerate(wk_patch):
        o.wk_patch[k] = int(p)
    o.nonorth_limit = float(nonorth_limit)
    o.conv = CONV_UPWIND if conv is None else int(conv)
    o.time_scheme = TIME_BE if time_scheme is None else int(time_scheme)
    return o


def decode_piso_info(buf):
    s = PisoInfo.from_buffer_copy(buf.cpu().numpy().tobytes())
    return dict(itU=list(s.itU), itp=list(s.itp), status=s.status, Q=list(s.Q), p_out=list(s.p_out))


class StepLog:
    """Per-step metrics of a PISO run as JSON lines, one object per step:
    the step index (and time, wall milliseconds when given), the BiCGStab
    iterations of each momentum component and the CG iterations of each
    pressure corrector, the step status, the outlet flux Q and pressure p_out
    of each Windkessel outlet and, when the face flux phi is passed, the
    continuity error of phi: sum over cells of |sum_f sigma_f phi_f|, computed
    on the device (difvm_div_flux of a unit field with zero-gradient boundary
    values), absolute and relative to sum_f |phi_f|.  `out` is a path (opened
    for appending) or a writable text file."""

    def __init__(self, out, mesh=None, n_out=0, n_corr=2):
        import json as _json
        self._json = _json
        self._own = isinstance(out, (str, os.PathLike))
        self.f = open(out, "a") if self._own else out
        self.mesh, self.n_out, self.n_corr = mesh, int(n_out), int(n_corr)
        self._ones = {}

    def continuity(self, phi):
        """(sum_cells |div phi|, the same relative to sum_f |phi_f|) of a face flux."""
        key = (phi.dtype, phi.device)
        if key not in self._ones:
            self._ones[key] = torch.ones(1, self.mesh.nc, dtype=phi.dtype, device=phi.device)
        d = difvm_div_flux(self.mesh, DIV_UPWIND, BC_ALL_ZEROGRAD, phi, self._ones[key])
        tot = torch.stack([d.abs().sum().double(), phi.abs().sum().double()]).cpu()
        a, b = float(tot[0]), float(tot[1])
        return a, (a / b if b > 0 else 0.0)

    def log(self, step, info, phi=None, t=None, ms=None):
        """Write the line of one step (info: the step's PISO info buffer) and return it."""
        d = decode_piso_info(info)
        rec = {"step": int(step), "status": int(d["status"]), "itU": d["itU"], "itp": d["itp"][:self.n_corr]}
        if t is not None:
            rec["t"] = float(t)
        if ms is not None:
            rec["ms"] = float(ms)
        if self.n_out:
            rec["Q"] = d["Q"][:self.n_out]
            rec["p_out"] = d["p_out"][:self.n_out]
        if phi is not None and self.mesh is not None:
            rec["continuity_abs"], rec["continuity_rel"] = self.continuity(phi)
        self.f.write(self._json.dumps(rec) + "\n")
        self.f.flush()
        return rec

    def close(self):
        if self._own and self.f:
            self.f.close()
        self.f = None


class Piso:
    """difvm_piso_create / difvm_piso_step on one mesh and precision."""

    def __init__(self, mesh, prec, opts):
        self.mesh, self.prec, self.opts = mesh, prec, opts
        h = C.c_void_p()
        _check(lib().difvm_piso_create(_mh(mesh), prec, C.byref(opts), C.byref(h)))
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.difvm_piso_destroy(h)
            self.h = None

    def step(self, U, p, phi, U_b, p_b, wk=None, info=None, stream=None):
        """One PISO step in place.  Returns (status, info buffer on device)."""
        if info is None:
            info = torch.zeros(PISO_INFO_NBYTES, dtype=torch.uint8, device=U.device)
        st = lib().difvm_piso_step(self.h, _ptr(U), _ptr(p), _ptr(phi), _ptr(U_b), _ptr(p_b), _ptr(wk),
                                   _ptr(info), _stream(stream))
        if st in (EINVAL, ECUDA, ENOMEM):
            _check(st)
        return st, info


    def step_graph(self, U, p, phi, U_b, p_b, wk=None, info=None, stream=None):
        """The step as one CUDA-graph launch (captured on the first call for these
        tensors).  Returns the info buffer; the status is in it (decode_piso_info)."""
        if info is None:
            info = torch.zeros(PISO_INFO_NBYTES, dtype=torch.uint8, device=U.device)
        _check(lib().difvm_piso_step_graph(self.h, _ptr(U), _ptr(p), _ptr(phi), _ptr(U_b), _ptr(p_b),
                                           _ptr(wk), _ptr(info), _stream(stream)))
        return info

    def tape_bytes(self):
        return int(lib().difvm_piso_tape_bytes(self.h))

    def new_tape(self, device):
        """A device tape for one recorded step (torch allocations are 512-byte aligned)."""
        return torch.empty(self.tape_bytes(), dtype=torch.uint8, device=device)

    def step_record(self, U, p, phi, U_b, p_b, tape, wk=None, info=None, stream=None):
        """difvm_piso_step that also writes the step's tape.  Returns (status, info)."""
        if info is None:
            info = torch.zeros(PISO_INFO_NBYTES, dtype=torch.uint8, device=U.device)
        st = lib().difvm_piso_step_record(self.h, _ptr(U), _ptr(p), _ptr(phi), _ptr(U_b), _ptr(p_b),
                                          _ptr(wk), _ptr(info), _ptr(tape), tape.numel(),
                                          _stream(stream))
        if st in (EINVAL, ECUDA, ENOMEM):
            _check(st)
        return st, info

    def step_bwd(self, tape, U_b, wk, U_bar, p_bar, phi_bar, p_b_bar=None, wk_bar=None,
                 U_b_bar=None, nu_bar=None, info=None, stream=None):
        """Adjoint of a recorded step, in place on the adjoint arrays (see the C header).
        Returns (status, info)."""
        if info is None:
            info = torch.zeros(PISO_INFO_NBYTES, dtype=torch.uint8, device=U_bar.device)
        st = lib().difvm_piso_step_bwd(self.h, _ptr(tape), tape.numel(), _ptr(U_b), _ptr(wk),
                                       _ptr(U_bar), _ptr(p_bar), _ptr(phi_bar), _ptr(p_b_bar),
                                       _ptr(wk_bar), _ptr(U_b_bar), _ptr(nu_bar), _ptr(info),
                                       _stream(stream))
        if st in (EINVAL, ECUDA, ENOMEM):
            _check(st)
        return st, info


    def adjoint_reset(self, stream=None):
        """Zero the starting guesses of the adjoint solves."""
        _check(lib().difvm_piso_adjoint_reset(self.h, _stream(stream)))


def difvm_piso_adjoint_reset(piso, stream=None):
    piso.adjoint_reset(stream)


def difvm_piso_step(piso, U, p, phi, U_b, p_b, wk=None, info=None, stream=None):
    return piso.step(U, p, phi, U_b, p_b, wk, info, stream)


def difvm_piso_step_graph(piso, U, p, phi, U_b, p_b, wk=None, info=None, stream=None):
    return piso.step_graph(U, p, phi, U_b, p_b, wk, info, stream)


def difvm_piso_tape_bytes(piso):
    return piso.tape_bytes()


def difvm_piso_step_record(piso, U, p, phi, U_b, p_b, tape, wk=None, info=None, stream=None):
    return piso.step_record(U, p, phi, U_b, p_b, tape, wk, info, stream)


def difvm_piso_step_bwd(piso, tape, U_b, wk, U_bar, p_bar, phi_bar, p_b_bar=None, wk_bar=None,
                        U_b_bar=None, nu_bar=None, info=None, stream=None):
    return piso.step_bwd(tape, U_b, wk, U_bar, p_bar, phi_bar, p_b_bar, wk_bar, U_b_bar, nu_bar,
                         info, stream)


# ------------------------------------------------- forward + adjoint trajectory
def binomial_cost(n, s):
    """Fewest plain forward steps that reverse n steps from a stored initial
    state with s further state slots (one tape): r n - beta(s + 2, r - 1), r the
    least integer with beta(s + 1, r) >= n, beta(c, r) = C(c + r, c) (Griewank's
    binomial bound; the initial state is one of the s + 1 checkpoints)."""
    from math import comb
    if n <= 1:
        return 0
    c, r = s + 1, 0
    while comb(c + r, c) < n:
        r += 1
    return r * n - (comb(c + 1 + r - 1, c + 1) if r >= 1 else 0)


def binomial_schedule(n, s):
    """Optimal (binomial) checkpoint schedule reversing steps 0..n-1 with the
    initial state in slot 0 and s further slots (Sec. 2.5, Eq. checkpointing).
    Actions on one working state: ("load", slot), ("advance", m) plain steps,
    ("save", slot), ("record", t) the taped step t (the working state is at t),
    ("bwd", t) its adjoint, ("free", slot).  A segment of length L with c free
    slots is split after the k that minimises k + cost(L - k, c - 1) + cost(k, c):
    advance k, save, reverse the right part, free, reverse the left part."""
    acts = []

    def rev(i, j, c, slot):
        if j - i == 1:
            acts.extend([("load", slot), ("record", i), ("bwd", i)])
            return
        if c == 0:
            for t in range(j - 1, i - 1, -1):
                acts.append(("load", slot))
                if t > i:
                    acts.append(("advance", t - i))
                acts.extend([("record", t), ("bwd", t)])
            return
        L = j - i
        k = min(range(1, L), key=lambda q: (q + binomial_cost(L - q, c - 1) + binomial_cost(q, c), q))
        new = s - c + 1
        acts.extend([("load", slot), ("advance", k), ("save", new)])
        rev(i + k, j, c - 1, new)
        acts.append(("free", new))
        rev(i, i + k, c, slot)

    if n > 0:
        rev(0, n, s, 0)
    return acts


def simulate_adjoint(piso, state, nsteps, loss_grad, wk=None, checkpoint_every=None, stream=None,
                     tapes=None, checkpoints=None):
    """n PISO steps forward, then the adjoint of a loss of the final state back
    to the initial state and the parameters (Sec. 2.5, Eq. vjp).

    state = [U, p, phi, U_b, p_b] (device tensors of the handle's precision;
    U, p, phi, p_b end at the final state), wk the Windkessel array or None.
    loss_grad(U, p, phi, p_b, wk) returns the seeds (U_bar, p_bar, phi_bar,
    p_b_bar or None, pc_bar or None) of the loss at the final state.

    checkpoint_every = k: the forward pass keeps the state every k steps and
    the reverse pass re-runs each k-step segment with tapes (memory: k tapes
    plus n/k states; cost: one extra forward step per step).  None: every step
    is recorded in the forward pass (n tapes, no recomputation).

    tapes: optional preallocated list of at least k tapes (piso.new_tape).

    checkpoints = s (instead of checkpoint_every): the optimal binomial schedule
    (binomial_schedule) with s stored states besides the initial one and a
    single tape: memory s + 1 states and one tape; plain forward steps
    binomial_cost(n, s) + 1 (the last one gives the final state for the loss).

    Returns dict(U, p, phi, p_b, pc: adjoints of the initial state; U_b, nu,
    Rp, C, Rd: parameter adjoints; status: worst step status; info: the
    adjoint solver record of the first step)."""
    if checkpoints is not None:
        return _simulate_adjoint_binomial(piso, state, nsteps, loss_grad, wk, int(checkpoints), stream,
                                          tapes)
    U, p, phi, Ub, pb = state
    k = nsteps if not checkpoint_every else max(1, min(int(checkpoint_every), nsteps))
    if tapes is None or len(tapes) < k:
        tapes = [piso.new_tape(U.device) for _ in range(k)]
    worst = OK
    n_out = piso.opts.n_out
    snaps = []

    def snap():
        return [t.clone() for t in (U, p, phi, pb)] + [wk.clone() if wk is not None else None]

    if k == nsteps:
        for j in range(nsteps):
            worst = max(worst, piso.step_record(U, p, phi, Ub, pb, tapes[j], wk=wk, stream=stream)[0])
    else:
        for j in range(nsteps):
            if j % k == 0:
                snaps.append(snap())
            worst = max(worst, piso.step(U, p, phi, Ub, pb, wk=wk, stream=stream)[0])
    Ubar, pbar, phibar, pbbar, pcbar = loss_grad(U, p, phi, pb, wk)
    Ubar, pbar, phibar = Ubar.clone(), pbar.clone(), phibar.clone()
    pbbar = torch.zeros_like(pb) if pbbar is None else pbbar.clone()
    wkbar = None
    if n_out:
        wkbar = torch.zeros(4 * n_out, dtype=torch.float64, device=U.device)
        if pcbar is not None:
            wkbar[3::4] = pcbar
    Ubbar = torch.zeros_like(Ub)
    nubar = torch.zeros(1, dtype=torch.float64, device=U.device)
    info = torch.zeros(PISO_INFO_NBYTES, dtype=torch.uint8, device=U.device)
    piso.adjoint_reset(stream)
    nseg = (nsteps + k - 1) // k
    for seg in reversed(range(nseg)):
        n0, n1 = seg * k, min(nsteps, seg * k + k)
        if k != nsteps:      # re-run the segment from its checkpoint, recording tapes
            sU, sp, sphi, spb, swk = snaps[seg]
            for j in range(n1 - n0):
                worst = max(worst, piso.step_record(sU, sp, sphi, Ub, spb, tapes[j], wk=swk,
                                                    stream=stream)[0])
        for j in reversed(range(n1 - n0)):
            st, _ = piso.step_bwd(tapes[j], Ub, wk, Ubar, pbar, phibar, pbbar, wkbar, Ubbar, nubar,
                                  info=info, stream=stream)
            worst = max(worst, st)
    out = dict(U=Ubar, p=pbar, phi=phibar, p_b=pbbar, U_b=Ubbar, nu=nubar, status=worst,
               info=info)   # info: device record of the first step's adjoint (decode_piso_info)
    if n_out:
        w = wkbar.view(n_out, 4)
        out.update(Rp=w[:, 0], C=w[:, 1], Rd=w[:, 2], pc=w[:, 3])
    return out


def trajectory_adjoint(piso, state, nsteps, boundary, step_loss_grad, wk=None, checkpoint_every=None,
                       stream=None, tapes=None):
    """n PISO steps with boundary values that change from step to step, then
    the adjoint of a loss summed over the steps' outputs,
    L = sum_j l_j(state after step j), back to the initial state and the
    parameters (Sec. 2.5, Eq. vjp, applied step by step in reverse).

    state = [U, p, phi, U_b, p_b] as for simulate_adjoint (U, p, phi, p_b end at
    the final state); boundary(j, U_b) writes the boundary values of step j into
    U_b in place (it is called again for the same j when a segment is re-run);
    step_loss_grad(j, U, p, phi, p_b, wk) returns the seeds (U_bar, p_bar,
    phi_bar, p_b_bar, pc_bar) of l_j at the output of step j, any of them None
    (no seed).  checkpoint_every = k keeps the state every k steps and re-runs
    each segment with tapes (k tapes); None tapes every step.

    Returns dict(U, p, phi, p_b, U_b, nu, status, and Rp, C, Rd, pc per outlet
    when the handle has Windkessel outlets); U_b is the adjoint summed over the
    steps' boundary values."""
    U, p, phi, Ub, pb = state
    k = nsteps if not checkpoint_every else max(1, min(int(checkpoint_every), nsteps))
    if tapes is None or len(tapes) < k:
        tapes = [piso.new_tape(U.device) for _ in range(k)]
    n_out = piso.opts.n_out
    worst = OK

    def snap(src):
        return [t.clone() for t in src[:4]] + [src[4].clone() if src[4] is not None else None]

    cur = [U, p, phi, pb, wk]
    snaps, outs = [], {}
    for j in range(nsteps):
        boundary(j, Ub)
        if k == nsteps:
            worst = max(worst, piso.step_record(U, p, phi, Ub, pb, tapes[j], wk=wk, stream=stream)[0])
            outs[j] = snap(cur)
        else:
            if j % k == 0:
                snaps.append(snap(cur))
            worst = max(worst, piso.step(U, p, phi, Ub, pb, wk=wk, stream=stream)[0])
    Ubar, pbar, phibar = torch.zeros_like(U), torch.zeros_like(p), torch.zeros_like(phi)
    pbbar, Ubbar = torch.zeros_like(pb), torch.zeros_like(Ub)
    nubar = torch.zeros(1, dtype=torch.float64, device=U.device)
    wkbar = torch.zeros(4 * n_out, dtype=torch.float64, device=U.device) if n_out else None
    info = torch.zeros(PISO_INFO_NBYTES, dtype=torch.uint8, device=U.device)

    def seed(j, st):
        g = step_loss_grad(j, *st)
        if g is None:
            return
        for bar, v in zip((Ubar, pbar, phibar, pbbar), g[:4]):
            if v is not None:
                bar += v
        if len(g) > 4 and g[4] is not None and n_out:
            wkbar[3::4] += g[4]

    seed(nsteps - 1, [U, p, phi, pb, wk])
    piso.adjoint_reset(stream)
    nseg = (nsteps + k - 1) // k
    for sg in reversed(range(nseg)):
        n0, n1 = sg * k, min(nsteps, sg * k + k)
        if k != nsteps:      # re-run the segment from its checkpoint, recording tapes and outputs
            seg = snaps[sg]
            if n0 > 0:
                outs[n0 - 1] = snap(seg)      # the checkpoint is step n0 - 1's output
            for j in range(n0, n1):
                boundary(j, Ub)
                worst = max(worst, piso.step_record(seg[0], seg[1], seg[2], Ub, seg[3], tapes[j - n0],
                                                    wk=seg[4], stream=stream)[0])
                outs[j] = snap(seg)
        for j in reversed(range(n0, n1)):
            boundary(j, Ub)
            st, _ = piso.step_bwd(tapes[j - n0], Ub, wk, Ubar, pbar, phibar, pbbar, wkbar, Ubbar, nubar,
                                  info=info, stream=stream)
            worst = max(worst, st)
            if j > 0:
                seed(j - 1, outs[j - 1])
            outs.pop(j, None)
    out = dict(U=Ubar, p=pbar, phi=phibar, p_b=pbbar, U_b=Ubbar, nu=nubar, status=worst, info=info)
    if n_out:
        w = wkbar.view(n_out, 4)
        out.update(Rp=w[:, 0], C=w[:, 1], Rd=w[:, 2], pc=w[:, 3])
    return out


def _simulate_adjoint_binomial(piso, state, nsteps, loss_grad, wk, s, stream, tapes):
    U, p, phi, Ub, pb = state
    acts = binomial_schedule(nsteps, s)
    tape = tapes[0] if tapes else piso.new_tape(U.device)
    n_out = piso.opts.n_out
    worst = OK

    def snap(src):
        return [t.clone() for t in src[:4]] + [src[4].clone() if src[4] is not None else None]

    def put(dst, src):
        for a, b in zip(dst, src):
            if a is not None:
                a.copy_(b)

    cur = [U, p, phi, pb, wk]                 # the working state (the caller's tensors)
    slots = {0: snap(cur)}
    # forward: the schedule's first descent (loads, advances and saves before its first
    # record) doubles as the forward pass; one more step gives the final state
    first = next(q for q, a in enumerate(acts) if a[0] == "record")
    for a in acts[:first]:
        if a[0] == "load":
            put(cur, slots[a[1]])
        elif a[0] == "advance":
            for _ in range(a[1]):
                worst = max(worst, piso.step(cur[0], cur[1], cur[2], Ub, cur[3], wk=cur[4], stream=stream)[0])
        elif a[0] == "save":
            slots[a[1]] = snap(cur)
    at_last = snap(cur)                       # state n - 1
    worst = max(worst, piso.step(cur[0], cur[1], cur[2], Ub, cur[3], wk=cur[4], stream=stream)[0])
    Ubar, pbar, phibar, pbbar, pcbar = loss_grad(cur[0], cur[1], cur[2], cur[3], cur[4])
    final = snap(cur)
    Ubar, pbar, phibar = Ubar.clone(), pbar.clone(), phibar.clone()
    pbbar = torch.zeros_like(pb) if pbbar is None else pbbar.clone()
    wkbar = None
    if n_out:
        wkbar = torch.zeros(4 * n_out, dtype=torch.float64, device=U.device)
        if pcbar is not None:
            wkbar[3::4] = pcbar
    Ubbar = torch.zeros_like(Ub)
    nubar = torch.zeros(1, dtype=torch.float64, device=U.device)
    info = torch.zeros(PISO_INFO_NBYTES, dtype=torch.uint8, device=U.device)
    piso.adjoint_reset(stream)
    put(cur, at_last)
    for a in acts[first:]:
        kind = a[0]
        if kind == "load":
            put(cur, slots[a[1]])
        elif kind == "advance":
            for _ in range(a[1]):
                worst = max(worst, piso.step(cur[0], cur[1], cur[2], Ub, cur[3], wk=cur[4], stream=stream)[0])
        elif kind == "save":
            slots[a[1]] = snap(cur)
        elif kind == "free":
            del slots[a[1]]
        elif kind == "record":
            worst = max(worst, piso.step_record(cur[0], cur[1], cur[2], Ub, cur[3], tape, wk=cur[4],
                                                stream=stream)[0])
        elif kind == "bwd":
            st, _ = piso.step_bwd(tape, Ub, wk, Ubar, pbar, phibar, pbbar, wkbar, Ubbar, nubar, info=info,
                                  stream=stream)
            worst = max(worst, st)
    put(cur, final)                           # the caller's state ends at step n
    out = dict(U=Ubar, p=pbar, phi=phibar, p_b=pbbar, U_b=Ubbar, nu=nubar, status=worst, info=info)
    if n_out:
        w = wkbar.view(n_out, 4)
        out.update(Rp=w[:, 0], C=w[:, 1], Rd=w[:, 2], pc=w[:, 3])
    return out
