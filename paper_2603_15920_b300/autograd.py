"""torch.autograd bindings of the library's hand-written adjoints (Sec. 2.5).

Every Function's forward calls a forward entry point of ``libdifvm`` and its
backward the matching ``_bwd`` entry point: the transposed gather/scatter of
the face operators, the transposed LDU apply with its coefficient gradients,
the transposed Krylov solve of implicit differentiation (Eq. implicit_diff),
the Windkessel update's derivatives and the reverse sweep of a recorded PISO
step.  Nothing here computes: arguments are marshalled, inputs the library
updates in place are cloned first, and the ``_bwd`` calls accumulate into
zero-initialised adjoint buffers.  Field layouts and numbering are those of
``difvm`` (internal numbering, SoA).
"""
from __future__ import annotations

import torch

from . import difvm as D


def _c(t):
    return None if t is None else t.contiguous()


def _zeros(t):
    return None if t is None else torch.zeros_like(t)


def _spec(t):
    """(shape, dtype, device) of an input, to allocate its adjoint later."""
    return None if t is None else (t.shape, t.dtype, t.device)


def _zeros_spec(sp):
    return None if sp is None else torch.zeros(sp[0], dtype=sp[1], device=sp[2])


# ------------------------------------------------------------ face operators
class _GradGauss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, bc_class, phi, phi_b):
        ctx.mesh, ctx.bc = mesh, bc_class
        ctx.specs = (_spec(phi), _spec(phi_b))
        return D.difvm_grad_gauss(mesh, bc_class, _c(phi), _c(phi_b))

    @staticmethod
    def backward(ctx, g):
        phi_bar, phib_bar = (_zeros_spec(sp) for sp in ctx.specs)
        D.difvm_grad_gauss_bwd(ctx.mesh, ctx.bc, g.contiguous(), phi_bar, phib_bar)
        return None, None, phi_bar, phib_bar


def grad_gauss(mesh, bc_class, phi, phi_b=None):
    """Gauss gradient [ncomp, 3, nc] of phi [ncomp, nc] (or [nc]), Eq. gauss_green."""
    return _GradGauss.apply(mesh, bc_class, phi, phi_b)


class _DivFlux(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, scheme, bc_class, mflux, phi, phi_b):
        ctx.mesh, ctx.scheme, ctx.bc = mesh, scheme, bc_class
        ctx.save_for_backward(mflux, phi, phi_b)
        return D.difvm_div_flux(mesh, scheme, bc_class, _c(mflux), _c(phi), _c(phi_b))

    @staticmethod
    def backward(ctx, g):
        mflux, phi, phi_b = ctx.saved_tensors
        m_bar, phi_bar, phib_bar = torch.zeros_like(mflux), torch.zeros_like(phi), _zeros(phi_b)
        D.difvm_div_flux_bwd(ctx.mesh, ctx.scheme, ctx.bc, _c(mflux), _c(phi), _c(phi_b), g.contiguous(),
                             m_bar, phi_bar, phib_bar)
        return None, None, None, m_bar, phi_bar, phib_bar


def div_flux(mesh, scheme, bc_class, mflux, phi, phi_b=None):
    """Convective divergence sum_f sigma m_f phi_f (upwind or linear), Eq. upwind / central."""
    return _DivFlux.apply(mesh, scheme, bc_class, mflux, phi, phi_b)


class _Laplacian(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, bc_class, gamma, phi, phi_b, grad):
        ctx.mesh, ctx.bc, ctx.gamma = mesh, bc_class, gamma
        ctx.specs = (_spec(phi), _spec(phi_b), _spec(grad))
        return D.difvm_laplacian(mesh, bc_class, gamma, _c(phi), _c(phi_b), _c(grad))

    @staticmethod
    def backward(ctx, g):
        phi_bar, phib_bar, grad_bar = (_zeros_spec(sp) for sp in ctx.specs)
        D.difvm_laplacian_bwd(ctx.mesh, ctx.bc, ctx.gamma, g.contiguous(), phi_bar, phib_bar, grad_bar)
        return None, None, None, phi_bar, phib_bar, grad_bar


def laplacian(mesh, bc_class, gamma, phi, phi_b=None, grad=None):
    """Diffusive flux sum (Eq. nonortho_flux): implicit part, plus the explicit
    non-orthogonal part when the cell gradient `grad` is given."""
    return _Laplacian.apply(mesh, bc_class, gamma, phi, phi_b, grad)


class _LduApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, diag, lower, upper, x):
        ctx.mesh = mesh
        ctx.save_for_backward(diag, lower, upper, x)
        return D.difvm_laplacian_apply(mesh, _c(diag), _c(lower), _c(upper), _c(x))

    @staticmethod
    def backward(ctx, g):
        diag, lower, upper, x = ctx.saved_tensors
        x_bar, d_bar, l_bar, u_bar = torch.zeros_like(x), torch.zeros_like(diag), _zeros(lower), _zeros(upper)
        D.difvm_laplacian_apply_bwd(ctx.mesh, _c(diag), _c(lower), _c(upper), _c(x), g.contiguous(),
                                    x_bar, d_bar, l_bar, u_bar)
        return None, d_bar, l_bar, u_bar, x_bar


def laplacian_apply(mesh, diag, lower, upper, x):
    """y = A x for the LDU matrix (diag, lower, upper; upper None = symmetric)."""
    return _LduApply.apply(mesh, diag, lower, upper, x)


# -------------------------------------------------------------------- Krylov
class _KrylovSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, opts, diag, lower, upper, b):
        ctx.mesh, ctx.opts = mesh, opts
        x = torch.zeros_like(b)
        D.difvm_krylov_solve(mesh, _c(diag), _c(lower), _c(upper), _c(b), x, opts=opts, raise_on_fail=True)
        ctx.save_for_backward(diag, lower, upper, x)
        return x

    @staticmethod
    def backward(ctx, g):
        diag, lower, upper, x = ctx.saved_tensors
        b_bar = torch.empty_like(x)     # overwritten with A^{-T} x_bar
        d_bar, l_bar, u_bar = torch.zeros_like(diag), _zeros(lower), _zeros(upper)
        st, _ = D.difvm_krylov_solve_bwd(ctx.mesh, _c(diag), _c(lower), _c(upper), x, g.contiguous(), b_bar,
                                         d_bar, l_bar, u_bar, opts=ctx.opts)
        if st != D.OK:
            raise D.DifvmError(f"transposed solve failed with status {st}")
        return None, None, d_bar, l_bar, u_bar, b_bar


def krylov_solve(mesh, diag, lower, upper, b, opts=None, **kw):
    """x = A^{-1} b by the library's Krylov solver (zero initial guess); its
    adjoint solves A^T with the same method (Eq. implicit_diff)."""
    return _KrylovSolve.apply(mesh, opts or D.solve_opts(**kw), diag, lower, upper, b)


# ---------------------------------------------------------------- Windkessel
class _Windkessel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scheme, dt, Rp, Cw, Rd, Q, pc):
        ctx.scheme, ctx.dt = scheme, dt
        pc_in = pc.detach().clone()
        pc_out, p_out = pc.detach().clone(), torch.empty_like(pc)
        D.difvm_windkessel_update(scheme, _c(Rp), _c(Cw), _c(Rd), _c(Q), dt, pc_out, p_out)
        ctx.save_for_backward(Rp, Cw, Rd, Q, pc_in)
        return pc_out, p_out

    @staticmethod
    def backward(ctx, pc_bar, p_bar):
        Rp, Cw, Rd, Q, pc_in = ctx.saved_tensors
        pc_bar = torch.zeros_like(pc_in) if pc_bar is None else pc_bar.contiguous()
        p_bar = torch.zeros_like(pc_in) if p_bar is None else p_bar.contiguous()
        pc_in_bar = torch.empty_like(pc_in)    # overwritten
        Q_bar, Rp_bar, C_bar, Rd_bar = (torch.zeros_like(t) for t in (Q, Rp, Cw, Rd))
        D.difvm_windkessel_update_bwd(ctx.scheme, _c(Rp), _c(Cw), _c(Rd), _c(Q), ctx.dt, pc_in, pc_bar, p_bar,
                                      pc_in_bar, Q_bar, Rp_bar, C_bar, Rd_bar)
        return None, None, Rp_bar, C_bar, Rd_bar, Q_bar, pc_in_bar


def windkessel_update(scheme, dt, Rp, Cw, Rd, Q, pc):
    """One RCR step (Eq. windkessel_discrete) on device double tensors [n_out]:
    returns (p_c after the step, outlet pressure p_out)."""
    return _Windkessel.apply(scheme, dt, Rp, Cw, Rd, Q, pc)


# ---------------------------------------------------------------- PISO step
class _PisoStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, piso, U, p, phi, U_b, p_b, wk, nu):
        Uo, po, phio, pbo = (t.detach().clone() for t in (U, p, phi, p_b))
        wko = None if wk is None else wk.detach().clone()
        tape = piso.new_tape(U.device)
        st, _ = piso.step_record(Uo, po, phio, _c(U_b), pbo, tape, wk=wko)
        if st != D.OK:
            raise D.DifvmError(f"PISO step failed with status {st}")
        ctx.piso, ctx.tape = piso, tape
        ctx.save_for_backward(U_b, None if wk is None else wk.detach().clone())
        ctx.has_wk, ctx.has_nu = wk is not None, nu is not None
        return (Uo, po, phio, pbo) if wk is None else (Uo, po, phio, pbo, wko)

    @staticmethod
    def backward(ctx, *gs):
        U_b, wk_in = ctx.saved_tensors
        gU, gp, gphi, gpb = gs[:4]
        U_bar = gU.contiguous().clone()
        p_bar = gp.contiguous().clone()
        phi_bar = gphi.contiguous().clone()
        pb_bar = gpb.contiguous().clone()
        wk_bar = gs[4].contiguous().clone() if ctx.has_wk else None
        Ub_bar = torch.zeros_like(U_b)
        nu_bar = torch.zeros(1, dtype=torch.float64, device=U_b.device)
        st, _ = ctx.piso.step_bwd(ctx.tape, _c(U_b), wk_in, U_bar, p_bar, phi_bar, pb_bar, wk_bar, Ub_bar, nu_bar)
        if st != D.OK:
            raise D.DifvmError(f"PISO step adjoint failed with status {st}")
        return (None, U_bar, p_bar, phi_bar, Ub_bar, pb_bar, wk_bar,
                nu_bar if ctx.has_nu else None)


def piso_step(piso, U, p, phi, U_b, p_b, wk=None, nu=None):
    """One PISO step (Sec. 2.4.2) as a differentiable function of (U, p, phi,
    U_b, p_b, wk): returns new tensors (U, p, phi, p_b[, wk]); the inputs are
    left unchanged.  The step's tape lives until the graph is freed.  Pass a
    one-element FP64 tensor `nu` (equal to the handle's viscosity; it is not
    read) to receive d(loss)/d(nu) in nu.grad."""
    return _PisoStep.apply(piso, U, p, phi, U_b, p_b, wk, nu)
