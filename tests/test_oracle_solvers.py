"""Pins of the CPU oracle's solvers, Windkessel and PISO step.

  * manufactured Poisson solution of Sec. 3.1.1 (closed form, second order on a
    smoothly distorted non-orthogonal mesh; the uncorrected scheme stalls),
  * RCR Windkessel against the closed-form ODE solution (Eqs. windkessel_ode,
    windkessel_discrete) and the first-order FE/BE rates,
  * PISO (Sec. 2.4.2): free-stream preservation on jittered tets, the
    Poiseuille channel against its discrete fully developed profile and the
    parabola, per-cell continuity after the last corrector, the pressure pin of
    an all-Neumann cavity, and the Windkessel outlet coupling.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_15920_b300 import meshgen as mg


def _om(m):
    return O.OMesh.from_mesh(m)


# ------------------------------------------------------------ Poisson, Sec. 3.1.1
def _phi_gt(X):
    x, y, z = X.T
    return 2 * np.sin(np.pi * x) * (y ** 4 - y) * np.sin(2 * np.pi * z) + 10


def _f(X):
    x, y, z = X.T
    s = np.sin(np.pi * x) * np.sin(2 * np.pi * z)
    return -10 * np.pi ** 2 * s * (y ** 4 - y) + 24 * s * y ** 2


def _poisson(m, nonorth=True, scheme=O.NONORTH_OVERRELAXED):
    om = O.OMesh.from_mesh(m, scheme)
    w, c, k = O.face_coeffs(om)
    D = np.bincount(m.owner, c, m.n_cells) + np.bincount(m.neighbour, c[:m.n_internal], m.n_cells)
    L = -c[:m.n_internal]
    pb = np.full(m.n_boundary, 10.0)
    phi = np.full(m.n_cells, 10.0)
    src = _f(m.C) * m.V
    for _ in range(80):           # defect correction on the lagged non-orthogonal term
        g = O.grad_gauss(om, O.BC_FIXED, phi, pb)[0] if nonorth else None
        r = O.laplacian(om, O.BC_FIXED, 1.0, phi, pb, g)[0] - src
        d, info = O.pcg(om, D, L, None, r, tol_rel=1e-12)
        assert info["status"] == 0
        phi += d
        if np.abs(d).max() < 1e-12:
            break
    e = phi - _phi_gt(m.C)
    return np.sqrt((e ** 2 * m.V).sum()), np.abs(e).max()


def test_manufactured_solution_is_exact_for_the_pde():
    # the printed source is the Laplacian of the printed solution, which is 10 on the cube sides
    X = np.random.default_rng(0).uniform(0.05, 0.95, (50, 3))
    h = 1e-4
    lap = sum((_phi_gt(X + h * e) - 2 * _phi_gt(X) + _phi_gt(X - h * e)) / h ** 2 for e in np.eye(3))
    np.testing.assert_allclose(lap, _f(X), rtol=1e-5, atol=1e-5)
    B = np.random.default_rng(1).uniform(0, 1, (60, 3))
    for ax in range(3):
        for v in (0.0, 1.0):
            Bs = B.copy(); Bs[:, ax] = v
            np.testing.assert_allclose(_phi_gt(Bs), 10.0, atol=1e-14)


def test_poisson_second_order_with_overrelaxed_correction():
    e = [_poisson(mg.distorted_box(n, 0.05)) for n in (8, 16, 32)]
    l2 = [a for a, b in e]
    orders = np.log2(np.array(l2[:-1]) / np.array(l2[1:]))
    assert np.all(orders > 1.9), orders
    mx = [b for a, b in e]
    assert np.log2(mx[1] / mx[2]) > 1.5


@pytest.mark.parametrize("scheme", [O.NONORTH_MINIMUM, O.NONORTH_ORTHOGONAL])
def test_poisson_second_order_with_minimum_and_orthogonal_corrections(scheme):
    # the other two corrected splits of Eq. nonortho_flux are second order too
    l2 = [_poisson(mg.distorted_box(n, 0.05), scheme=scheme)[0] for n in (8, 16, 32)]
    orders = np.log2(np.array(l2[:-1]) / np.array(l2[1:]))
    assert np.all(orders > 1.9), orders


def test_poisson_two_point_flux_does_not_converge():
    # Eq. diff_ortho alone (no correction) on the distorted mesh stalls
    l2 = [_poisson(mg.distorted_box(n, 0.05), nonorth=False, scheme=O.NONORTH_NONE)[0] for n in (8, 16, 32)]
    assert np.log2(l2[1] / l2[2]) < 0.5


def test_poisson_without_correction_does_not_converge():
    # the same mesh without the non-orthogonal term stalls: the pin above has teeth
    l2 = [_poisson(mg.distorted_box(n, 0.05), nonorth=False)[0] for n in (8, 16, 32)]
    assert np.log2(l2[1] / l2[2]) < 0.5


def test_poisson_uniform_hex_second_order():
    l2 = [_poisson(mg.hex_box(n, n, n))[0] for n in (8, 16)]
    assert np.log2(l2[0] / l2[1]) > 1.9


# ----------------------------------------------------------------- Windkessel
def test_windkessel_exact_update_matches_ode_solution():
    Rp, Cw, Rd, Q, pc0 = 0.1, 0.7, 1.3, 2.5, 0.4
    dt, n = 0.013, 250
    pc = np.array([pc0])
    for _ in range(n):
        pc, po = O.windkessel_update(O.WK_EXACT, Rp, Cw, Rd, Q, dt, pc)
    t = n * dt
    exact = Rd * Q + (pc0 - Rd * Q) * np.exp(-t / (Rd * Cw))
    np.testing.assert_allclose(pc[0], exact, rtol=1e-13)
    np.testing.assert_allclose(po[0], exact + Rp * Q, rtol=1e-13)


@pytest.mark.parametrize("scheme", [O.WK_FE, O.WK_BE])
def test_windkessel_fe_be_first_order(scheme):
    Rp, Cw, Rd, Q, pc0, T = 0.1, 1.0, 1.0, 1.0, 0.0, 1.0

    def run(n):
        pc = np.array([pc0])
        for _ in range(n):
            pc, _ = O.windkessel_update(scheme, Rp, Cw, Rd, Q, T / n, pc)
        return pc[0]
    exact = Rd * Q + (pc0 - Rd * Q) * np.exp(-T / (Rd * Cw))
    e1, e2 = abs(run(100) - exact), abs(run(200) - exact)
    assert 1.9 < e1 / e2 < 2.1


def test_windkessel_steady_state_and_multiple_outlets():
    Rp = np.array([0.1, 0.2]); Cw = np.array([1.0, 0.5]); Rd = np.array([1.0, 2.0])
    Q = np.array([1.5, 0.3]); pc = np.zeros(2)
    for _ in range(4000):
        pc, po = O.windkessel_update(O.WK_EXACT, Rp, Cw, Rd, Q, 0.01, pc)
    np.testing.assert_allclose(po, (Rp + Rd) * Q, rtol=1e-12)


# ----------------------------------------------------------------------- PISO
def _freestream_mesh():
    return mg.kuhn_cube(4, 0.2, 5, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET))


def test_piso_preserves_free_stream_on_jittered_tets():
    m = _freestream_mesh()
    om = _om(m)
    U0 = np.array([1.0, 0.0, 0.0])
    Ub = np.broadcast_to(U0[:, None], (3, m.n_boundary)).copy()
    U = np.broadcast_to(U0[:, None], (3, m.n_cells)).copy()
    p = np.zeros(m.n_cells)
    pb = np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    for _ in range(3):
        U, p, phi, pb, _, info = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.01)
        assert info["status"] == 0
    assert np.abs(U - U0[:, None]).max() < 1e-12
    assert np.abs(p).max() < 1e-12


def _discrete_fully_developed(ny, nu, H=1.0, Umean=1.0):
    """Fully developed channel profile of the same cell-centred scheme.

    Rows: nu/h^2 (u_{j+1} - 2u_j + u_{j-1}) = G with the wall faces at h/2
    (coefficient 2/h), closed by the flow rate sum u_j h = Umean H."""
    h = H / ny
    A = np.zeros((ny + 1, ny + 1))
    rhs = np.zeros(ny + 1)
    for j in range(ny):
        A[j, j] = -2 - (1 if j in (0, ny - 1) else 0)
        if j > 0:
            A[j, j - 1] = 1
        if j < ny - 1:
            A[j, j + 1] = 1
        A[j] *= nu / h ** 2
        A[j, ny] = -1
    A[ny, :ny] = h
    rhs[ny] = Umean * H
    s = np.linalg.solve(A, rhs)
    return s[:ny], s[ny]


def test_poiseuille_channel_steady_profile():
    m = mg.channel_2d(64, 16)
    om = _om(m)
    nu = 0.05
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("inlet") - m.n_internal] = 1.0
    pb = np.zeros(m.n_boundary)
    U = np.zeros((3, m.n_cells)); p = np.zeros(m.n_cells)
    phi = O.flux_from_U(om, U, Ub)
    for _ in range(400):
        U1, p, phi, pb, _, info = O.piso_step(om, U, p, phi, Ub, pb, nu=nu, dt=0.05,
                                              tolU=1e-13, tolp=1e-13)
        assert info["status"] == 0
        dU = np.abs(U1 - U).max()
        U = U1
        if dU < 1e-12:
            break
    assert dU < 1e-12
    u1d, G = _discrete_fully_developed(16, nu)
    x, y = m.C[:, 0], m.C[:, 1]
    last = np.abs(x - x.max()) < 1e-9
    prof = U[0, last][np.argsort(y[last])]
    yy = np.sort(y[last])
    np.testing.assert_allclose(prof, u1d, atol=2e-5)                 # discrete closed form
    np.testing.assert_allclose(prof, 6 * yy * (1 - yy), atol=0.01)    # parabola, 16 cells
    assert abs(G - (-12 * nu)) < 0.01
    assert np.abs(U[1][x > 3.0]).max() < 1e-4 and np.abs(U[2]).max() == 0.0
    # developed region: p is linear with slope G of the discrete problem
    gp = O.grad_gauss(om, om.bc_p(), p, pb)[0][0]
    np.testing.assert_allclose(gp[np.abs(x - 3.90625) < 1e-9], G, rtol=1e-4)


def _continuity(m, phi, bcU):
    r = np.bincount(m.owner, phi, m.n_cells) - np.bincount(m.neighbour, phi[:m.n_internal], m.n_cells)
    return np.abs(r).max() / np.abs(phi).max()


def test_piso_continuity_after_last_corrector_lid_cavity():
    # all-Neumann pressure (every patch a wall): the pinned cell carries p = 0
    m = mg.kuhn_cube(4, 0.2, 8)
    om = _om(m)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    U = np.zeros((3, m.n_cells)); p = np.zeros(m.n_cells); pb = np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    for _ in range(3):
        U, p, phi, pb, _, info = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.02,
                                             tolp=1e-12, pref_cell=5)
        assert info["status"] == 0
        assert _continuity(m, phi, None) < 1e-10
        assert abs(p[5]) < 1e-10 * np.abs(p).max()
    assert np.abs(U).max() > 0.1
    # no flux through the walls: the lid moves tangentially
    assert np.abs(phi[m.n_internal:]).max() < 1e-15


def test_piso_windkessel_outlet_coupling():
    m = mg.channel_2d(16, 8)
    om = _om(m)
    out = m.patch_index("outlet")
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("inlet") - m.n_internal] = 1.0
    U = np.zeros((3, m.n_cells)); p = np.zeros(m.n_cells); pb = np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    Rp, Cw, Rd = 0.1, 1.0, 2.0
    pc = np.array([0.0])
    pc_ref = 0.0
    dt = 0.02
    for _ in range(5):
        Q = phi[m.patch_faces("outlet")].sum()
        U, p, phi, pb, pc, info = O.piso_step(om, U, p, phi, Ub, pb, nu=0.05, dt=dt,
                                              wk_patch=[out], Rp=[Rp], Cw=[Cw], Rd=[Rd], pc=pc)
        e = np.exp(-dt / (Rd * Cw))
        pc_ref = pc_ref * e + Rd * Q * (1 - e)
        np.testing.assert_allclose(info["Q"][0], Q, rtol=1e-14)
        np.testing.assert_allclose(pc[0], pc_ref, rtol=1e-13)
        np.testing.assert_allclose(pb[m.patch_faces("outlet") - m.n_internal], pc_ref + Rp * Q, rtol=1e-13)
    # after the first step all inflow leaves through the outlet
    inflow = -phi[m.patch_faces("inlet")].sum()
    np.testing.assert_allclose(phi[m.patch_faces("outlet")].sum(), inflow, rtol=1e-9)


# ----------------------------------------------------------- limited correction
def _cavity_run(n, dt, psi, steps, jitter=0.2):
    m = mg.kuhn_cube(n, jitter, 0)
    om = _om(m)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    peak = []
    for _ in range(steps):
        U, p, phi, pb, _, info = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=dt, psi=psi)
        assert info["status"] == 0
        peak.append(np.abs(U).max())
    return np.array(peak)


def test_limited_nonorthogonal_correction_keeps_the_tet_cavity_bounded():
    # jittered Kuhn tets (max non-orthogonality ~65 deg) at CFL ~0.25: the lagged,
    # unlimited over-relaxed pressure correction feeds a growing mode; capping the
    # explicit part at psi/(1-psi) = 1/2 of the orthogonal part keeps |U| below the lid speed
    limited = _cavity_run(16, 0.016, 1.0 / 3.0, 14)
    assert limited.max() < 1.0
    unlimited = _cavity_run(16, 0.016, 1.0, 14)
    assert unlimited.max() > 2.0


def test_limiter_caps_the_explicit_correction():
    m = mg.kuhn_cube(4, 0.2, 3)
    om = _om(m)
    rng = np.random.default_rng(0)
    U = rng.standard_normal((3, m.n_cells))
    g = 50.0 * rng.standard_normal((3, 3, m.n_cells))     # large gradients: the cap is active
    zero = np.zeros((3, m.n_boundary))
    mf = np.zeros(m.n_faces)
    nu, dt, psi = 0.3, 1.0, 0.25
    b_plain = O.momentum_assemble(om, nu, dt, mf, U, zero, None)[3]
    b_full = O.momentum_assemble(om, nu, dt, mf, U, zero, g)[3]
    b_lim = O.momentum_assemble(om, nu, dt, mf, U, zero, g, psi=psi)[3]
    # per-cell bound: the limited correction of every face is at most psi/(1-psi) |orth|
    w, c, k = O.face_coeffs(om)
    ni = m.n_internal
    orth = np.abs(c[:ni] * (U[:, m.neighbour] - U[:, m.owner[:ni]]))      # [3, ni]
    bound = np.zeros((3, m.n_cells))
    for q in range(3):
        np.add.at(bound[q], m.owner[:ni], nu * psi / (1 - psi) * orth[q])
        np.add.at(bound[q], m.neighbour, nu * psi / (1 - psi) * orth[q])
    assert np.all(np.abs(b_lim - b_plain) <= bound * (1 + 1e-12) + 1e-15)
    assert np.abs(b_full - b_plain).max() > 2 * np.abs(b_lim - b_plain).max()
    # psi = 1 is the unlimited over-relaxed correction
    np.testing.assert_array_equal(O.momentum_assemble(om, nu, dt, mf, U, zero, g, psi=1.0)[3], b_full)


def test_crank_nicolson_momentum_rows_are_second_order_in_time():
    # The momentum rows as a linear ODE V dU/dt = -(A U - b) (fixed face flux, no
    # pressure): backward Euler is first order in dt, the Crank-Nicolson form of
    # the rows second order, against the matrix exponential of the same system.
    from scipy.linalg import expm
    m = mg.kuhn_cube(2, 0.2, 4)
    om = _om(m)
    rng = np.random.default_rng(8)
    mf = O.flux_from_U(om, np.tile([[0.6], [-0.3], [0.2]], (1, m.n_cells)), np.tile([[0.6], [-0.3], [0.2]],
                                                                                        (1, m.n_boundary)))
    Ub = rng.standard_normal((3, m.n_boundary))
    U0 = rng.standard_normal((3, m.n_cells))
    nu, T = 0.05, 0.2
    nc, ni = m.n_cells, m.n_internal

    def dense(D, Lo, Up):
        A = np.diag(D)
        A[m.owner[:ni], m.neighbour] += Up
        A[m.neighbour, m.owner[:ni]] += Lo
        return A

    D, Lo, Up, b = O.momentum_assemble(om, nu, 1.0, mf, U0, Ub)
    Acd = dense(D - m.V, Lo, Up)                    # dt = 1: D = V + D_cd
    bcd = b - m.V * U0
    Uinf = np.linalg.solve(Acd, bcd.T).T
    E = expm(-np.diag(1.0 / m.V) @ Acd * T)
    exact = Uinf + (E @ (U0 - Uinf).T).T
    err = {}
    for time in (O.TIME_BE, O.TIME_CN):
        err[time] = []
        for n in (8, 16, 32):
            dt, U = T / n, U0.copy()
            for _ in range(n):
                D, Lo, Up, b = O.momentum_assemble(om, nu, dt, mf, U, Ub, time=time)
                U = np.linalg.solve(dense(D, Lo, Up), b.T).T
            err[time].append(np.abs(U - exact).max())
    be = np.log2(np.array(err[O.TIME_BE][:-1]) / np.array(err[O.TIME_BE][1:]))
    cn = np.log2(np.array(err[O.TIME_CN][:-1]) / np.array(err[O.TIME_CN][1:]))
    assert np.all(np.abs(be - 1) < 0.15), be
    assert np.all(np.abs(cn - 2) < 0.1), cn
