"""Pins of the CPU oracle's face operators against closed forms and invariants.

Each test fixes the oracle to something other than itself: an exact result
that the finite-volume definitions reach on a mesh where they are exact
(linear fields on uniform hexes, constant fields anywhere, the over-relaxed
split recovering g.S for a linear field), a conservation identity, or a
brute-force dense construction of a matrix from its definition (Eq. Ap_H).
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_15920_b300 import meshgen as mg

FIX, ZG, EMPTY = O.BC_FIXED, O.BC_ZEROGRAD, O.BC_EMPTY


def _om(m):
    return O.OMesh.from_mesh(m)


def _kuhn(n=5, jitter=0.2, seed=3):
    return mg.kuhn_cube(n, jitter, seed)


def test_geometry_checks():
    for m in (mg.hex_box(4, 3, 2, (1, 2, 3)), _kuhn(), mg.pipe_ohgrid(8, 4, 5), mg.channel_2d(seed=1)):
        bad, closure = O.check_geometry(_om(m))
        assert bad == 0
        assert closure < 1e-13


def test_interp_weight_places_face_value_on_face_plane():
    # linear interpolation w phi_O + (1-w) phi_N is the value of a linear
    # field at the point where the segment C_O-C_N pierces the face plane
    m = _kuhn(4, 0.25, 7)
    om = _om(m)
    w, c, k = O.face_coeffs(om)
    ni = m.n_internal
    CO, CN = m.C[m.owner[:ni]], m.C[m.neighbour]
    xs = w[:, None] * CO + (1 - w[:, None]) * CN
    S = m.Sf[:ni]
    assert np.abs(np.einsum("ij,ij->i", S, xs - m.Cf[:ni])).max() < 1e-15
    # on a uniform hex box every internal weight is exactly one half
    om2 = _om(mg.hex_box(3, 4, 5, (1.0, 0.7, 0.3)))
    np.testing.assert_allclose(O.face_coeffs(om2)[0], 0.5, rtol=1e-14)


def test_overrelaxed_split():
    # Delta = (|S|/|S^.d^|) d^  =>  |Delta| = |S|^2/(S.d) |d|,  k = S - Delta
    m = _kuhn(4, 0.25, 11)
    w, c, k = O.face_coeffs(_om(m))
    ni = m.n_internal
    d = m.C[m.neighbour] - m.C[m.owner[:ni]]
    S = m.Sf[:ni]
    Sn = np.linalg.norm(S, axis=1)
    dn = np.linalg.norm(d, axis=1)
    cos = np.einsum("ij,ij->i", S / Sn[:, None], d / dn[:, None])
    Delta = (Sn / np.abs(cos))[:, None] * d / dn[:, None]
    np.testing.assert_allclose(c[:ni] * dn, np.linalg.norm(Delta, axis=1), rtol=1e-13)
    np.testing.assert_allclose(k, S - Delta, atol=1e-15)


@pytest.mark.parametrize("scheme", [O.NONORTH_OVERRELAXED, O.NONORTH_MINIMUM, O.NONORTH_ORTHOGONAL,
                                    O.NONORTH_NONE])
def test_nonorth_split_defining_property(scheme):
    # Each split S = Delta + k of Eq. nonortho_flux (Delta along d) is fixed by one
    # geometric property: over-relaxed k . S = 0, minimum k . d = 0 (Delta the
    # projection of S on d), orthogonal |Delta| = |S|; no correction: k = 0 with
    # the two-point coefficient |S|/|d| of Eq. diff_ortho.
    m = _kuhn(4, 0.25, 11)
    w, c, k = O.face_coeffs(O.OMesh.from_mesh(m, scheme))
    ni = m.n_internal
    d = m.C[m.neighbour] - m.C[m.owner[:ni]]
    S = m.Sf[:ni]
    Sn, dn = np.linalg.norm(S, axis=1), np.linalg.norm(d, axis=1)
    Delta = c[:ni, None] * d
    if scheme == O.NONORTH_NONE:
        assert np.all(k == 0)
        np.testing.assert_allclose(c[:ni] * dn, Sn, rtol=1e-14)
    else:
        np.testing.assert_allclose(Delta + k, S, atol=1e-15)
        if scheme == O.NONORTH_OVERRELAXED:
            res = np.einsum("ij,ij->i", k, S) / Sn ** 2
        elif scheme == O.NONORTH_MINIMUM:
            res = np.einsum("ij,ij->i", k, d) / (Sn * dn)
        else:
            res = (np.linalg.norm(Delta, axis=1) - Sn) / Sn
        assert np.abs(res).max() < 1e-13
        # the correction is small but present on these jittered tetrahedra
        assert np.abs(k).max() > 1e-3 * Sn.max()
    # boundary faces have no cell-to-cell vector: the same coefficient for every scheme
    c0 = O.face_coeffs(O.OMesh.from_mesh(m))[1]
    np.testing.assert_array_equal(c[ni:], c0[ni:])


def test_nonorth_splits_agree_on_an_orthogonal_mesh():
    m = mg.hex_box(3, 4, 5, (1.0, 0.7, 0.3))
    ref = O.face_coeffs(O.OMesh.from_mesh(m))
    for scheme in (O.NONORTH_MINIMUM, O.NONORTH_ORTHOGONAL, O.NONORTH_NONE):
        w, c, k = O.face_coeffs(O.OMesh.from_mesh(m, scheme))
        np.testing.assert_allclose(c, ref[1], rtol=1e-14)
        assert np.abs(k).max() < 1e-15
    # c = |S| / h per direction: areas 0.7/4 * 0.3/5 with spacing 1/3 along x, ...
    np.testing.assert_allclose(sorted(set(np.round(ref[1][:m.n_internal], 12))),
                               sorted({round(0.7 / 4 * 0.3 / 5 * 3, 12), round(1 / 3 * 0.3 / 5 * 4 / 0.7, 12),
                                       round(1 / 3 * 0.7 / 4 * 5 / 0.3, 12)}), rtol=1e-12)


# ------------------------------------------------------------------ gradient
def test_grad_constant_is_zero_on_jittered_tets():
    m = _kuhn(6, 0.2, 1)
    om = _om(m)
    phi = np.full(m.n_cells, 3.7)
    g_fix = O.grad_gauss(om, FIX, phi, np.full(m.n_boundary, 3.7))
    g_zg = O.grad_gauss(om, ZG, phi)
    scale = 3.7 * (np.abs(m.Sf).sum() / m.n_faces) / m.V.min()
    assert np.abs(g_fix).max() < 1e-13 * scale
    assert np.abs(g_zg).max() < 1e-13 * scale


def test_grad_linear_exact_on_uniform_hex():
    m = mg.hex_box(5, 4, 3, (1.0, 2.0, 3.0), origin=(0.3, -0.2, 0.1))
    om = _om(m)
    a = np.array([[1.5, -2.0, 0.25], [0.0, 3.0, -1.0], [2.0, 0.5, 4.0]])
    b0 = np.array([0.7, -1.1, 2.0])
    phi = (m.C @ a.T + b0).T                      # [3, nc]
    phib = (m.Cf[m.n_internal:] @ a.T + b0).T     # [3, nb]
    g = O.grad_gauss(om, FIX, phi, phib)          # [3, 3, nc]
    for q in range(3):
        for d in range(3):
            np.testing.assert_allclose(g[q, d], a[q, d], atol=1e-12)


def test_grad_zero_gradient_boundary_closed_form():
    # phi = x on a row of 4 hexes: the end cells see a face value phi_O,
    # so their x-gradient is 1/2; interior cells get 1; y,z gradients vanish
    m = mg.hex_box(4, 1, 1, (1.0, 1.0, 1.0))
    g = O.grad_gauss(_om(m), ZG, m.C[:, 0])[0]
    order = np.argsort(m.C[:, 0])
    np.testing.assert_allclose(g[0][order], [0.5, 1.0, 1.0, 0.5], atol=1e-14)
    assert np.abs(g[1:]).max() < 1e-14


def test_grad_empty_faces_are_excluded():
    m = mg.channel_2d(8, 4, (2.0, 1.0, 0.1))
    om = _om(m)
    bc = om.bc_U()                                  # fixed, zg outlet, empty front/back
    phi = 2.0 * m.C[:, 0] - 3.0 * m.C[:, 1] + 5.0 * m.C[:, 2]
    phib = 2.0 * m.Cf[m.n_internal:, 0] - 3.0 * m.Cf[m.n_internal:, 1] + 5.0 * m.Cf[m.n_internal:, 2]
    g = O.grad_gauss(om, bc, phi, phib)[0]
    assert np.abs(g[2]).max() < 1e-13               # no z faces contribute
    interior = m.C[:, 0] < 2.0 - 0.25
    np.testing.assert_allclose(g[0][interior], 2.0, atol=1e-12)
    np.testing.assert_allclose(g[1], -3.0, atol=1e-12)


# ---------------------------------------------------------------- convection
@pytest.mark.parametrize("scheme", [O.DIV_UPWIND, O.DIV_LINEAR])
def test_div_constant_field_with_closed_flux_is_zero(scheme):
    m = _kuhn(5, 0.2, 5)
    om = _om(m)
    U0 = np.array([0.3, -1.2, 0.8])
    mf = m.Sf @ U0
    phi = np.full((3, m.n_cells), 1.0) * np.array([[2.0], [-1.0], [0.5]])
    phib = np.full((3, m.n_boundary), 1.0) * np.array([[2.0], [-1.0], [0.5]])
    r = O.div_flux(om, FIX, scheme, mf, phi, phib)
    assert np.abs(r).max() < 1e-14 * np.abs(mf).max() * 4


@pytest.mark.parametrize("scheme", [O.DIV_UPWIND, O.DIV_LINEAR])
def test_div_global_conservation(scheme):
    # internal faces cancel in the sum over cells; only boundary fluxes remain
    m = _kuhn(4, 0.2, 9)
    om = _om(m)
    rng = np.random.default_rng(0)
    mf = rng.standard_normal(m.n_faces)
    phi = rng.standard_normal((2, m.n_cells))
    phib = rng.standard_normal((2, m.n_boundary))
    bc = np.array([FIX, ZG, FIX, ZG, FIX, FIX], np.int32)
    r = O.div_flux(om, bc, scheme, mf, phi, phib)
    bpid = m.boundary_patch_id()
    ob = m.owner[m.n_internal:]
    for q in range(2):
        fb = np.where(bc[bpid] == FIX, phib[q], phi[q][ob])
        np.testing.assert_allclose(r[q].sum(), (mf[m.n_internal:] * fb).sum(), rtol=1e-12, atol=1e-12)


def test_div_upwind_closed_form_on_a_row():
    m = mg.hex_box(6, 1, 1, (1.0, 1.0, 1.0))
    om = _om(m)
    x = m.C[:, 0]
    phi = x ** 2
    order = np.argsort(x)
    for sgn in (1.0, -1.0):
        mf = np.zeros(m.n_faces)
        mf[np.abs(m.Sf[:, 0]) > 0] = sgn * m.Sf[np.abs(m.Sf[:, 0]) > 0, 0]   # m = sgn*u.S with u = (1,0,0)
        r = O.div_flux(om, ZG, O.DIV_UPWIND, mf, phi)[0][order]
        p = phi[order]
        if sgn > 0:       # upwind value is the left cell: R_i = phi_i - phi_{i-1}, outflow at the end
            ref = np.concatenate([[p[0] - p[0]], p[1:] - p[:-1]])
        else:             # flow from right to left: R_i = phi_i - phi_{i+1}, inflow at the end
            ref = np.concatenate([p[:-1] - p[1:], [p[-1] - p[-1]]])
        np.testing.assert_allclose(r, ref, atol=1e-14)
    rl = O.div_flux(om, ZG, O.DIV_LINEAR, np.where(np.abs(m.Sf[:, 0]) > 0, m.Sf[:, 0], 0.0), phi)[0][order]
    pf = np.concatenate([[p[0]], 0.5 * (p[1:] + p[:-1]), [p[-1]]])
    np.testing.assert_allclose(rl, pf[1:] - pf[:-1], atol=1e-14)


# ----------------------------------------------------------------- diffusion
def test_laplacian_linear_field_vanishes_on_uniform_hex():
    m = mg.hex_box(5, 4, 3, (1.0, 0.8, 1.3))
    om = _om(m)
    a = np.array([0.4, -1.3, 2.2])
    phi, phib = m.C @ a + 1.0, m.Cf[m.n_internal:] @ a + 1.0
    r = O.laplacian(om, FIX, 0.7, phi, phib)[0]
    assert np.abs(r).max() < 1e-12


def test_laplacian_quadratic_gives_2V_in_interior():
    m = mg.hex_box(6, 5, 4, (1.0, 0.9, 1.1))
    om = _om(m)
    phi = m.C[:, 0] ** 2
    r = O.laplacian(om, ZG, 1.0, phi)[0]
    x = m.C[:, 0]
    interior = (x > x.min() + 1e-9) & (x < x.max() - 1e-9)
    np.testing.assert_allclose(r[interior], 2.0 * m.V[interior], rtol=1e-10)


def test_overrelaxed_correction_recovers_gS_for_linear_field():
    # c (phi_N - phi_O) + g.k = c g.d + g.(S - c d) = g.S for linear phi with its exact gradient:
    # every interior cell of a jittered tet mesh then sums g.S over a closed surface = 0
    m = _kuhn(6, 0.2, 2)
    om = _om(m)
    g = np.array([1.3, -0.4, 2.1])
    phi, phib = m.C @ g - 0.5, m.Cf[m.n_internal:] @ g - 0.5
    grad = np.broadcast_to(g[:, None], (3, m.n_cells)).copy()
    r = O.laplacian(om, FIX, 0.9, phi, phib, grad)[0]
    r_ortho = O.laplacian(om, FIX, 0.9, phi, phib, None)[0]
    interior = np.ones(m.n_cells, bool)
    interior[m.owner[m.n_internal:]] = False
    assert np.abs(r[interior]).max() < 1e-13
    assert np.abs(r_ortho[interior]).max() > 1e-3      # the correction is doing real work


def test_laplacian_neumann_rows_sum_to_zero_and_conserve():
    m = _kuhn(4, 0.2, 4)
    om = _om(m)
    rng = np.random.default_rng(1)
    phi = rng.standard_normal(m.n_cells)
    grad = rng.standard_normal((3, m.n_cells))
    r = O.laplacian(om, ZG, 1.3, phi, None, grad)[0]
    assert abs(r.sum()) < 1e-12 * np.abs(r).sum()
    r1 = O.laplacian(om, ZG, 1.3, np.ones(m.n_cells), None, None)[0]
    assert np.abs(r1).max() < 1e-14


# ------------------------------------------------------------------- LDU apply
def _dense(m, D, L, U):
    n = m.n_cells
    A = np.zeros((n, n))
    A[np.arange(n), np.arange(n)] = D
    np.add.at(A, (m.owner[:m.n_internal], m.neighbour), U)
    np.add.at(A, (m.neighbour, m.owner[:m.n_internal]), L)
    return A


def test_ldu_apply_matches_dense_matrix_and_transpose():
    m = mg.shuffle(_kuhn(3, 0.2, 6), 5)
    om = _om(m)
    rng = np.random.default_rng(2)
    D = rng.standard_normal(m.n_cells)
    L = rng.standard_normal(m.n_internal)
    U = rng.standard_normal(m.n_internal)
    x = rng.standard_normal((3, m.n_cells))
    A = _dense(m, D, L, U)
    np.testing.assert_allclose(O.ldu_apply(om, D, L, U, x), x @ A.T, atol=1e-13)
    np.testing.assert_allclose(O.ldu_apply(om, D, U, L, x), x @ A, atol=1e-13)
    np.testing.assert_allclose(O.ldu_apply(om, D, L, None, x[0])[0], _dense(m, D, L, L) @ x[0], atol=1e-13)


# ---------------------------------------------------------------------- Krylov
def _spd(m, dt=0.01):
    om = _om(m)
    w, c, k = O.face_coeffs(om)
    D = m.V / dt + np.bincount(m.owner, c, m.n_cells) \
        + np.bincount(m.neighbour, c[:m.n_internal], m.n_cells)      # Dirichlet boundary
    return om, D, -c[:m.n_internal]


def test_pcg_matches_dense_solve():
    m = _kuhn(4, 0.2, 8)
    om, D, L = _spd(m, dt=1e3)
    b = np.random.default_rng(3).standard_normal(m.n_cells)
    x, info = O.pcg(om, D, L, None, b, tol_rel=1e-13)
    xd = np.linalg.solve(_dense(m, D, L, L), b)
    assert info["status"] == 0 and info["iters"] > 5
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-11 * np.abs(xd).max())
    assert np.linalg.norm(b - _dense(m, D, L, L) @ x) <= 1.01e-13 * np.linalg.norm(b)


def test_bicgstab_matches_dense_solve():
    m = _kuhn(4, 0.2, 10)
    om = _om(m)
    rng = np.random.default_rng(4)
    mf = rng.standard_normal(m.n_faces)
    Ub = np.zeros((3, m.n_boundary))
    D, Lo, Up, b = O.momentum_assemble(om, 0.05, 0.05, mf, rng.standard_normal((3, m.n_cells)), Ub)
    A = _dense(m, D, Lo, Up)
    assert np.abs(A - A.T).max() > 1e-3                 # genuinely non-symmetric
    x, info = O.bicgstab(om, D, Lo, Up, b[0], tol_rel=1e-13)
    xd = np.linalg.solve(A, b[0])
    assert info["status"] == 0
    np.testing.assert_allclose(x, xd, atol=1e-11 * np.abs(xd).max())


def test_krylov_zero_rhs_and_iteration_cap():
    m = _kuhn(3, 0.2, 1)
    om, D, L = _spd(m, dt=1e3)
    x, info = O.pcg(om, D, L, None, np.zeros(m.n_cells), x0=np.ones(m.n_cells))
    assert info["status"] == 0 and np.all(x == 0)
    b = np.random.default_rng(0).standard_normal(m.n_cells)
    x, info = O.pcg(om, D, L, None, b, tol_rel=1e-14, maxit=2)
    assert info["status"] == 3 and info["iters"] == 2


# ------------------------------------------------------------ momentum matrix
def test_momentum_matrix_row_sums_and_diagonal_dominance():
    # with a closed (divergence-free) flux the off-diagonal row sum cancels the
    # convective diagonal: D_i + sum_j A_ij = V/dt + sum nu c over fixed boundary faces
    m = _kuhn(4, 0.2, 12)
    om = _om(m)
    U0 = np.array([0.5, -0.2, 0.9])
    mf = m.Sf @ U0
    nu, dt = 0.03, 0.02
    D, Lo, Up, b = O.momentum_assemble(om, nu, dt, mf, np.zeros((3, m.n_cells)),
                                       np.zeros((3, m.n_boundary)))
    A = _dense(m, D, Lo, Up)
    w, c, k = O.face_coeffs(om)
    ob = m.owner[m.n_internal:]
    cb = np.bincount(ob, nu * c[m.n_internal:] - mf[m.n_internal:], m.n_cells)
    np.testing.assert_allclose(A.sum(1), m.V / dt + cb, rtol=1e-12, atol=1e-12)
    # interior rows: upwind + orthogonal diffusion leave exactly V/dt of dominance
    interior = np.ones(m.n_cells, bool)
    interior[ob] = False
    off = np.abs(A).sum(1) - np.abs(np.diag(A))
    np.testing.assert_allclose((np.diag(A) - off)[interior], (m.V / dt)[interior], rtol=1e-12)


def test_sou_deferred_correction_gives_exact_face_values_for_linear_fields():
    # Eqs. deferred_correction, sou: with the Gauss gradient exact (a linear field on
    # a uniform hex box with exact boundary values), the explicit part moves each
    # internal face's convective flux from m phi_upwind to m phi(x_f) exactly:
    # b_SOU - b_upwind = -sum_f sigma m_f (phi(x_f) - phi(x_C)), C the upwind cell.
    m = mg.hex_box(4, 3, 5, (1.0, 0.8, 1.3))
    om = _om(m)
    rng = np.random.default_rng(21)
    A0, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    lin = lambda X: A0[:, None] + B @ X.T                 # [3, n]
    U, Ub = lin(m.C), lin(m.Cf[m.n_internal:])
    mf = rng.standard_normal(m.n_faces)
    g = O.grad_gauss(om, O.BC_FIXED, U, Ub)
    np.testing.assert_allclose(g, np.broadcast_to(B[:, :, None], g.shape), atol=1e-12)
    b_up = O.momentum_assemble(om, 0.03, 0.02, mf, U, Ub)[3]
    b_sou = O.momentum_assemble(om, 0.03, 0.02, mf, U, Ub, gradS=g)[3]
    ni = m.n_internal
    o, n = m.owner[:ni], m.neighbour
    up = np.where(mf[:ni] >= 0, o, n)
    t = mf[:ni] * (lin(m.Cf[:ni]) - lin(m.C[up]))        # [3, ni]
    expect = np.zeros((3, m.n_cells))
    for q in range(3):
        expect[q] -= np.bincount(o, t[q], m.n_cells)
        expect[q] += np.bincount(n, t[q], m.n_cells)
    np.testing.assert_allclose(b_sou - b_up, expect, atol=1e-12)
    assert np.abs(expect).max() > 0.1
