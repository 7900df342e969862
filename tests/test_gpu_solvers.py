"""GPU parity of the Krylov solvers, the Windkessel and the PISO step.

Every GPU result is compared with the FP64 CPU oracle on the same seeded
inputs, in the input numbering.  Bars: FP64 1e-12 per operator / 1e-9 per
solved step; FP32 with FP64 refinement 1e-4 on fields.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_15920_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_15920_b300 import difvm as D  # noqa: E402


def nrel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cuda(x, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda").contiguous()


def host(t):
    return t.double().cpu().numpy()


@pytest.fixture(scope="module")
def kuhn():
    m = mg.shuffle(mg.kuhn_cube(10, 0.2, 3, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET)), 11)
    return m, O.OMesh.from_mesh(m), D.Mesh(m)


def _face_to_internal(dm, L, U):
    """Input-numbered lower/upper -> internal (swap on re-oriented faces)."""
    ni = dm.ni
    idx = dm.face_old_of_new[:ni]
    flip = dm.face_flip[:ni] != 0
    return np.where(flip, U[idx], L[idx]), np.where(flip, L[idx], U[idx])


def _spd(m, om, dt=0.05):
    w, c, k = O.face_coeffs(om)
    Dg = m.V / dt + np.bincount(m.owner, c, m.n_cells) + np.bincount(m.neighbour, c[:m.n_internal], m.n_cells)
    return Dg, -c[:m.n_internal]


@pytest.mark.parametrize("dt", [0.05, 1e3])
def test_pcg_f64_matches_oracle(kuhn, dt):
    m, om, dm = kuhn
    Dg, L = _spd(m, om, dt)
    b = np.random.default_rng(0).standard_normal(m.n_cells)
    x0 = np.random.default_rng(1).standard_normal(m.n_cells)
    xr, ir = O.pcg(om, Dg, L, None, b, x0=x0, tol_rel=1e-12, maxit=5000)
    Li, _ = _face_to_internal(dm, L, L)
    x = cuda(dm.to_cells(x0))
    st, info = D.difvm_krylov_solve(dm, cuda(dm.to_cells(Dg)), cuda(Li), None, cuda(dm.to_cells(b)), x,
                                    method=D.PCG, tol_rel=1e-12, max_iter=5000)
    assert st == D.OK and info[0]["status"] == D.OK
    assert abs(info[0]["iters"] - ir["iters"]) <= 1, (info[0]["iters"], ir["iters"])
    assert nrel(dm.from_cells(host(x)), xr) < 1e-9
    assert info[0]["res"] <= 1e-12 * info[0]["bnorm"] * 1.0001


def test_bicgstab_f64_three_components_match_oracle(kuhn):
    m, om, dm = kuhn
    rng = np.random.default_rng(2)
    mf = m.Sf @ np.array([0.7, -0.3, 0.4]) + 0.05 * rng.standard_normal(m.n_faces)
    Dg, Lo, Up, b = O.momentum_assemble(om, 0.02, 0.02, mf, rng.standard_normal((3, m.n_cells)),
                                        rng.standard_normal((3, m.n_boundary)))
    ref = [O.bicgstab(om, Dg, Lo, Up, b[c], tol_rel=1e-12) for c in range(3)]
    Li, Ui = _face_to_internal(dm, Lo, Up)
    x = torch.zeros(3, m.n_cells, dtype=torch.float64, device="cuda")
    st, info = D.difvm_krylov_solve(dm, cuda(dm.to_cells(Dg)), cuda(Li), cuda(Ui), cuda(dm.to_cells(b)),
                                    x, method=D.BICGSTAB, tol_rel=1e-12)
    assert st == D.OK
    got = dm.from_cells(host(x))
    for c in range(3):
        assert nrel(got[c], ref[c][0]) < 1e-9
        # BiCGStab's iteration count is sensitive to rounding; the residual is the contract
        assert info[c]["status"] == D.OK and info[c]["res"] <= 1e-12 * info[c]["bnorm"] * 1.0001
        assert info[c]["iters"] <= 2 * ref[c][1]["iters"] + 5


def test_pcg_f32_and_refinement(kuhn):
    m, om, dm = kuhn
    Dg, L = _spd(m, om, 0.05)
    D32, L32 = Dg.astype(np.float32), L.astype(np.float32)
    b = np.random.default_rng(3).standard_normal(m.n_cells)
    # reference: the FP32-rounded matrix solved in FP64 by the oracle
    xr, _ = O.pcg(om, D32.astype(np.float64), L32.astype(np.float64), None, b, tol_rel=1e-13)
    Li, _ = _face_to_internal(dm, L32, L32)
    x32 = torch.zeros(m.n_cells, dtype=torch.float32, device="cuda")
    st, info = D.difvm_krylov_solve(dm, cuda(dm.to_cells(D32), torch.float32), cuda(Li, torch.float32), None,
                                    cuda(dm.to_cells(b), torch.float32), x32, method=D.PCG, tol_rel=1e-6)
    assert st == D.OK
    assert nrel(dm.from_cells(host(x32)), xr) < 1e-5
    x64 = torch.zeros(m.n_cells, dtype=torch.float64, device="cuda")
    st, info = D.difvm_krylov_solve_refine(dm, cuda(dm.to_cells(D32), torch.float32), cuda(Li, torch.float32),
                                           None, cuda(dm.to_cells(b)), x64, method=D.PCG, tol_rel=1e-10,
                                           max_iter=5000)
    assert st == D.OK, info
    assert info[0]["refinements"] >= 2
    assert info[0]["res"] <= 1e-10 * info[0]["bnorm"]
    assert nrel(dm.from_cells(host(x64)), xr) < 1e-8


def test_krylov_status_codes(kuhn):
    m, om, dm = kuhn
    Dg, L = _spd(m, om, 0.05)
    Li, _ = _face_to_internal(dm, L, L)
    # zero right-hand side: x = 0 without iterating
    x = torch.ones(m.n_cells, dtype=torch.float64, device="cuda")
    st, info = D.difvm_krylov_solve(dm, cuda(dm.to_cells(Dg)), cuda(Li), None,
                                    torch.zeros_like(x), x, method=D.PCG)
    assert st == D.OK and info[0]["iters"] == 0 and float(x.abs().max()) == 0.0
    # iteration cap
    b = cuda(np.random.default_rng(0).standard_normal(m.n_cells))
    x = torch.zeros_like(b)
    st, info = D.difvm_krylov_solve(dm, cuda(dm.to_cells(Dg)), cuda(Li), None, b, x, method=D.PCG,
                                    tol_rel=1e-14, max_iter=3)
    assert st == D.ENOTCONV and info[0]["iters"] == 3 and info[0]["status"] == D.ENOTCONV
    # non-finite right-hand side is reported, not hung on
    bn = b.clone(); bn[5] = float("nan")
    x = torch.zeros_like(b)
    st, info = D.difvm_krylov_solve(dm, cuda(dm.to_cells(Dg)), cuda(Li), None, bn, x, method=D.PCG)
    assert st == D.ENONFINITE


def test_krylov_bwd_adjoint_and_coefficient_gradients(kuhn):
    m, om, dm = kuhn
    rng = np.random.default_rng(5)
    mf = m.Sf @ np.array([0.7, -0.3, 0.4])
    Dg, Lo, Up, _ = O.momentum_assemble(om, 0.02, 0.02, mf, np.zeros((3, m.n_cells)), np.zeros((3, m.n_boundary)))
    b = rng.standard_normal(m.n_cells)
    xbar = rng.standard_normal(m.n_cells)
    x, _ = O.bicgstab(om, Dg, Lo, Up, b, tol_rel=1e-13)
    Li, Ui = _face_to_internal(dm, Lo, Up)
    Dd, Ld, Ud = cuda(dm.to_cells(Dg)), cuda(Li), cuda(Ui)
    bbar = torch.zeros(m.n_cells, dtype=torch.float64, device="cuda")
    Dbar, Lbar, Ubar = torch.zeros_like(Dd), torch.zeros_like(Ld), torch.zeros_like(Ud)
    st, _ = D.difvm_krylov_solve_bwd(dm, Dd, Ld, Ud, cuda(dm.to_cells(x)), cuda(dm.to_cells(xbar)), bbar,
                                     Dbar, Lbar, Ubar, method=D.BICGSTAB, tol_rel=1e-13)
    assert st == D.OK
    # b_bar = A^{-T} x_bar: the oracle solve with lower and upper swapped
    ref, _ = O.bicgstab(om, Dg, Up, Lo, xbar, tol_rel=1e-13)
    assert nrel(dm.from_cells(host(bbar)), ref) < 1e-9
    # coefficient gradients against central differences of <x_bar, x(A)>
    def L_of(Dx, Lx, Ux):
        xx, _ = O.bicgstab(om, Dx, Lx, Ux, b, tol_rel=1e-14)
        return xbar @ xx
    Dbar_in = dm.from_cells(host(Dbar))
    for i in rng.choice(m.n_cells, 4, replace=False):
        h = 1e-6 * abs(Dg[i])
        Dp, Dm = Dg.copy(), Dg.copy(); Dp[i] += h; Dm[i] -= h
        fd = (L_of(Dp, Lo, Up) - L_of(Dm, Lo, Up)) / (2 * h)
        assert abs(fd - Dbar_in[i]) < 1e-6 * max(1.0, abs(fd))
    idx = dm.face_old_of_new[:m.n_internal]
    flip = dm.face_flip[:m.n_internal] != 0
    Lbar_h, Ubar_h = host(Lbar), host(Ubar)
    for k in rng.choice(m.n_internal, 4, replace=False):
        f = idx[k]
        h = 1e-6
        Lp_, Lm_ = Lo.copy(), Lo.copy(); Lp_[f] += h; Lm_[f] -= h
        fd = (L_of(Dg, Lp_, Up) - L_of(Dg, Lm_, Up)) / (2 * h)
        got = Ubar_h[k] if flip[k] else Lbar_h[k]
        assert abs(fd - got) < 1e-6 * max(1.0, abs(fd))


# ---------------------------------------------------------------- Windkessel
@pytest.mark.parametrize("scheme", [D.WK_EXACT, D.WK_FE, D.WK_BE])
def test_windkessel_update_and_bwd(scheme):
    rng = np.random.default_rng(0)
    n = 5
    Rp, Cw, Rd = rng.uniform(0.05, 0.3, n), rng.uniform(0.5, 1.5, n), rng.uniform(0.5, 2.0, n)
    Q, pc0, dt = rng.uniform(-1, 2, n), rng.uniform(0, 1, n), 0.013
    pc_ref, po_ref = O.windkessel_update(scheme, Rp, Cw, Rd, Q, dt, pc0)
    pc = cuda(pc0); po = torch.zeros_like(pc)
    D.difvm_windkessel_update(scheme, cuda(Rp), cuda(Cw), cuda(Rd), cuda(Q), dt, pc, po)
    assert nrel(host(pc), pc_ref) < 1e-14 and nrel(host(po), po_ref) < 1e-14
    # adjoint vs central differences of the oracle
    gpc, gpo = rng.standard_normal(n), rng.standard_normal(n)
    bars = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(5)]
    D.difvm_windkessel_update_bwd(scheme, cuda(Rp), cuda(Cw), cuda(Rd), cuda(Q), dt, cuda(pc0), cuda(gpc),
                                  cuda(gpo), *bars)
    args = dict(pc=pc0, Q=Q, Rp=Rp, Cw=Cw, Rd=Rd)
    def J(a):
        pcn, pon = O.windkessel_update(scheme, a["Rp"], a["Cw"], a["Rd"], a["Q"], dt, a["pc"])
        return gpc @ pcn + gpo @ pon
    for name, bar in zip(["pc", "Q", "Rp", "Cw", "Rd"], bars):
        fd = np.zeros(n)
        for o in range(n):
            h = 1e-6 * max(1.0, abs(args[name][o]))
            ap = {k: v.copy() for k, v in args.items()}; am = {k: v.copy() for k, v in args.items()}
            ap[name][o] += h; am[name][o] -= h
            fd[o] = (J(ap) - J(am)) / (2 * h)
        assert np.abs(host(bar) - fd).max() < 1e-7 * max(1.0, np.abs(fd).max()), name


# ---------------------------------------------------------------------- PISO
def _state_to_gpu(dm, U, p, phi, Ub, pb, dt=torch.float64):
    return (cuda(dm.to_cells(U), dt), cuda(dm.to_cells(p), dt), cuda(dm.to_faces(phi), dt),
            cuda(dm.to_bnd(Ub), dt), cuda(dm.to_bnd(pb), dt))


def _piso(dm, prec, nu, dt, pref=0, tol=1e-12, refine=0, wk_patch=(), ncorr=2, psi=1.0, nonorth=True):
    o = D.piso_opts(nu, dt, ncorr, nonorth,
                    solve_U=D.solve_opts(D.BICGSTAB, tol, max_iter=2000),
                    solve_p=D.solve_opts(D.PCG, tol, max_iter=20000, refine_max=refine),
                    pref_cell=int(dm.cell_new_of_old[pref]), wk_patch=wk_patch, nonorth_limit=psi)
    return D.Piso(dm, prec, o)


def _channel_bc(m):
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("inlet") - m.n_internal] = 1.0
    return Ub


def test_piso_channel_per_step_parity_f64():
    """Poiseuille channel (64x16 hexes, shuffled ids; the run is 200 steps of
    dt = 0.01): one GPU step from the oracle's state at every tenth step of the
    whole trajectory: 1e-9 per solved step."""
    m = mg.channel_2d(64, 16, seed=7)
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    nu, dt = 0.05, 0.01
    Ub, pb = _channel_bc(m), np.zeros(m.n_boundary)
    U, p = np.zeros((3, m.n_cells)), np.zeros(m.n_cells)
    phi = O.flux_from_U(om, U, Ub)
    pg = _piso(dm, D.F64, nu, dt)
    worst = 0.0
    for step in range(200):
        g = _state_to_gpu(dm, U, p, phi, Ub, pb) if step % 10 == 0 else None
        if g is not None:
            st, info = pg.step(*g)
            assert st == D.OK
        U, p, phi, pb, _, oi = O.piso_step(om, U, p, phi, Ub, pb, nu=nu, dt=dt, tolU=1e-12, tolp=1e-12)
        if g is None:
            continue
        for got, ref in ((dm.from_cells(host(g[0])), U), (dm.from_cells(host(g[1])), p),
                         (dm.from_faces(host(g[2])), phi)):
            worst = max(worst, nrel(got, ref))
        gi = D.decode_piso_info(info)
        assert abs(gi["itp"][0] - oi["itp"][0]) <= 2
    assert worst < 1e-9, worst


def test_piso_channel_trajectory_f64():
    """The channel run as a whole trajectory, all 200 steps (dt = 0.01, t = 2):
    GPU and oracle evolve independently from the same initial state."""
    m = mg.channel_2d(64, 16, seed=3)
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    nu, dt = 0.05, 0.01
    Ub, pb = _channel_bc(m), np.zeros(m.n_boundary)
    U, p = np.zeros((3, m.n_cells)), np.zeros(m.n_cells)
    phi = O.flux_from_U(om, U, Ub)
    g = _state_to_gpu(dm, U, p, phi, Ub, pb)
    pg = _piso(dm, D.F64, nu, dt)
    for _ in range(200):
        assert pg.step(*g)[0] == D.OK
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=nu, dt=dt, tolU=1e-12, tolp=1e-12)
    errs = (nrel(dm.from_cells(host(g[0])), U), nrel(dm.from_cells(host(g[1])), p),
            nrel(dm.from_faces(host(g[2])), phi))
    assert max(errs) < 1e-8, errs


def _cavity(n=6, seed=8):
    m = mg.shuffle(mg.kuhn_cube(n, 0.2, seed), seed + 1)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    return m, Ub


@pytest.mark.parametrize("psi,mask", [(1.0, 3), (1.0 / 3.0, 3), (1.0, 1)])
def test_piso_lid_cavity_f64_pinned_pressure(psi, mask):
    m, Ub = _cavity()
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    pref = 17
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    pg = _piso(dm, D.F64, 0.01, 0.05, pref=pref, psi=psi, nonorth=mask)
    worst = 0.0
    for _ in range(4):
        g = _state_to_gpu(dm, U, p, phi, Ub, pb)
        assert pg.step(*g)[0] == D.OK
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.05, tolU=1e-12,
                                          tolp=1e-12, pref_cell=pref, psi=psi, nonorth=mask)
        worst = max(worst, nrel(dm.from_cells(host(g[0])), U), nrel(dm.from_cells(host(g[1])), p),
                    nrel(dm.from_faces(host(g[2])), phi))
    assert worst < 1e-9, worst


@pytest.mark.parametrize("split", [(D.NONORTH_MINIMUM, O.NONORTH_MINIMUM),
                                   (D.NONORTH_ORTHOGONAL, O.NONORTH_ORTHOGONAL)], ids=["minimum", "orthogonal"])
def test_piso_lid_cavity_f64_other_splits(split):
    # the PISO step on a mesh created with another split of Eq. nonortho_flux
    m, Ub = _cavity()
    om, dm = O.OMesh.from_mesh(m, split[1]), D.Mesh(m, nonorth=split[0])
    pref = 17
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    pg = _piso(dm, D.F64, 0.01, 0.05, pref=pref, nonorth=3)
    worst = 0.0
    for _ in range(3):
        g = _state_to_gpu(dm, U, p, phi, Ub, pb)
        assert pg.step(*g)[0] == D.OK
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.05, tolU=1e-12,
                                          tolp=1e-12, pref_cell=pref, nonorth=3)
        worst = max(worst, nrel(dm.from_cells(host(g[0])), U), nrel(dm.from_cells(host(g[1])), p),
                    nrel(dm.from_faces(host(g[2])), phi))
    assert worst < 1e-9, worst


@pytest.mark.parametrize("mask,conv,time", [(0, O.CONV_SOU, O.TIME_BE), (3, O.CONV_SOU, O.TIME_BE),
                                            (3, O.CONV_UPWIND, O.TIME_CN), (1, O.CONV_SOU, O.TIME_CN)],
                         ids=["sou", "sou-nonorth", "cn", "sou-cn"])
def test_piso_sou_and_crank_nicolson_f64(mask, conv, time):
    # second-order upwind convection by deferred correction and the Crank-Nicolson
    # momentum rows, against the oracle per step: a lid cavity (all walls) and an
    # inlet/outlet Kuhn box
    for kind in ("cavity", "channel"):
        if kind == "cavity":
            m, Ub = _cavity()
            pref = 17
        else:
            m = mg.shuffle(mg.kuhn_cube(6, 0.2, 4, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET)), 5)
            Ub = np.zeros((3, m.n_boundary))
            Ub[0, m.patch_faces("x0") - m.n_internal] = 1.0
            pref = 0
        om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
        U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
        phi = O.flux_from_U(om, U, Ub)
        o = D.piso_opts(0.01, 0.05, 2, mask, conv=conv, time_scheme=time,
                        solve_U=D.solve_opts(D.BICGSTAB, 1e-12, max_iter=2000),
                        solve_p=D.solve_opts(D.PCG, 1e-12, max_iter=20000),
                        pref_cell=int(dm.cell_new_of_old[pref]))
        pg = D.Piso(dm, D.F64, o)
        worst = 0.0
        for _ in range(4):
            g = _state_to_gpu(dm, U, p, phi, Ub, pb)
            assert pg.step(*g)[0] == D.OK
            U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.05, tolU=1e-12,
                                              tolp=1e-12, pref_cell=pref, nonorth=mask, conv=conv, time=time)
            worst = max(worst, nrel(dm.from_cells(host(g[0])), U), nrel(dm.from_cells(host(g[1])), p),
                        nrel(dm.from_faces(host(g[2])), phi))
        assert worst < 1e-9, (kind, worst)
        # the scheme matters: the upwind backward-Euler step from the same state differs
        Uu = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.05, tolU=1e-12, tolp=1e-12, pref_cell=pref,
                         nonorth=mask)[0]
        Us = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.05, tolU=1e-12, tolp=1e-12, pref_cell=pref,
                         nonorth=mask, conv=conv, time=time)[0]
        assert nrel(Us, Uu) > 1e-4


def test_piso_free_stream_on_gpu():
    m = mg.kuhn_cube(5, 0.2, 5, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET))
    dm = D.Mesh(m)
    U0 = np.array([1.0, 0.0, 0.0])
    Ub = np.broadcast_to(U0[:, None], (3, m.n_boundary)).copy()
    U = np.broadcast_to(U0[:, None], (3, m.n_cells)).copy()
    g = list(_state_to_gpu(dm, U, np.zeros(m.n_cells), np.zeros(m.n_faces), Ub, np.zeros(m.n_boundary)))
    D.difvm_flux_from_U(dm, g[0], g[3], g[2])
    pg = _piso(dm, D.F64, 0.01, 0.01)
    for _ in range(3):
        assert pg.step(*g)[0] == D.OK
    assert float((g[0][0] - 1).abs().max()) < 1e-12 and float(g[0][1:].abs().max()) < 1e-12
    assert float(g[1].abs().max()) < 1e-12


def test_piso_windkessel_channel_f64():
    m = mg.channel_2d(32, 8, seed=5)
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    out = m.patch_index("outlet")
    Ub, pb = _channel_bc(m), np.zeros(m.n_boundary)
    U, p = np.zeros((3, m.n_cells)), np.zeros(m.n_cells)
    phi = O.flux_from_U(om, U, Ub)
    Rp, Cw, Rd = 0.1, 1.0, 2.0
    pc = np.array([0.3])
    wk = cuda(np.array([Rp, Cw, Rd, pc[0]]))
    pg = _piso(dm, D.F64, 0.05, 0.02, wk_patch=[out])
    g = _state_to_gpu(dm, U, p, phi, Ub, pb)
    for _ in range(6):
        st, info = pg.step(*g, wk=wk)
        assert st == D.OK
        U, p, phi, pb, pc, oi = O.piso_step(om, U, p, phi, Ub, pb, nu=0.05, dt=0.02, tolU=1e-12, tolp=1e-12,
                                            wk_patch=[out], Rp=[Rp], Cw=[Cw], Rd=[Rd], pc=pc)
    gi = D.decode_piso_info(info)
    assert abs(gi["Q"][0] - oi["Q"][0]) < 1e-9 * abs(oi["Q"][0])
    assert abs(float(wk[3]) - pc[0]) < 1e-9 * abs(pc[0])
    assert nrel(dm.from_bnd(host(g[4])), pb) < 1e-9
    assert nrel(dm.from_cells(host(g[1])), p) < 1e-8


def test_piso_f32_refine_within_1e4_of_f64_oracle():
    m, Ub = _cavity(6, 21)
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    pref = 3
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    g = _state_to_gpu(dm, U, p, phi, Ub, pb, torch.float32)
    pg = _piso(dm, D.F32, 0.01, 0.02, pref=pref, tol=1e-10, refine=20)
    pg.opts.solve_U.tol_rel = 1e-6
    pg = D.Piso(dm, D.F32, pg.opts)
    for _ in range(5):
        st, info = pg.step(*g)
        assert st == D.OK, D.decode_piso_info(info)
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.02, tolU=1e-12, tolp=1e-12,
                                          pref_cell=pref)
    assert nrel(dm.from_cells(host(g[0])), U) < 1e-4
    assert nrel(dm.from_cells(host(g[1])), p) < 1e-4
    assert nrel(dm.from_faces(host(g[2])), phi) < 1e-4


def test_phase_profile_splits_host_loop_steps():
    # events at the phase boundaries of difvm_piso_step: one record per host-loop
    # step, none for graph-launched steps; the phases cover the step
    m, Ub = _cavity()
    dm = D.Mesh(m)
    pg = _piso(dm, D.F64, 0.01, 0.05, pref=17)
    om = O.OMesh.from_mesh(m)
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    g = _state_to_gpu(dm, U, p, O.flux_from_U(om, U, Ub), Ub, pb)
    torch.cuda.synchronize()
    D.difvm_phase_prof_start(1000)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(3):
        assert pg.step(*g)[0] == D.OK
    b.record()
    pg.step_graph(*g)
    torch.cuda.synchronize()
    ms, n = D.difvm_phase_prof_stop()
    assert n == 3
    assert set(ms) == set(D.PHASES)
    assert ms["momentum_solve"] > 0 and ms["pressure_solve"] > 0 and ms["pressure_assembly"] > 0
    assert sum(ms.values()) <= a.elapsed_time(b) * 1.01
    with pytest.raises(D.DifvmError):
        D.difvm_phase_prof_stop()
