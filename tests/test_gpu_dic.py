"""GPU parity of the incomplete factorisations (DIFVM_PRECOND_DIC, the
preconditioning the paper names, Sec. 2.6.1) against the oracle with the same
elimination order (the library's internal RCM numbering): DIC-preconditioned CG
(FP64 solutions at 1e-9 with the iteration count within one, FP32 to its
tolerance) and DILU-preconditioned BiCGStab on non-symmetric matrices (1 and 3
right-hand sides); PISO steps with the DIC pressure solve and with DILU momentum
plus DIC pressure against the oracle's step (1e-9), their CUDA-graph forms
bitwise equal to the host-driven steps."""
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
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def cuda(x, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda").contiguous()


def host(t):
    return t.double().cpu().numpy()


def _spd(m, seed):
    om = O.OMesh.from_mesh(m)
    w, c, k = O.face_coeffs(om)
    rng = np.random.default_rng(seed)
    a = c[:m.n_internal] * rng.uniform(0.5, 2.0, m.n_internal)
    Dg = np.bincount(m.owner[:m.n_internal], a, m.n_cells) + np.bincount(m.neighbour, a, m.n_cells) + 0.01 * m.V
    return om, Dg, -a


@pytest.mark.parametrize("n", [6, 11])
def test_dic_cg_matches_oracle_in_the_same_order(n):
    m = mg.shuffle(mg.kuhn_cube(n, 0.2, n), n + 1)
    om, Dg, L = _spd(m, 3)
    dm = D.Mesh(m)
    rank = dm.cell_new_of_old.astype(np.int32)            # the library's elimination order
    b = np.random.default_rng(4).standard_normal(m.n_cells)
    ref, ri = O.pcg_dic(om, Dg, L, b, rank, tol_rel=1e-12, maxit=5000)
    assert ri["status"] == 0
    Lk = dm.to_faces(np.concatenate([L, np.zeros(m.n_boundary)]), flux=False)[:m.n_internal]
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-6)):
        # FP32 on a well-conditioned shift (D + V): on the nearly singular matrix the
        # solution is ~1e4 and its FP32 rounding alone leaves a 1e-3 residual
        Dd = Dg if dt == torch.float64 else Dg + m.V
        x = torch.zeros(dm.nc, dtype=dt, device="cuda")
        st, info = D.difvm_krylov_solve(dm, cuda(dm.to_cells(Dd), dt), cuda(Lk, dt), None,
                                        cuda(dm.to_cells(b), dt), x, method=D.PCG, precond=D.PRECOND_DIC,
                                        tol_rel=tol, max_iter=5000)
        assert st == D.OK, info
        got = dm.from_cells(host(x))
        if dt == torch.float32:
            # FP64 residual of the FP32 solve: its 1e-6 stop plus the FP32 rounding of A and b
            r = b - O.ldu_apply(om, Dd, L, None, got[None])[0]
            assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(b)
            ref32, _ = O.pcg_dic(om, Dd, L, b, rank, tol_rel=1e-12, maxit=5000)
            assert nrel(got, ref32) < 1e-4
        else:
            assert nrel(got, ref) < 1e-9, nrel(got, ref)
            assert abs(info[0]["iters"] - ri["iters"]) <= 1, (info[0]["iters"], ri["iters"])
            xj, ij = O.pcg(om, Dg, L, None, b, tol_rel=1e-12, maxit=5000)
            assert info[0]["iters"] < ij["iters"]


def test_piso_step_with_dic_pressure_matches_oracle_and_graph():
    m = mg.shuffle(mg.kuhn_cube(6, 0.2, 8), 9)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    pref = 17
    o = D.piso_opts(0.01, 0.05, 2, 3, solve_U=D.solve_opts(D.BICGSTAB, 1e-12, max_iter=2000),
                    solve_p=D.solve_opts(D.PCG, 1e-12, max_iter=5000, precond=D.PRECOND_DIC),
                    pref_cell=int(dm.cell_new_of_old[pref]))
    pg = D.Piso(dm, D.F64, o)
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    state = lambda: [cuda(dm.to_cells(U)), cuda(dm.to_cells(p)), cuda(dm.to_faces(phi)), cuda(dm.to_bnd(Ub)),
                     cuda(dm.to_bnd(pb))]
    worst = 0.0
    for _ in range(3):
        g, gg = state(), state()
        assert pg.step(*g)[0] == D.OK
        info = pg.step_graph(*gg)
        assert D.decode_piso_info(info)["status"] == D.OK
        for a, b in zip(g, gg):
            assert torch.equal(a, b)
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.05, tolU=1e-12, tolp=1e-12,
                                          pref_cell=pref, nonorth=3)
        worst = max(worst, nrel(dm.from_cells(host(g[0])), U), nrel(dm.from_cells(host(g[1])), p),
                    nrel(dm.from_faces(host(g[2])), phi))
    assert worst < 1e-9, worst


def test_incomplete_factorisations_reject_batched_meshes():
    ms = [mg.kuhn_cube(3, 0.2, 1), mg.kuhn_cube(4, 0.2, 2)]
    u, cs = mg.batch(ms)
    with pytest.raises(D.DifvmError):
        D.Piso(D.Mesh(u, case_cell_start=cs), D.F64,
               D.piso_opts(0.01, 0.05, 2, 3, solve_p=D.solve_opts(D.PCG, 1e-10, precond=D.PRECOND_DIC)))
    with pytest.raises(D.DifvmError):
        D.Piso(D.Mesh(u, case_cell_start=cs), D.F64,
               D.piso_opts(0.01, 0.05, 2, 3, solve_U=D.solve_opts(D.BICGSTAB, 1e-10, precond=D.PRECOND_DIC)))


def _nonsym(m, seed):
    """A diagonally dominant convection-diffusion-like LDU matrix (input numbering)."""
    om = O.OMesh.from_mesh(m)
    w, c, k = O.face_coeffs(om)
    rng = np.random.default_rng(seed)
    ni = m.n_internal
    a = c[:ni] * rng.uniform(0.5, 2.0, ni)
    mf = rng.normal(size=ni) * a.mean()
    L, U = -a - np.maximum(mf, 0.0), -a + np.minimum(mf, 0.0)
    Dg = np.bincount(m.owner[:ni], -U, m.n_cells) + np.bincount(m.neighbour, -L, m.n_cells) + 0.05 * a.mean()
    return om, Dg, L, U


@pytest.mark.parametrize("nq", [1, 3])
@pytest.mark.parametrize("n", [5, 10])
def test_dilu_bicgstab_matches_oracle_in_the_same_order(n, nq):
    # BiCGStab preconditioned by DILU (DIFVM_PRECOND_DIC on a non-symmetric
    # matrix), eliminated in the library's internal order, against the oracle's
    # DILU BiCGStab in that order: FP64 solutions at 1e-9, iteration counts within one
    m = mg.shuffle(mg.kuhn_cube(n, 0.2, 40 + n), 41 + n)
    om, Dg, L, U = _nonsym(m, 5)
    dm = D.Mesh(m)
    rank = dm.cell_new_of_old.astype(np.int32)
    ni = m.n_internal
    fo, flip = dm.face_old_of_new[:ni], dm.face_flip[:ni] != 0
    Li, Ui = np.where(flip, U[fo], L[fo]), np.where(flip, L[fo], U[fo])
    B = np.random.default_rng(6).standard_normal((nq, m.n_cells))
    x = torch.zeros(nq, dm.nc, dtype=torch.float64, device="cuda")
    st, info = D.difvm_krylov_solve(dm, cuda(dm.to_cells(Dg)), cuda(Li), cuda(Ui), cuda(dm.to_cells(B)), x,
                                    method=D.BICGSTAB, precond=D.PRECOND_DIC, tol_rel=1e-12, max_iter=2000)
    assert st == D.OK, info
    got = dm.from_cells(host(x))
    for c in range(nq):
        ref, ri = O.bicgstab_dilu(om, Dg, L, U, B[c], rank, tol_rel=1e-12, maxit=2000)
        assert ri["status"] == 0
        assert nrel(got[c], ref) < 1e-9, (c, nrel(got[c], ref))
        assert abs(info[c]["iters"] - ri["iters"]) <= 1, (c, info[c]["iters"], ri["iters"])
        _, rj = O.bicgstab(om, Dg, L, U, B[c], tol_rel=1e-12, maxit=2000)
        assert ri["iters"] < rj["iters"]


def test_piso_step_with_dilu_momentum_matches_oracle_and_graph():
    # the paper's preconditioning of both solves: DILU for the momentum BiCGStab,
    # DIC for the pressure CG; the solutions are the oracle step's to solver tolerance
    m = mg.shuffle(mg.kuhn_cube(6, 0.2, 18), 19)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    pref = 7
    o = D.piso_opts(0.01, 0.05, 2, 3,
                    solve_U=D.solve_opts(D.BICGSTAB, 1e-12, max_iter=2000, precond=D.PRECOND_DIC),
                    solve_p=D.solve_opts(D.PCG, 1e-12, max_iter=5000, precond=D.PRECOND_DIC),
                    pref_cell=int(dm.cell_new_of_old[pref]))
    pg = D.Piso(dm, D.F64, o)
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    state = lambda: [cuda(dm.to_cells(U)), cuda(dm.to_cells(p)), cuda(dm.to_faces(phi)), cuda(dm.to_bnd(Ub)),
                     cuda(dm.to_bnd(pb))]
    worst = 0.0
    for _ in range(3):
        g, gg = state(), state()
        assert pg.step(*g)[0] == D.OK
        assert D.decode_piso_info(pg.step_graph(*gg))["status"] == D.OK
        for a, b in zip(g, gg):
            assert torch.equal(a, b)
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.05, tolU=1e-12, tolp=1e-12,
                                          pref_cell=pref, nonorth=3)
        worst = max(worst, nrel(dm.from_cells(host(g[0])), U), nrel(dm.from_cells(host(g[1])), p),
                    nrel(dm.from_faces(host(g[2])), phi))
    assert worst < 1e-9, worst


def test_piso_adjoint_with_incomplete_factorisations_matches_oracle():
    # the step's adjoint solves use the same preconditioners on the transposed
    # matrices (DILU of A^T for the momentum, DIC for the pressure)
    m = mg.shuffle(mg.kuhn_cube(5, 0.2, 28), 29)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    pref = 3
    o = D.piso_opts(0.01, 0.05, 2, 3,
                    solve_U=D.solve_opts(D.BICGSTAB, 1e-13, max_iter=2000, precond=D.PRECOND_DIC),
                    solve_p=D.solve_opts(D.PCG, 1e-13, max_iter=5000, precond=D.PRECOND_DIC),
                    pref_cell=int(dm.cell_new_of_old[pref]))
    pg = D.Piso(dm, D.F64, o)
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    g = [cuda(dm.to_cells(U)), cuda(dm.to_cells(p)), cuda(dm.to_faces(phi)), cuda(dm.to_bnd(Ub)),
         cuda(dm.to_bnd(pb))]
    tape = pg.new_tape("cuda")
    assert pg.step_record(*g, tape)[0] == D.OK
    U1, _, _, _, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=0.01, dt=0.05, tolU=1e-13, tolp=1e-13,
                                    pref_cell=pref, nonorth=3)
    wU = m.V * U1
    Ubar, pbar, phibar = cuda(dm.to_cells(wU)), cuda(np.zeros(dm.nc)), cuda(np.zeros(dm.nf))
    Ubbar = torch.zeros_like(g[3])
    nubar = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, _ = pg.step_bwd(tape, g[3], None, Ubar, pbar, phibar, None, None, Ubbar, nubar)
    assert st == D.OK
    ref = O.piso_step_bwd(om, U, p, phi, Ub, pb, wU, np.zeros(m.n_cells), np.zeros(m.n_faces), nu=0.01,
                          dt=0.05, tolU=1e-13, tolp=1e-13, pref_cell=pref, nonorth=3)
    for got, r in ((dm.from_cells(host(Ubar)), ref["U"]), (dm.from_faces(host(phibar)), ref["phi"]),
                   (dm.from_bnd(host(Ubbar)), ref["Ub"])):
        assert nrel(got, r) < 1e-9, nrel(got, r)
    assert abs(float(nubar[0]) - ref["nu"]) < 1e-9 * abs(ref["nu"])
