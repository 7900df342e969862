"""Batched (segmented) solves and PISO steps on a disjoint union of cases.

Each case of a batch keeps its own Krylov scalars, convergence flag and
iteration count.  Checks: every case against the FP64 oracle run on that case
alone (1e-9), and bitwise equality between a case inside a batch and the same
case solved alone (a one-case segmented mesh), for the solvers, the PISO step
and its adjoint.
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


def _cases():
    # sizes 162, 2,058 and 4,374 cells: one, two and three solver blocks (2,048 rows each)
    return [mg.shuffle(mg.kuhn_cube(n, 0.2, 10 + n), n) for n in (3, 7, 9)]


@pytest.fixture(scope="module")
def batch():
    ms = _cases()
    u, cs = mg.batch(ms)
    return ms, u, cs, D.Mesh(u, case_cell_start=cs), [D.Mesh(m, case_cell_start=[0, m.n_cells]) for m in ms]


def test_batched_numbering_keeps_cases_contiguous(batch):
    ms, u, cs, dmu, dms = batch
    for k, dm in enumerate(dms):
        got = dmu.cell_new_of_old[cs[k]:cs[k + 1]] - cs[k]
        assert np.array_equal(got, dm.cell_new_of_old)


def _spd(m, seed, diag_frac=None):
    """Pressure-like SPD LDU matrix of one case: D = sum c_f + shift, L = -c_f
    (shift 0.01 V, or diag_frac * sum c_f: condition number ~2 / diag_frac)."""
    om = O.OMesh.from_mesh(m)
    w, c, k = O.face_coeffs(om)
    rng = np.random.default_rng(seed)
    a = c[:m.n_internal] * rng.uniform(0.5, 2.0, m.n_internal)
    rs = np.bincount(m.owner[:m.n_internal], a, m.n_cells) + np.bincount(m.neighbour, a, m.n_cells)
    Dg = rs + (0.01 * m.V if diag_frac is None else diag_frac * rs)
    return om, Dg, -a


def _to_union_faces(dmu, per_case, u, cs, ms):
    """Input-numbered per-case internal-face arrays -> the union's internal numbering."""
    full = np.concatenate(per_case)
    return dmu.to_faces(np.concatenate([full, np.zeros(u.n_boundary)]), flux=False)[:u.n_internal]


@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
def test_batched_solve_matches_oracle_and_unbatched_bitwise(batch, method):
    ms, u, cs, dmu, dms = batch
    rng = np.random.default_rng(4)
    mats = [_spd(m, k) for k, m in enumerate(ms)]
    ncomp = 1 if method == "pcg" else 3
    meth = D.PCG if method == "pcg" else D.BICGSTAB
    bs = [rng.normal(size=(ncomp, m.n_cells)) for m in ms]
    # the union: cell-wise arrays concatenate in case order (input numbering)
    Du = np.concatenate([mt[1] for mt in mats])
    Lu = _to_union_faces(dmu, [mt[2] for mt in mats], u, cs, ms)
    bu = np.concatenate(bs, axis=1)
    x = torch.zeros((ncomp, dmu.nc), dtype=torch.float64, device="cuda")
    st, iters_u = D.difvm_krylov_solve(dmu, cuda(dmu.to_cells(Du)), cuda(Lu), None,
                                       cuda(dmu.to_cells(bu)), x, method=meth, tol_rel=1e-12,
                                       max_iter=5000)
    assert st == D.OK and len(iters_u) == len(ms) * ncomp
    xu = dmu.from_cells(host(x))
    for k, (m, dm) in enumerate(zip(ms, dms)):
        om, Dg, Lg = mats[k]
        # the oracle, case alone
        for c in range(ncomp):
            solver = O.pcg if method == "pcg" else O.bicgstab
            ref, oi = solver(om, Dg, Lg, None, bs[k][c], tol_rel=1e-12)
            xc = xu[c, cs[k]:cs[k + 1]]
            # each case converged on its own: true residual of that case alone
            r = bs[k][c] - O.ldu_apply(om, Dg, Lg, None, xc[None])[0]
            # (the solvers stop on the recursive residual; the true one may be a few times larger)
            assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(bs[k][c])
            # the solution error is bounded by cond(A) x tolerance (both sides at 1e-12)
            assert nrel(xc, ref) < 1e-8
        # the same case alone on a one-case segmented mesh: bitwise equal
        Lk = dm.to_faces(np.concatenate([Lg, np.zeros(m.n_boundary)]), flux=False)[:m.n_internal]
        xk = torch.zeros((ncomp, dm.nc), dtype=torch.float64, device="cuda")
        st, alone = D.difvm_krylov_solve(dm, cuda(dm.to_cells(Dg)), cuda(Lk), None,
                                         cuda(dm.to_cells(bs[k])), xk, method=meth, tol_rel=1e-12,
                                         max_iter=5000)
        assert st == D.OK
        assert np.array_equal(dm.from_cells(host(xk)), xu[:, cs[k]:cs[k + 1]])
        for c in range(ncomp):
            assert alone[c]["iters"] == iters_u[k * ncomp + c]["iters"]


def _cavity_state(m, lid):
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = lid
    return Ub


def _piso(dm, prec, pref):
    o = D.piso_opts(0.02, 0.05, 2, 3,
                    solve_U=D.solve_opts(D.BICGSTAB, 1e-13, max_iter=2000),
                    solve_p=D.solve_opts(D.PCG, 1e-13, max_iter=20000),
                    pref_cell=pref, nonorth_limit=0.5)
    return D.Piso(dm, prec, o)


def test_batched_piso_step_and_adjoint(batch):
    """Three lid cavities of different sizes and lid speeds in one batch: each
    case against the oracle (pinned at its own first input cell), and the batch
    bitwise against each case stepped alone, forward and adjoint."""
    ms, u, cs, dmu, dms = batch
    lids = [1.0, 0.7, 1.3]
    Ubs = [_cavity_state(m, l) for m, l in zip(ms, lids)]
    # the pinned cell is case-relative in the internal numbering: the same
    # internal cell in the batch and alone
    pref = 0
    hu = _piso(dmu, D.F64, pref)
    st_u = [torch.zeros((3, dmu.nc), dtype=torch.float64, device="cuda"),
            torch.zeros(dmu.nc, dtype=torch.float64, device="cuda"), None,
            cuda(dmu.to_bnd(np.concatenate(Ubs, axis=1))),
            torch.zeros(dmu.nb, dtype=torch.float64, device="cuda")]
    st_u[2] = D.difvm_flux_from_U(dmu, st_u[0], st_u[3])
    tapes_u = []
    for _ in range(2):
        tapes_u.append(hu.new_tape("cuda"))
        s, info = hu.step_record(*st_u, tapes_u[-1])
        assert s == D.OK, D.decode_piso_info(info)
    for k, (m, dm) in enumerate(zip(ms, dms)):
        om = O.OMesh.from_mesh(m)
        pin_old = int(np.where(dm.cell_new_of_old == pref)[0][0])
        U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
        phi = O.flux_from_U(om, U, Ubs[k])
        for _ in range(2):
            U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ubs[k], pb, nu=0.02, dt=0.05, tolU=1e-13,
                                              tolp=1e-13, pref_cell=pin_old, psi=0.5, nonorth=3)
        Uu = dmu.from_cells(host(st_u[0]))[:, cs[k]:cs[k + 1]]
        assert nrel(Uu, U) < 1e-9
        pu = dmu.from_cells(host(st_u[1]))[cs[k]:cs[k + 1]]
        assert nrel(pu, p) < 1e-9
    # alone, bitwise
    alone = []
    for k, (m, dm) in enumerate(zip(ms, dms)):
        h = _piso(dm, D.F64, pref)
        s_ = [torch.zeros((3, dm.nc), dtype=torch.float64, device="cuda"),
              torch.zeros(dm.nc, dtype=torch.float64, device="cuda"), None,
              cuda(dm.to_bnd(Ubs[k])), torch.zeros(dm.nb, dtype=torch.float64, device="cuda")]
        s_[2] = D.difvm_flux_from_U(dm, s_[0], s_[3])
        tapes = []
        for _ in range(2):
            tapes.append(h.new_tape("cuda"))
            assert h.step_record(*s_, tapes[-1])[0] == D.OK
        assert np.array_equal(dm.from_cells(host(s_[0])),
                              dmu.from_cells(host(st_u[0]))[:, cs[k]:cs[k + 1]])
        alone.append((h, dm, s_, tapes))
    # adjoint of the kinetic energy, batch vs alone
    V = cuda(dmu.to_cells(u.V))
    Ubar = (V * st_u[0]).contiguous()
    pbar, phibar = torch.zeros_like(st_u[1]), torch.zeros_like(st_u[2])
    Ubbar = torch.zeros_like(st_u[3])
    nubar = torch.zeros(1, dtype=torch.float64, device="cuda")
    for tp in reversed(tapes_u):
        assert hu.step_bwd(tp, st_u[3], None, Ubar, pbar, phibar, None, None, Ubbar, nubar)[0] == D.OK
    Ubar_u = dmu.from_cells(host(Ubar))
    for k, (h, dm, s_, tapes) in enumerate(alone):
        Vk = cuda(dm.to_cells(ms[k].V))
        ub = (Vk * s_[0]).contiguous()
        pb_, fb = torch.zeros_like(s_[1]), torch.zeros_like(s_[2])
        ubb = torch.zeros_like(s_[3])
        nb_ = torch.zeros(1, dtype=torch.float64, device="cuda")
        for tp in reversed(tapes):
            assert h.step_bwd(tp, s_[3], None, ub, pb_, fb, None, None, ubb, nb_)[0] == D.OK
        assert np.array_equal(dm.from_cells(host(ub)), Ubar_u[:, cs[k]:cs[k + 1]])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_multigrid_cg_matches_oracle(batch, prec):
    """Multigrid-preconditioned CG on the union: each case converges on its own
    (its own CG scalars and stopping test) to the oracle's solution of that case
    alone; a case with b = 0 returns x = 0 after no iteration; the iteration
    counts stay far below Jacobi's."""
    ms, u, cs, dmu, dms = batch
    rng = np.random.default_rng(5)
    # FP32: a matrix of condition ~100, so that the FP32 floor of the true
    # residual (u32 cond(A) ~ 6e-6) sits near the 1e-6 stopping tolerance
    mats = [_spd(m, 20 + k, None if prec == "f64" else 0.02) for k, m in enumerate(ms)]
    bs = [rng.normal(size=m.n_cells) for m in ms]
    bs[1][:] = 0.0                        # the middle case: zero right-hand side
    Du = np.concatenate([mt[1] for mt in mats])
    Lu = _to_union_faces(dmu, [mt[2] for mt in mats], u, cs, ms)
    dt = torch.float64 if prec == "f64" else torch.float32
    tol = 1e-12 if prec == "f64" else 1e-6
    x = torch.full((dmu.nc,), 0.5, dtype=dt, device="cuda")   # nonzero guess
    st, info = D.difvm_krylov_solve(dmu, cuda(dmu.to_cells(Du), dt), cuda(Lu, dt), None,
                                    cuda(dmu.to_cells(np.concatenate(bs)), dt), x,
                                    method=D.PCG, precond=D.PRECOND_AMG, tol_rel=tol, max_iter=500)
    assert st == D.OK and len(info) == len(ms)
    _, jac = D.difvm_krylov_solve(dmu, cuda(dmu.to_cells(Du)), cuda(Lu), None,
                                  cuda(dmu.to_cells(np.concatenate(bs))),
                                  torch.zeros(dmu.nc, dtype=torch.float64, device="cuda"),
                                  method=D.PCG, tol_rel=tol, max_iter=5000)
    xu = dmu.from_cells(host(x))
    for k, m in enumerate(ms):
        om, Dg, Lg = mats[k]
        xc = xu[cs[k]:cs[k + 1]]
        if k == 1:
            assert info[k]["iters"] == 0 and np.all(xc == 0.0)
            continue
        assert info[k]["status"] == D.OK and 0 < info[k]["iters"] <= 40
        assert info[k]["iters"] * 2 < jac[k]["iters"]
        r = bs[k] - O.ldu_apply(om, Dg, Lg, None, xc[None])[0]
        ref, _ = O.pcg(om, Dg, Lg, None, bs[k], tol_rel=1e-13)
        if prec == "f64":
            assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(bs[k])
            assert nrel(xc, ref) < 1e-8
        else:
            # FP32 vectors and matrix: the recursive residual reaches 1e-6, the
            # true one stays within a few times the floor u32 cond(A); the
            # solution error within cond(A) times that
            assert np.linalg.norm(r) <= 5e-5 * np.linalg.norm(bs[k])
            assert nrel(xc, ref) < 5e-3


def test_batched_piso_step_multigrid_pressure(batch):
    """The batched PISO step with the multigrid pressure CG: each case against
    the oracle (which solves its pressure with Jacobi CG to the same tight
    tolerance) at 1e-9, over two steps; then the adjoint of the second step
    (its pressure solves transposed through the same multigrid CG) against the
    oracle's adjoint of that step, case by case."""
    ms, u, cs, dmu, dms = batch
    lids = [1.0, 0.7, 1.3]
    Ubs = [_cavity_state(m, l) for m, l in zip(ms, lids)]
    pref = 0
    o = D.piso_opts(0.02, 0.05, 2, 3,
                    solve_U=D.solve_opts(D.BICGSTAB, 1e-13, max_iter=2000),
                    solve_p=D.solve_opts(D.PCG, 1e-13, max_iter=500, precond=D.PRECOND_AMG),
                    pref_cell=pref, nonorth_limit=0.5)
    hu = D.Piso(dmu, D.F64, o)
    st_u = [torch.zeros((3, dmu.nc), dtype=torch.float64, device="cuda"),
            torch.zeros(dmu.nc, dtype=torch.float64, device="cuda"), None,
            cuda(dmu.to_bnd(np.concatenate(Ubs, axis=1))),
            torch.zeros(dmu.nb, dtype=torch.float64, device="cuda")]
    st_u[2] = D.difvm_flux_from_U(dmu, st_u[0], st_u[3])
    s, info = hu.step(*st_u)
    assert s == D.OK, D.decode_piso_info(info)
    tape = hu.new_tape("cuda")
    s, info = hu.step_record(*st_u, tape)
    assert s == D.OK, D.decode_piso_info(info)
    Ubar = (cuda(dmu.to_cells(u.V)) * st_u[0]).contiguous()     # d(KE)/dU of the step's output
    pbar, phibar = torch.zeros_like(st_u[1]), torch.zeros_like(st_u[2])
    Ubbar = torch.zeros_like(st_u[3])
    nubar = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert hu.step_bwd(tape, st_u[3], None, Ubar, pbar, phibar, None, None, Ubbar, nubar)[0] == D.OK
    Ubar_u = dmu.from_cells(host(Ubar))
    for k, (m, dm) in enumerate(zip(ms, dms)):
        om = O.OMesh.from_mesh(m)
        pin_old = int(np.where(dm.cell_new_of_old == pref)[0][0])
        kw = dict(nu=0.02, dt=0.05, tolU=1e-13, tolp=1e-13, pref_cell=pin_old, psi=0.5, nonorth=3)
        U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
        phi = O.flux_from_U(om, U, Ubs[k])
        U1, p1, phi1, pb1, _, _ = O.piso_step(om, U, p, phi, Ubs[k], pb, **kw)
        U2, p2, _, _, _, _ = O.piso_step(om, U1, p1, phi1, Ubs[k], pb1, **kw)
        assert nrel(dmu.from_cells(host(st_u[0]))[:, cs[k]:cs[k + 1]], U2) < 1e-9
        assert nrel(dmu.from_cells(host(st_u[1]))[cs[k]:cs[k + 1]], p2) < 1e-9
        ref = O.piso_step_bwd(om, U1, p1, phi1, Ubs[k], pb1, m.V * U2, np.zeros(m.n_cells),
                              np.zeros(m.n_faces), **kw)
        assert ref["status"] == 0
        assert nrel(Ubar_u[:, cs[k]:cs[k + 1]], ref["U"]) < 1e-8


def test_refinement_is_rejected_on_batched_meshes(batch):
    ms, u, cs, dmu, dms = batch
    o = D.piso_opts(0.02, 0.05, 2, 3, solve_p=D.solve_opts(D.PCG, 1e-10, refine_max=20))
    with pytest.raises(D.DifvmError):
        D.Piso(dmu, D.F32, o)
