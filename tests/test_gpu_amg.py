"""Multigrid-preconditioned CG (DIFVM_PRECOND_AMG) against the oracle.

The preconditioner changes the iteration count, not the solution: every solve
is checked against the FP64 oracle's Jacobi-CG solution and by its true
residual; PISO steps and their adjoints with the multigrid pressure solve are
checked against the oracle at the same bars as the Jacobi path.
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


def _pressure_matrix(m, seed, pin=None):
    """Weighted graph Laplacian of the pressure equation: a_f = rAU_f c_f,
    D = sum a_f (+ a small shift, or a doubled pinned cell)."""
    om = O.OMesh.from_mesh(m)
    w, c, k = O.face_coeffs(om)
    rng = np.random.default_rng(seed)
    rau = m.V / (m.V / 0.002 + 0.05 * rng.uniform(0.5, 1.5, m.n_cells))
    ni = m.n_internal
    a = (w * rau[m.owner[:ni]] + (1 - w) * rau[m.neighbour]) * c[:ni]
    Dg = np.bincount(m.owner[:ni], a, m.n_cells) + np.bincount(m.neighbour, a, m.n_cells)
    if pin is None:
        Dg = Dg + 1e-3 * Dg.mean()
    else:
        Dg[pin] *= 2.0
    return om, Dg, -a


def _solve(dm, m, Dg, Lg, b, precond, prec=D.F64, refine=0, tol=1e-12):
    dt = torch.float64 if (prec == D.F64 or refine) else torch.float32
    Lk = dm.to_faces(np.concatenate([Lg, np.zeros(m.n_boundary)]), flux=False)[:m.n_internal]
    mdt = torch.float64 if prec == D.F64 else torch.float32
    x = torch.zeros(dm.nc, dtype=dt, device="cuda")
    if refine:
        st, info = D.difvm_krylov_solve_refine(dm, cuda(dm.to_cells(Dg), mdt), cuda(Lk, mdt), None,
                                               cuda(dm.to_cells(b)), x, method=D.PCG, tol_rel=tol,
                                               max_iter=2000, precond=precond, refine_max=20,
                                               inner_tol=1e-4)
    else:
        st, info = D.difvm_krylov_solve(dm, cuda(dm.to_cells(Dg), mdt), cuda(Lk, mdt), None,
                                        cuda(dm.to_cells(b), mdt), x, method=D.PCG, tol_rel=tol,
                                        max_iter=20000, precond=precond)
    return st, info[0], dm.from_cells(host(x))


@pytest.mark.parametrize("n,pin", [(10, None), (14, 7), (3, None)])
def test_amg_cg_solves_the_pressure_system(n, pin):
    m = mg.shuffle(mg.kuhn_cube(n, 0.2, n), n + 1)
    dm = D.Mesh(m)
    om, Dg, Lg = _pressure_matrix(m, 1, pin)
    b = np.random.default_rng(2).normal(size=m.n_cells)
    if pin is not None:
        b -= b.mean()
    st, ia, x = _solve(dm, m, Dg, Lg, b, D.PRECOND_AMG)
    assert st == D.OK and ia["status"] == D.OK
    r = b - O.ldu_apply(om, Dg, Lg, None, x[None])[0]
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(b)
    ref, _ = O.pcg(om, Dg, Lg, None, b, tol_rel=1e-13, maxit=100000)
    assert nrel(x, ref) < 1e-7
    st, ij, _ = _solve(dm, m, Dg, Lg, b, D.PRECOND_JACOBI)
    if n >= 10:
        assert ia["iters"] * 5 < ij["iters"], (ia["iters"], ij["iters"])


def test_amg_mixed_precision_reaches_fp64_tolerance():
    m = mg.shuffle(mg.kuhn_cube(12, 0.2, 5), 6)
    dm = D.Mesh(m)
    om, Dg, Lg = _pressure_matrix(m, 3, pin=11)
    b = np.random.default_rng(4).normal(size=m.n_cells)
    b -= b.mean()
    Dg32 = Dg.astype(np.float32).astype(np.float64)   # the FP32 matrix is the matrix solved
    Lg32 = Lg.astype(np.float32).astype(np.float64)
    st, info, x = _solve(dm, m, Dg, Lg, b, D.PRECOND_AMG, prec=D.F32, refine=1, tol=1e-10)
    assert st == D.OK, info
    # one FP64 CG around the FP32 V-cycle: no refinement sweeps, few iterations
    assert info["refinements"] == 0 and info["iters"] < 60
    r = b - O.ldu_apply(om, Dg32, Lg32, None, x[None])[0]
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)


def test_amg_solve_is_deterministic():
    m = mg.shuffle(mg.kuhn_cube(9, 0.2, 8), 9)
    dm = D.Mesh(m)
    om, Dg, Lg = _pressure_matrix(m, 5)
    b = np.random.default_rng(6).normal(size=m.n_cells)
    a = _solve(dm, m, Dg, Lg, b, D.PRECOND_AMG)[2]
    c = _solve(dm, m, Dg, Lg, b, D.PRECOND_AMG)[2]
    assert np.array_equal(a, c)


def _piso(dm, prec, pref, refine=0, tol=1e-12):
    o = D.piso_opts(0.02, 0.05, 2, 3,
                    solve_U=D.solve_opts(D.BICGSTAB, tol if prec == D.F64 else 1e-7, max_iter=2000),
                    solve_p=D.solve_opts(D.PCG, tol, max_iter=2000, refine_max=refine,
                                         precond=D.PRECOND_AMG),
                    pref_cell=int(dm.cell_new_of_old[pref]), nonorth_limit=0.5)
    return D.Piso(dm, prec, o)


def _cavity(n, seed):
    m = mg.shuffle(mg.kuhn_cube(n, 0.2, seed), seed + 1)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    return m, Ub


@pytest.mark.parametrize("prec,refine,bar", [(D.F64, 0, 1e-9), (D.F32, 20, 1e-4)])
def test_piso_with_amg_pressure_matches_oracle(prec, refine, bar):
    m, Ub = _cavity(8, 21)
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    pref = 13
    dt = torch.float64 if prec == D.F64 else torch.float32
    pg = _piso(dm, prec, pref, refine, tol=1e-12 if prec == D.F64 else 1e-10)
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    g = [cuda(dm.to_cells(U), dt), cuda(dm.to_cells(p), dt), cuda(dm.to_faces(phi), dt),
         cuda(dm.to_bnd(Ub), dt), cuda(dm.to_bnd(pb), dt)]
    for _ in range(3):
        st, info = pg.step(*g)
        assert st == D.OK, D.decode_piso_info(info)
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=0.02, dt=0.05, tolU=1e-12,
                                          tolp=1e-12, pref_cell=pref, psi=0.5, nonorth=3)
    errs = nrel(dm.from_cells(host(g[0])), U), nrel(dm.from_cells(host(g[1])), p)
    assert max(errs) < bar, errs
    assert max(D.decode_piso_info(info)["itp"][:2]) < 60


def test_piso_adjoint_with_amg_pressure_matches_oracle():
    m, Ub = _cavity(6, 31)
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    pref = 5
    rng = np.random.default_rng(1)
    U = 0.3 * rng.normal(size=(3, m.n_cells))
    p = rng.normal(size=m.n_cells)
    phi = O.flux_from_U(om, U, Ub)
    pb = np.zeros(m.n_boundary)
    pg = _piso(dm, D.F64, pref, tol=1e-13)
    g = [cuda(dm.to_cells(U)), cuda(dm.to_cells(p)), cuda(dm.to_faces(phi)), cuda(dm.to_bnd(Ub)),
         cuda(dm.to_bnd(pb))]
    tape = pg.new_tape("cuda")
    assert pg.step_record(*g, tape)[0] == D.OK
    wU, wp = rng.normal(size=(3, m.n_cells)), rng.normal(size=m.n_cells)
    Ubar, pbar, phibar = cuda(dm.to_cells(wU)), cuda(dm.to_cells(wp)), cuda(np.zeros(dm.nf))
    Ubbar = torch.zeros_like(g[3])
    nubar = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert pg.step_bwd(tape, g[3], None, Ubar, pbar, phibar, None, None, Ubbar, nubar)[0] == D.OK
    ref = O.piso_step_bwd(om, U, p, phi, Ub, pb, wU, wp, np.zeros(m.n_faces), nu=0.02, dt=0.05,
                          tolU=1e-13, tolp=1e-13, pref_cell=pref, psi=0.5, nonorth=3)
    assert nrel(dm.from_cells(host(Ubar)), ref["U"]) < 1e-9
    assert nrel(dm.from_cells(host(pbar)), ref["p"]) < 1e-9
    assert nrel(dm.from_bnd(host(Ubbar)), ref["Ub"]) < 1e-9
    assert abs(float(nubar[0]) - ref["nu"]) < 1e-9 * abs(ref["nu"])


@pytest.mark.parametrize("prec,refine", [(D.F64, 0), (D.F32, 20)])
def test_graph_step_with_amg_equals_plain(prec, refine):
    m, Ub = _cavity(9, 41)
    dm = D.Mesh(m)
    dt = torch.float64 if prec == D.F64 else torch.float32
    outs = []
    for graph in (False, True):
        pg = _piso(dm, prec, 3, refine, tol=1e-10)
        U = torch.zeros((3, dm.nc), dtype=dt, device="cuda")
        p = torch.zeros(dm.nc, dtype=dt, device="cuda")
        ub = cuda(dm.to_bnd(Ub), dt)
        pb = torch.zeros(dm.nb, dtype=dt, device="cuda")
        phi = D.difvm_flux_from_U(dm, U, ub)
        info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")
        for _ in range(3):
            if graph:
                pg.step_graph(U, p, phi, ub, pb, info=info)
            else:
                assert pg.step(U, p, phi, ub, pb, info=info)[0] == D.OK
        torch.cuda.synchronize()
        assert D.decode_piso_info(info)["status"] == D.OK
        outs.append([host(t) for t in (U, p, phi)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_batched_multigrid_limits():
    """On a batched mesh the multigrid CG is accepted (per-case scalars; parity in
    the batched tests) but its FP64-refinement form and BiCGStab are not."""
    ms = [mg.kuhn_cube(3, 0.2, 1), mg.kuhn_cube(4, 0.2, 2)]
    u, cs = mg.batch(ms)
    dm = D.Mesh(u, case_cell_start=cs)
    D.Piso(dm, D.F64, D.piso_opts(0.02, 0.05, 2, 3,
                                  solve_p=D.solve_opts(D.PCG, 1e-10, precond=D.PRECOND_AMG)))
    for prec, sp in ((D.F32, D.solve_opts(D.PCG, 1e-10, precond=D.PRECOND_AMG, refine_max=20)),
                     (D.F64, D.solve_opts(D.BICGSTAB, 1e-10, precond=D.PRECOND_AMG))):
        with pytest.raises(D.DifvmError):
            D.Piso(dm, prec, D.piso_opts(0.02, 0.05, 2, 3, solve_p=sp))


@pytest.mark.parametrize("prec,refine", [(D.F64, 0), (D.F32, 1)])
def test_fused_coarse_levels_match_per_level_kernels(prec, refine):
    # the levels below the fused-kernel threshold run as phases of one cooperative
    # launch; each phase computes what its per-level kernel computes, in the same order
    m = mg.shuffle(mg.kuhn_cube(16, 0.2, 12), 13)
    dm = D.Mesh(m)
    om, Dg, Lg = _pressure_matrix(m, 7, pin=5)
    b = np.random.default_rng(8).normal(size=m.n_cells)
    b -= b.mean()
    out = {}
    for rows in (0, 100000, 2000):       # per-level kernels; every coarse level fused; only the smallest
        D.difvm_mesh_amg_config(dm, rows, -1)
        st, info, x = _solve(dm, m, Dg, Lg, b, D.PRECOND_AMG, prec=prec, refine=refine,
                             tol=1e-12 if prec == D.F64 else 1e-10)
        assert st == D.OK, info
        out[rows] = (info["iters"], x)
    assert out[0][0] == out[100000][0] == out[2000][0]
    assert np.array_equal(out[0][1], out[100000][1]) and np.array_equal(out[0][1], out[2000][1])
    with pytest.raises(D.DifvmError):
        D.difvm_mesh_amg_config(dm, 100, 0)


def test_fused_coarse_levels_batched_match_per_level_kernels():
    ms = [mg.kuhn_cube(n, 0.2, 30 + n) for n in (5, 9, 7)]
    u, cs = mg.batch(ms)
    dmu = D.Mesh(u, case_cell_start=cs)
    om, Dg, Lg = _pressure_matrix(u, 9)
    b = np.random.default_rng(10).normal(size=u.n_cells)
    xs = []
    for rows in (0, 100000):
        D.difvm_mesh_amg_config(dmu, rows, -1)
        st, info, x = _solve(dmu, u, Dg, Lg, b, D.PRECOND_AMG)
        assert st == D.OK
        xs.append((info["iters"], x))
    assert xs[0][0] == xs[1][0] and np.array_equal(xs[0][1], xs[1][1])


def test_multigrid_launch_shapes_are_tuned_and_solve_the_same_system():
    # the hierarchy's lanes per row and restriction lanes are timed when it is
    # built; the defaults (mode 0) and the tuned shapes solve to the same bar
    m = mg.shuffle(mg.kuhn_cube(14, 0.2, 21), 22)
    dm = D.Mesh(m)
    om, Dg, Lg = _pressure_matrix(m, 11, pin=3)
    b = np.random.default_rng(12).normal(size=m.n_cells)
    b -= b.mean()
    st, info, x = _solve(dm, m, Dg, Lg, b, D.PRECOND_AMG)
    assert st == D.OK
    kept = D.difvm_mesh_tuning(dm)
    lanes = {k: v for k, v in kept.items() if k[0] == 5}
    rlanes = {k: v for k, v in kept.items() if k[0] == 6}
    assert lanes and set(lanes.values()) <= {2, 4, 8} and set(rlanes.values()) <= {1, 8}
    D.difvm_mesh_autotune(dm, 0)
    st0, info0, x0 = _solve(dm, m, Dg, Lg, b, D.PRECOND_AMG)
    assert st0 == D.OK
    ref, _ = O.pcg(om, Dg, Lg, None, b, tol_rel=1e-13, maxit=100000)
    assert nrel(x, ref) < 1e-7 and nrel(x0, ref) < 1e-7
    assert abs(info["iters"] - info0["iters"]) <= 1


@pytest.mark.parametrize("prec,refine", [(D.F64, 0), (D.F32, 20)])
def test_wide_index_layouts_step_bitwise_the_same(prec, refine):
    # the solvers' 16-bit ELL column offsets (used where the RCM bandwidth allows)
    # and the 32-bit columns of DIFVM_WIDE_INDICES address the same entries: the
    # multigrid-CG pressure and BiCGStab momentum solves of a PISO step agree bitwise
    m, Ub = _cavity(10, 51)
    dt = torch.float64 if prec == D.F64 else torch.float32
    outs = []
    for flags in (D.RENUMBER_RCM | D.SORT_FACES, D.RENUMBER_RCM | D.SORT_FACES | D.WIDE_INDICES):
        dm = D.Mesh(m, flags=flags)
        assert D.difvm_mesh_layout(dm) == ((True, True) if not flags & D.WIDE_INDICES else (False, False))
        D.difvm_mesh_autotune(dm, 0)          # the same launch shapes on both
        pg = _piso(dm, prec, 3, refine, tol=1e-10)
        U = torch.zeros((3, dm.nc), dtype=dt, device="cuda")
        p = torch.zeros(dm.nc, dtype=dt, device="cuda")
        ub = cuda(dm.to_bnd(Ub), dt)
        pb = torch.zeros(dm.nb, dtype=dt, device="cuda")
        phi = D.difvm_flux_from_U(dm, U, ub)
        info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")
        for _ in range(3):
            pg.step_graph(U, p, phi, ub, pb, info=info)
        torch.cuda.synchronize()
        assert D.decode_piso_info(info)["status"] == D.OK
        outs.append([dm.from_cells(host(U)), dm.from_cells(host(p))])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
