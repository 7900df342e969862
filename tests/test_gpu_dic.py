"""GPU parity of the incomplete-Cholesky-preconditioned CG (DIFVM_PRECOND_DIC, the
preconditioner the paper names, Sec. 2.6.1) against the oracle's DIC CG with the
same elimination order (the library's internal RCM numbering): FP64 solutions at
1e-9 with the iteration count within one, FP32 to its tolerance; a PISO step with
the DIC pressure solve against the oracle's step (1e-9), and its CUDA-graph form
bitwise equal to the host-driven step."""
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


def test_dic_rejects_batched_meshes_and_momentum():
    ms = [mg.kuhn_cube(3, 0.2, 1), mg.kuhn_cube(4, 0.2, 2)]
    u, cs = mg.batch(ms)
    with pytest.raises(D.DifvmError):
        D.Piso(D.Mesh(u, case_cell_start=cs), D.F64,
               D.piso_opts(0.01, 0.05, 2, 3, solve_p=D.solve_opts(D.PCG, 1e-10, precond=D.PRECOND_DIC)))
    with pytest.raises(D.DifvmError):
        D.Piso(D.Mesh(ms[0]), D.F64,
               D.piso_opts(0.01, 0.05, 2, 3, solve_U=D.solve_opts(D.BICGSTAB, 1e-10, precond=D.PRECOND_DIC)))
