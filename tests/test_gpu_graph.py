"""The PISO step as one CUDA graph (difvm_piso_step_graph): every Krylov solve
runs as a device-side WHILE loop, with no host synchronisation.  Results must
equal the plain step's bit for bit, and the step record must agree."""
import numpy as np
import pytest

from paper_2603_15920_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_15920_b300 import difvm as D  # noqa: E402


def cuda(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda").contiguous()


def _state(dm, m, Ub, dt):
    U = torch.zeros((3, dm.nc), dtype=dt, device="cuda")
    p = torch.zeros(dm.nc, dtype=dt, device="cuda")
    ub = cuda(dm.to_bnd(Ub), dt)
    pb = torch.zeros(dm.nb, dtype=dt, device="cuda")
    phi = D.difvm_flux_from_U(dm, U, ub)
    return [U, p, phi, ub, pb]


def _opts(prec, refine=0, wk_patch=(), pref=0):
    tol_u = 1e-12 if prec == D.F64 else 1e-6
    return D.piso_opts(0.01, 0.02, 2, 3,
                       solve_U=D.solve_opts(D.BICGSTAB, tol_u, max_iter=1000, check_every=4),
                       solve_p=D.solve_opts(D.PCG, 1e-10, max_iter=20000, check_every=16,
                                            refine_max=refine),
                       pref_cell=pref, wk_patch=wk_patch, nonorth_limit=0.5)


def _compare(dm, m, Ub, prec, opts, nsteps=3, wk=None):
    dt = torch.float64 if prec == D.F64 else torch.float32
    a, b = _state(dm, m, Ub, dt), _state(dm, m, Ub, dt)
    wa = None if wk is None else wk.clone()
    wb = None if wk is None else wk.clone()
    ha, hb = D.Piso(dm, prec, opts), D.Piso(dm, prec, opts)
    info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")
    for _ in range(nsteps):
        st, ia = ha.step(*a, wk=wa)
        assert st == D.OK
        hb.step_graph(*b, wk=wb, info=info)
        ra, rb = D.decode_piso_info(ia), D.decode_piso_info(info)
        assert rb["status"] == D.OK
        assert ra["itU"] == rb["itU"] and ra["itp"] == rb["itp"]
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    if wk is not None:
        assert torch.equal(wa, wb)


def _cavity(n, seed):
    m = mg.shuffle(mg.kuhn_cube(n, 0.2, seed), seed + 1)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    return m, Ub


def test_graph_step_equals_plain_step_f64():
    m, Ub = _cavity(8, 2)
    dm = D.Mesh(m)
    _compare(dm, m, Ub, D.F64, _opts(D.F64))


def test_graph_step_equals_plain_step_f32_refined():
    m, Ub = _cavity(8, 3)
    dm = D.Mesh(m)
    _compare(dm, m, Ub, D.F32, _opts(D.F32, refine=20))


def test_graph_step_with_windkessel_outlet():
    m = mg.channel_2d(32, 8, seed=5)
    dm = D.Mesh(m)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("inlet") - m.n_internal] = 1.0
    wk = torch.tensor([0.1, 1.0, 2.0, 0.3], dtype=torch.float64, device="cuda")
    _compare(dm, m, Ub, D.F64, _opts(D.F64, wk_patch=[m.patch_index("outlet")]), wk=wk)


def test_graph_step_batched_mesh():
    ms = [_cavity(n, 10 + n)[0] for n in (3, 6, 8)]
    u, cs = mg.batch(ms)
    Ub = np.zeros((3, u.n_boundary))
    for k in range(3):
        Ub[0, u.patch_faces(f"c{k}/y1") - u.n_internal] = 0.5 + 0.5 * k
    dm = D.Mesh(u, case_cell_start=cs)
    _compare(dm, u, Ub, D.F32, _opts(D.F32))


def test_graph_is_reused_for_the_same_arguments():
    m, Ub = _cavity(5, 4)
    dm = D.Mesh(m)
    h = D.Piso(dm, D.F64, _opts(D.F64))
    s = _state(dm, m, Ub, torch.float64)
    info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")
    h.step_graph(*s, info=info)
    n0 = D.launch_count()
    for _ in range(3):
        h.step_graph(*s, info=info)
    torch.cuda.synchronize()
    assert D.launch_count() == n0          # replays: no kernel launched from the host
    assert D.decode_piso_info(info)["status"] == D.OK
