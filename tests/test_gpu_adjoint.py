"""GPU parity of the adjoint of a PISO step (Sec. 2.5, Eqs. vjp, implicit_diff).

difvm_piso_step_bwd is compared element by element with the oracle's adjoint
(itself pinned against central differences of the oracle's forward step) on
the same seeded inputs, in the input numbering.  Bars: FP64 1e-9 relative to
each output's largest entry (both sides solve their adjoint systems to 1e-13);
FP32 with FP64 pressure refinement 2e-3.  A multi-step loss gradient is checked
against central differences of the oracle's forward steps.
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


TOL = 1e-13


def _case(kind, n, seed):
    if kind == "cavity":
        m = mg.shuffle(mg.kuhn_cube(n, 0.2, seed), seed + 7)
    else:
        m = mg.shuffle(mg.kuhn_cube(n, 0.2, seed, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET)),
                       seed + 7)
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    rng = np.random.default_rng(seed)
    U = 0.5 * rng.normal(size=(3, m.n_cells))
    Ub = 0.5 * rng.normal(size=(3, m.n_boundary))
    x = dict(U=U, p=rng.normal(size=m.n_cells), Ub=Ub,
             phi=O.flux_from_U(om, U, Ub) + 0.01 * rng.normal(size=m.n_faces),
             pb=rng.normal(size=m.n_boundary), pc=np.zeros(0))
    kw = dict(nu=0.05, dt=0.02, ncorr=2, pref_cell=5, wk_patch=[], Rp=[], Cw=[], Rd=[])
    if kind.startswith("wk"):
        kw.update(wk_patch=[m.patch_index("x1")], Rp=[0.3], Cw=[0.8], Rd=[1.2],
                  wk_scheme=dict(wk_exact=O.WK_EXACT, wk_fe=O.WK_FE, wk_be=O.WK_BE)[kind])
        x["pc"] = np.array([0.4])
    return m, om, dm, x, kw


def _gpu_piso(dm, prec, kw, mask, psi, refine=0, conv=None, time=None):
    o = D.piso_opts(kw["nu"], kw["dt"], kw["ncorr"], mask, conv=conv, time_scheme=time,
                    solve_U=D.solve_opts(D.BICGSTAB, TOL if prec == D.F64 else 1e-7, max_iter=5000),
                    solve_p=D.solve_opts(D.PCG, TOL if prec == D.F64 else 1e-12, max_iter=20000,
                                         refine_max=refine),
                    pref_cell=int(dm.cell_new_of_old[kw["pref_cell"]]),
                    wk_scheme=kw.get("wk_scheme", D.WK_EXACT), wk_patch=kw["wk_patch"],
                    nonorth_limit=psi)
    return D.Piso(dm, prec, o)


def _gpu_adjoint(dm, pg, x, kw, w, dt=torch.float64):
    """Record one GPU step from x, then run its adjoint with output weights w."""
    g = [cuda(dm.to_cells(x["U"]), dt), cuda(dm.to_cells(x["p"]), dt),
         cuda(dm.to_faces(x["phi"]), dt), cuda(dm.to_bnd(x["Ub"]), dt), cuda(dm.to_bnd(x["pb"]), dt)]
    n_out = len(kw["wk_patch"])
    wk = cuda(np.ravel(np.column_stack([kw["Rp"], kw["Cw"], kw["Rd"], x["pc"]]))) if n_out else None
    tape = pg.new_tape("cuda")
    st, _ = pg.step_record(*g, tape, wk=wk)
    assert st == D.OK
    Ubar, pbar = cuda(dm.to_cells(w["U"]), dt), cuda(dm.to_cells(w["p"]), dt)
    phibar, pbbar = cuda(dm.to_faces(w["phi"]), dt), cuda(dm.to_bnd(w["pb"]), dt)
    wkbar = cuda(np.ravel(np.column_stack([np.zeros((n_out, 3)), w["pc"]]))) if n_out else None
    Ubbar = torch.zeros((3, dm.nb), dtype=dt, device="cuda")
    nubar = torch.zeros(1, dtype=torch.float64, device="cuda")
    st, info = pg.step_bwd(tape, g[3], wk, Ubar, pbar, phibar, pbbar, wkbar, Ubbar, nubar)
    assert st == D.OK, D.decode_piso_info(info)
    out = dict(U=dm.from_cells(host(Ubar)), p=dm.from_cells(host(pbar)),
               phi=dm.from_faces(host(phibar)), pb=dm.from_bnd(host(pbbar)),
               Ub=dm.from_bnd(host(Ubbar)), nu=float(nubar[0]))
    if n_out:
        wb = host(wkbar).reshape(n_out, 4)
        out.update(Rp=wb[:, 0], Cw=wb[:, 1], Rd=wb[:, 2], pc=wb[:, 3])
    return out, g, tape


def _weights(m, x, seed):
    rng = np.random.default_rng(seed)
    return dict(U=rng.normal(size=(3, m.n_cells)), p=rng.normal(size=m.n_cells),
                phi=rng.normal(size=m.n_faces), pb=rng.normal(size=m.n_boundary),
                pc=rng.normal(size=len(x["pc"])))


UP, SOU = O.CONV_UPWIND, O.CONV_SOU
BE, CN = O.TIME_BE, O.TIME_CN
CASES = [  # (outlet kind, mesh n, non-orthogonal mask, limiter psi, correctors, convection, time)
    ("wk_exact", 6, 3, 1.0, 2, UP, BE),
    ("wk_exact", 6, 3, 0.5, 2, UP, BE),
    ("wk_fe", 5, 1, 0.3, 2, UP, BE),
    ("wk_be", 5, 0, 1.0, 1, UP, BE),
    ("outlet", 6, 3, 0.5, 3, UP, BE),
    ("cavity", 6, 3, 0.5, 2, UP, BE),
    ("cavity", 7, 2, 1.0, 3, UP, BE),
    ("outlet", 6, 0, 1.0, 2, SOU, BE),
    ("cavity", 6, 3, 0.5, 2, SOU, BE),
    ("wk_exact", 5, 1, 1.0, 2, SOU, BE),
    ("outlet", 6, 3, 1.0, 2, UP, CN),
    ("cavity", 6, 1, 0.5, 2, SOU, CN),
]


@pytest.mark.parametrize("kind,n,mask,psi,ncorr,conv,time", CASES)
def test_piso_step_bwd_matches_oracle_f64(kind, n, mask, psi, ncorr, conv, time):
    m, om, dm, x, kw = _case(kind, n, seed=n + mask)
    kw["ncorr"] = ncorr
    w = _weights(m, x, 3)
    pg = _gpu_piso(dm, D.F64, kw, mask, psi, conv=conv, time=time)
    got, _, _ = _gpu_adjoint(dm, pg, x, kw, w)
    ref = O.piso_step_bwd(om, x["U"], x["p"], x["phi"], x["Ub"], x["pb"], w["U"], w["p"], w["phi"],
                          w["pb"], w["pc"], pc=x["pc"], nonorth=mask, psi=psi, tolU=TOL, tolp=TOL,
                          maxitU=5000, maxitp=20000, conv=conv, time=time, **kw)
    assert ref["status"] == 0
    for key in ("U", "p", "phi", "pb", "Ub"):
        assert nrel(got[key], ref[key]) < 1e-9, (key, nrel(got[key], ref[key]))
    assert abs(got["nu"] - ref["nu"]) < 1e-9 * abs(ref["nu"])
    if kw["wk_patch"]:
        for key in ("pc", "Rp", "Cw", "Rd"):
            assert nrel(got[key], ref[key]) < 1e-9, (key, got[key], ref[key])


def test_record_step_equals_plain_step_bitwise():
    m, om, dm, x, kw = _case("wk_exact", 6, 2)
    pg = _gpu_piso(dm, D.F64, kw, 3, 0.5)
    outs = []
    for record in (False, True):
        g = [cuda(dm.to_cells(x["U"])), cuda(dm.to_cells(x["p"])), cuda(dm.to_faces(x["phi"])),
             cuda(dm.to_bnd(x["Ub"])), cuda(dm.to_bnd(x["pb"]))]
        wk = cuda(np.array([0.3, 0.8, 1.2, 0.4]))
        if record:
            st, _ = pg.step_record(*g, pg.new_tape("cuda"), wk=wk)
        else:
            st, _ = pg.step(*g, wk=wk)
        assert st == D.OK
        outs.append([host(t) for t in g] + [host(wk)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_piso_step_bwd_is_deterministic():
    m, om, dm, x, kw = _case("wk_exact", 6, 4)
    w = _weights(m, x, 5)
    pg = _gpu_piso(dm, D.F64, kw, 3, 0.5)
    a, _, _ = _gpu_adjoint(dm, pg, x, kw, w)
    warm, _, _ = _gpu_adjoint(dm, pg, x, kw, w)     # adjoint solves start from a's solutions
    pg.adjoint_reset()
    b, _, _ = _gpu_adjoint(dm, pg, x, kw, w)
    for key in a:
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key
        assert nrel(warm[key], a[key]) < 1e-10, key


def test_piso_step_bwd_f32_refine_close_to_oracle():
    m, om, dm, x, kw = _case("wk_exact", 6, 6)
    w = _weights(m, x, 7)
    pg = _gpu_piso(dm, D.F32, kw, 1, 1.0, refine=20)
    got, _, _ = _gpu_adjoint(dm, pg, x, kw, w, dt=torch.float32)
    ref = O.piso_step_bwd(om, x["U"], x["p"], x["phi"], x["Ub"], x["pb"], w["U"], w["p"], w["phi"],
                          w["pb"], w["pc"], pc=x["pc"], nonorth=1, psi=1.0, tolU=TOL, tolp=TOL,
                          maxitU=5000, maxitp=20000, **kw)
    for key in ("U", "p", "phi", "pb", "Ub", "pc", "Rp", "Cw", "Rd"):
        assert nrel(got[key], ref[key]) < 1e-4, (key, nrel(got[key], ref[key]))
    assert abs(got["nu"] - ref["nu"]) < 1e-4 * abs(ref["nu"]), (got["nu"], ref["nu"])


def test_tape_too_small_is_rejected():
    m, om, dm, x, kw = _case("cavity", 4, 1)
    pg = _gpu_piso(dm, D.F64, kw, 3, 1.0)
    g = [cuda(dm.to_cells(x["U"])), cuda(dm.to_cells(x["p"])), cuda(dm.to_faces(x["phi"])),
         cuda(dm.to_bnd(x["Ub"])), cuda(dm.to_bnd(x["pb"]))]
    short = torch.empty(pg.tape_bytes() - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(D.DifvmError):
        pg.step_record(*g, short)


def test_multi_step_lid_gradient_matches_oracle_differences():
    """Loss = kinetic energy after 3 steps of a lid cavity from rest; dL/d(lid
    speed) and dL/d(nu) from the recorded steps' adjoints against central
    differences of the oracle's forward steps."""
    m = mg.shuffle(mg.kuhn_cube(4, 0.2, 9), 10)
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    lid = np.zeros((3, m.n_boundary))
    lid[0, m.patch_faces("y1") - m.n_internal] = 1.0
    nu, dt, nsteps, pref = 0.02, 0.05, 3, 3
    kw = dict(nu=nu, dt=dt, ncorr=2, pref_cell=pref, wk_patch=[], Rp=[], Cw=[], Rd=[])

    def oracle_loss(ulid, nu_):
        U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
        Ub = ulid * lid
        phi = O.flux_from_U(om, U, Ub)
        for _ in range(nsteps):
            U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=nu_, dt=dt, tolU=1e-15,
                                              tolp=1e-15, maxitU=5000, maxitp=20000,
                                              pref_cell=pref)
        return 0.5 * float(np.sum(m.V * (U ** 2).sum(0)))

    pg = _gpu_piso(dm, D.F64, kw, 3, 1.0)
    Ub = cuda(dm.to_bnd(lid))
    U = torch.zeros((3, dm.nc), dtype=torch.float64, device="cuda")
    p = torch.zeros(dm.nc, dtype=torch.float64, device="cuda")
    pb = torch.zeros(dm.nb, dtype=torch.float64, device="cuda")
    phi = D.difvm_flux_from_U(dm, U, Ub)
    tapes = [pg.new_tape("cuda") for _ in range(nsteps)]
    for k in range(nsteps):
        assert pg.step_record(U, p, phi, Ub, pb, tapes[k])[0] == D.OK
    V = cuda(dm.to_cells(m.V))
    Ubar = (V * U).contiguous()                       # dL/dU
    pbar = torch.zeros_like(p)
    phibar = torch.zeros_like(phi)
    Ubbar = torch.zeros_like(Ub)
    nubar = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in reversed(range(nsteps)):
        assert pg.step_bwd(tapes[k], Ub, None, Ubar, pbar, phibar, None, None, Ubbar, nubar)[0] == D.OK
    # the initial flux is phi = flux_from_U(0, U_b): its adjoint reaches U_b through
    # the boundary faces, phi_f = U_b . S_f on fixed-velocity faces
    phib_bnd = dm.from_faces(host(phibar))[m.n_internal:]
    ub_from_phi = phib_bnd[None, :] * m.Sf[m.n_internal:].T
    dL_dlid = float(np.sum((dm.from_bnd(host(Ubbar)) + ub_from_phi) * lid))
    h = 1e-5
    fd_lid = (oracle_loss(1 + h, nu) - oracle_loss(1 - h, nu)) / (2 * h)
    fd_nu = (oracle_loss(1.0, nu + h * nu) - oracle_loss(1.0, nu - h * nu)) / (2 * h * nu)
    assert abs(dL_dlid - fd_lid) < 1e-6 * abs(fd_lid), (dL_dlid, fd_lid)
    assert abs(float(nubar[0]) - fd_nu) < 1e-6 * abs(fd_nu), (float(nubar[0]), fd_nu)


def test_checkpointed_trajectory_adjoint_equals_fully_taped():
    """simulate_adjoint with the state kept every 2 steps (segments re-run with
    tapes), or with the binomial schedule (one tape, 0 or 2 extra states), gives
    bitwise the same adjoint as recording all 5 steps."""
    m, om, dm, x, kw = _case("wk_exact", 5, 12)
    pg = _gpu_piso(dm, D.F64, kw, 3, 0.5)
    V = cuda(dm.to_cells(m.V))

    def loss_grad(U, p, phi, pb, wk):
        return (V * U).contiguous(), torch.zeros_like(p), torch.zeros_like(phi), None, \
            torch.ones(1, dtype=torch.float64, device="cuda")

    res, finals = [], []
    for ck in (dict(), dict(checkpoint_every=2), dict(checkpoints=0), dict(checkpoints=2)):
        g = [cuda(dm.to_cells(x["U"])), cuda(dm.to_cells(x["p"])), cuda(dm.to_faces(x["phi"])),
             cuda(dm.to_bnd(x["Ub"])), cuda(dm.to_bnd(x["pb"]))]
        wk = cuda(np.array([0.3, 0.8, 1.2, 0.4]))
        r = D.simulate_adjoint(pg, g, 5, loss_grad, wk=wk, **ck)
        assert r["status"] == D.OK
        res.append(r)
        finals.append([t.clone() for t in g] + [wk.clone()])
    # uniform segments and the binomial schedule (no extra slot, two slots): bitwise equal
    for r, fin in zip(res[1:], finals[1:]):
        for key in ("U", "p", "phi", "p_b", "U_b", "nu", "Rp", "C", "Rd", "pc"):
            assert torch.equal(res[0][key], r[key]), key
        for a, b in zip(finals[0], fin):      # the caller's state ends at the final step
            assert torch.equal(a, b)
