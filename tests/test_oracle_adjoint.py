"""Pins of the oracle's adjoint of one PISO step (Sec. 2.5, Eqs. vjp, implicit_diff).

The adjoint is checked against central differences of the oracle's own forward
step, one input or parameter at a time: for random output weights w and a
random direction v,  <w, (F(x + h v) - F(x - h v)) / 2h>  must equal
<J^T w, v>.  The forward step is pinned elsewhere (free stream, Poiseuille,
continuity, Windkessel closed forms), so this ties the hand-written reverse
sweep to the method itself.  Solver tolerances are set near round-off so the
difference quotient is limited by truncation (h^2) and round-off / h only.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_15920_b300 import meshgen as mg


def _case(kind, seed):
    if kind == "cavity":                    # all walls: pressure pinned at one cell
        m = mg.shuffle(mg.kuhn_cube(3, 0.2, seed), seed + 7)
    else:
        m = mg.shuffle(mg.kuhn_cube(3, 0.2, seed, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET)),
                       seed + 7)
    om = O.OMesh.from_mesh(m)
    rng = np.random.default_rng(seed)
    U = 0.5 * rng.normal(size=(3, m.n_cells))
    Ub = 0.5 * rng.normal(size=(3, m.n_boundary))
    x = dict(U=U, p=rng.normal(size=m.n_cells), Ub=Ub,
             phi=O.flux_from_U(om, U, Ub) + 0.01 * rng.normal(size=m.n_faces),
             pb=rng.normal(size=m.n_boundary), pc=np.zeros(0))
    kw = dict(nu=0.05, dt=0.02, ncorr=2, tolU=1e-15, tolp=1e-15, maxitU=5000, maxitp=5000,
              pref_cell=5)
    if kind.startswith("wk"):
        outlet = [k for k, t in enumerate(m.patch_type) if t == mg.OUTLET]
        kw.update(wk_patch=outlet, Rp=[0.3], Cw=[0.8], Rd=[1.2],
                  wk_scheme=dict(wk_exact=O.WK_EXACT, wk_fe=O.WK_FE, wk_be=O.WK_BE)[kind])
        x["pc"] = np.array([0.4])
    return om, x, kw


def _fwd(om, x, kw):
    U, p, phi, pb, pc, info = O.piso_step(om, x["U"], x["p"], x["phi"], x["Ub"], x["pb"],
                                          pc=x["pc"], **kw)
    return dict(U=U, p=p, phi=phi, pb=pb, pc=pc)


UP, SOU = O.CONV_UPWIND, O.CONV_SOU
BE, CN = O.TIME_BE, O.TIME_CN
CASES = [  # (mesh / outlet kind, non-orthogonal mask, limiter psi, correctors, convection, time)
    ("wk_exact", 3, 1.0, 2, UP, BE),
    ("wk_exact", 3, 0.5, 2, UP, BE),
    ("wk_fe", 1, 0.3, 2, UP, BE),
    ("wk_be", 0, 1.0, 1, UP, BE),
    ("outlet", 3, 0.5, 3, UP, BE),
    ("cavity", 3, 0.5, 2, UP, BE),
    ("cavity", 2, 1.0, 3, UP, BE),
    ("outlet", 0, 1.0, 2, SOU, BE),
    ("cavity", 3, 0.5, 2, SOU, BE),
    ("wk_exact", 1, 1.0, 2, SOU, BE),
    ("outlet", 3, 1.0, 2, UP, CN),
    ("cavity", 1, 0.5, 2, SOU, CN),
]


@pytest.mark.parametrize("kind,mask,psi,ncorr,conv,time", CASES)
def test_piso_step_adjoint_matches_central_differences(kind, mask, psi, ncorr, conv, time):
    om, x, kw = _case(kind, seed=len(kind) + mask)
    kw.update(nonorth=mask, psi=psi, ncorr=ncorr, conv=conv, time=time)
    y = _fwd(om, x, kw)
    rng = np.random.default_rng(11)
    w = {k: rng.normal(size=np.shape(v)) for k, v in y.items()}
    adj = O.piso_step_bwd(om, x["U"], x["p"], x["phi"], x["Ub"], x["pb"], w["U"], w["p"],
                          w["phi"], w["pb"], w["pc"], pc=x["pc"], **kw)
    assert adj["status"] == 0
    keys = ["U", "p", "phi", "pb", "Ub", "nu"]
    if kind.startswith("wk"):
        keys += ["pc", "Rp", "Cw", "Rd"]
    h = 1e-5
    for key in keys:
        v = rng.normal(size=np.shape(x[key])) if key in x else 1.0

        def shifted(s):
            xx = {k: np.array(a, float) for k, a in x.items()}
            kk = dict(kw)
            if key in xx:
                xx[key] = xx[key] + s * h * v
            elif key == "nu":
                kk["nu"] = kw["nu"] + s * h
            else:
                kk[key] = [kw[key][0] + s * h]
            return _fwd(om, xx, kk)

        yp, ym = shifted(1), shifted(-1)
        dp = sum(np.sum(w[k] * (yp[k] - y[k])) for k in w) / h
        dm = sum(np.sum(w[k] * (y[k] - ym[k])) for k in w) / h
        an = float(np.sum(np.asarray(adj[key]) * v))
        s = max(abs(an), 1.0)
        if abs(0.5 * (dp + dm) - an) > 2e-6 * s:   # central difference, O(h^2), failed:
            # only acceptable if an upwind or limiter switch lies within h of x; the
            # adjoint is then the derivative of the branch taken at x, which the
            # one-sided difference on that side sees
            assert min(abs(dp - an), abs(dm - an)) <= 1e-5 * s, (key, dp, dm, an)


def test_adjoint_of_windkessel_outlet_pressure_is_the_flux_adjoint():
    # With only p_out weighted (through pb on the outlet), the adjoint reaching the
    # outlet face fluxes is the same on every face of the patch: Q = sum of phi_f.
    om, x, kw = _case("wk_exact", 2)
    kw.update(nonorth=0, psi=1.0)
    nb = om.nb
    pbbar = np.zeros(nb)
    q = kw["wk_patch"][0]
    f0, nq = int(om.patch_start[q]) - om.nint, int(om.patch_size[q])
    pbbar[f0:f0 + nq] = 1.0 / nq
    adj = O.piso_step_bwd(om, x["U"], x["p"], x["phi"], x["Ub"], x["pb"], np.zeros((3, om.nc)),
                          np.zeros(om.nc), np.zeros(om.nf), pbbar, [0.0], pc=x["pc"], **kw)
    e = np.exp(-kw["dt"] / (1.2 * 0.8))
    dpo_dQ = 1.2 * (1 - e) + 0.3             # d p_out / d Q of the exact RCR update
    g = adj["phi"][om.nint + f0:om.nint + f0 + nq]
    np.testing.assert_allclose(g, dpo_dQ, rtol=1e-14)
    assert np.all(adj["pb"][f0:f0 + nq] == 0.0)       # the input p_b there is overwritten
    np.testing.assert_allclose(adj["pc"], e, rtol=1e-14)


# ------------------------------------- pulsatile pipe with an RCR outlet (trajectory)
def _pipe_run(om, m, theta, steps, dt, probes, target=None, keep=False):
    """Forward trajectory of the pulsatile pipe; returns the probe-pressure MSE
    (or the probe pressures when target is None) and, with keep, every step's
    inputs (for the reverse sweep)."""
    Rp, Cw, Rd = theta
    out = m.patch_index("outlet")
    fin = m.patch_faces("inlet")
    r2 = (m.Cf[fin, 0] ** 2 + m.Cf[fin, 1] ** 2)
    shape = 1.0 - r2 / r2.max() * 0.999          # parabolic, positive on every face
    area = np.linalg.norm(m.Sf[fin], axis=1)
    kw = dict(nu=0.035, dt=dt, tolU=1e-14, tolp=1e-14, maxitU=5000, maxitp=5000, pref_cell=0,
              wk_patch=[out], Rp=[Rp], Cw=[Cw], Rd=[Rd])
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    pc = np.array([0.0])
    Ub = np.zeros((3, m.n_boundary))
    phi = O.flux_from_U(om, U, Ub)
    probe_p, inputs = [], []
    for k in range(steps):
        t = (k + 1) * dt                           # boundary values at t^{n+1}
        Q = 1.0 + 0.5 * np.sin(2 * np.pi * t) + 0.2 * np.sin(4 * np.pi * t)
        Ub = np.zeros((3, m.n_boundary))
        Ub[2, fin - m.n_internal] = shape * Q / (shape * area).sum()   # inflow along +z, sum u|S| = Q
        if keep:
            inputs.append((U, p, phi, Ub, pb, pc))
        U, p, phi, pb, pc, info = O.piso_step(om, U, p, phi, Ub, pb, pc=pc, **kw)
        assert info["status"] == 0
        probe_p.append(p[probes])
    P = np.array(probe_p)
    if target is None:
        return P
    loss = ((P - target) ** 2).mean()
    return (loss, P, inputs, kw) if keep else loss


def test_pulsatile_pipe_windkessel_gradient_matches_central_differences():
    """A small version of the differentiable pulsatile pipe: d(loss)/d(R_p, C, R_d)
    from the per-step adjoints chained over the trajectory (Sec. 2.5) equals central
    differences of the forward loss."""
    m = mg.pipe_ohgrid(4, 2, 6, L=3.0)
    om = O.OMesh.from_mesh(m)
    steps, dt = 6, 0.0025 * 8
    probes = np.random.default_rng(11).choice(m.n_cells, size=4, replace=False)
    target = _pipe_run(om, m, (0.15, 0.7, 1.3), steps, dt, probes)
    theta = np.array([0.1, 1.0, 1.0])
    loss, P, inputs, kw = _pipe_run(om, m, theta, steps, dt, probes, target, keep=True)
    # reverse sweep: dL/dp at the probes of each step's output, chained through the steps
    Ubar, pbar = np.zeros((3, m.n_cells)), np.zeros(m.n_cells)
    phibar, pbbar, pcbar = np.zeros(m.n_faces), np.zeros(m.n_boundary), np.zeros(1)
    g = np.zeros(3)
    for k in reversed(range(steps)):
        pbar = pbar.copy()
        pbar[probes] += 2.0 * (P[k] - target[k]) / P.size
        U, p, phi, Ub, pb, pc = inputs[k]
        r = O.piso_step_bwd(om, U, p, phi, Ub, pb, Ubar, pbar, phibar, pbbar, pcbar, pc=pc, **kw)
        assert r["status"] == 0
        g += [r["Rp"][0], r["Cw"][0], r["Rd"][0]]
        Ubar, pbar, phibar, pbbar, pcbar = r["U"], r["p"], r["phi"], r["pb"], r["pc"]
    for i in range(3):
        h = 1e-5 * theta[i]
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (_pipe_run(om, m, tp, steps, dt, probes, target) -
              _pipe_run(om, m, tm, steps, dt, probes, target)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-5 * abs(fd) + 1e-12, (i, g[i], fd)
