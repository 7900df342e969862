"""torch.autograd over the library's hand-written adjoints.

* Every operator Function passes torch.autograd.gradcheck in FP64 (central
  differences of the library's own forward against the ``_bwd`` kernels) on a
  small jittered Kuhn mesh: Gauss gradient, convective divergence (upwind and
  linear), the Laplacian with its explicit non-orthogonal part, the LDU apply
  (symmetric and not), the Krylov solve (implicit differentiation w.r.t. the
  coefficients and the right-hand side) and the Windkessel update.
* The PISO-step Function's gradients of a weighted sum of the step's outputs
  (w.r.t. U, p, phi, U_b and nu) equal the oracle's adjoint of that step.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_15920_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_15920_b300 import autograd as A  # noqa: E402
from paper_2603_15920_b300 import difvm as D  # noqa: E402


def nrel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cuda(x, grad=False):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda", requires_grad=grad)


def host(t):
    return t.detach().double().cpu().numpy()


def gradcheck(fn, inputs, atol=1e-7, rtol=1e-5):
    assert torch.autograd.gradcheck(fn, inputs, eps=1e-6, atol=atol, rtol=rtol)


@pytest.fixture(scope="module")
def tiny():
    m = mg.kuhn_cube(2, 0.2, 3)
    return m, D.Mesh(m)


def test_grad_gauss(tiny):
    m, dm = tiny
    rng = np.random.default_rng(0)
    phi, pb = cuda(rng.normal(size=(2, dm.nc)), True), cuda(rng.normal(size=(2, dm.nb)), True)
    gradcheck(lambda a, b: A.grad_gauss(dm, D.BC_VELOCITY, a, b), (phi, pb))


@pytest.mark.parametrize("scheme", [D.DIV_UPWIND, D.DIV_LINEAR])
def test_div_flux(tiny, scheme):
    m, dm = tiny
    rng = np.random.default_rng(1)
    mf = rng.normal(size=dm.nf)
    mf += np.sign(mf) * 0.1          # no face within the perturbation of the upwind switch
    mf, U = cuda(mf, True), cuda(rng.normal(size=(3, dm.nc)), True)
    Ub = cuda(rng.normal(size=(3, dm.nb)), True)
    gradcheck(lambda a, b, c: A.div_flux(dm, scheme, D.BC_VELOCITY, a, b, c), (mf, U, Ub))


def test_laplacian_with_nonorthogonal_part(tiny):
    m, dm = tiny
    rng = np.random.default_rng(2)
    phi, pb = cuda(rng.normal(size=dm.nc), True), cuda(rng.normal(size=dm.nb), True)
    g = cuda(rng.normal(size=(1, 3, dm.nc)), True)
    gradcheck(lambda a, b, c: A.laplacian(dm, D.BC_PRESSURE, 0.7, a, b, c), (phi, pb, g))


@pytest.mark.parametrize("sym", [True, False])
def test_laplacian_apply(tiny, sym):
    m, dm = tiny
    rng = np.random.default_rng(3)
    d = cuda(rng.uniform(1, 2, size=dm.nc), True)
    lo = cuda(rng.normal(size=dm.ni), True)
    up = None if sym else cuda(rng.normal(size=dm.ni), True)
    x = cuda(rng.normal(size=(3, dm.nc)), True)
    if sym:
        gradcheck(lambda a, b, c: A.laplacian_apply(dm, a, b, None, c), (d, lo, x))
    else:
        gradcheck(lambda a, b, c, e: A.laplacian_apply(dm, a, b, c, e), (d, lo, up, x))


def test_krylov_solve_implicit_differentiation(tiny):
    m, dm = tiny
    rng = np.random.default_rng(4)
    ni = m.n_internal
    a = rng.uniform(0.5, 2.0, size=ni)     # SPD: D = row sums of |L| + 0.5, L = -a
    rs = np.bincount(m.owner[:ni], a, m.n_cells) + np.bincount(m.neighbour, a, m.n_cells)
    d = cuda(dm.to_cells(rs + 0.5), True)
    lo = cuda(dm.to_faces(np.concatenate([-a, np.zeros(m.n_boundary)]), flux=False)[:ni], True)
    b = cuda(dm.to_cells(rng.normal(size=m.n_cells)), True)
    opts = D.solve_opts(D.PCG, 1e-14, max_iter=2000)
    gradcheck(lambda p, q, r: A.krylov_solve(dm, p, q, None, r, opts=opts), (d, lo, b), atol=1e-6, rtol=1e-4)


@pytest.mark.parametrize("scheme", [D.WK_EXACT, D.WK_FE, D.WK_BE])
def test_windkessel_update(scheme):
    rng = np.random.default_rng(5)
    Rp, Cw, Rd = (cuda(rng.uniform(0.5, 1.5, size=2), True) for _ in range(3))
    Q, pc = cuda(rng.normal(size=2), True), cuda(rng.normal(size=2), True)
    gradcheck(lambda a, b, c, q, p: A.windkessel_update(scheme, 0.01, a, b, c, q, p), (Rp, Cw, Rd, Q, pc))


def test_piso_step_function_matches_oracle_adjoint():
    m = mg.kuhn_cube(3, 0.2, 5)
    dm, om = D.Mesh(m), O.OMesh.from_mesh(m)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    kw = dict(nu=0.02, dt=0.05, tolU=1e-13, tolp=1e-13, pref_cell=0, nonorth=3)
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    for _ in range(2):   # a developed input state
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, **kw)
    h = D.Piso(dm, D.F64, D.piso_opts(0.02, 0.05, 2, 3,
                                      solve_U=D.solve_opts(D.BICGSTAB, 1e-13, max_iter=5000),
                                      solve_p=D.solve_opts(D.PCG, 1e-13, max_iter=20000),
                                      pref_cell=int(dm.cell_new_of_old[0])))
    x = [cuda(dm.to_cells(U), True), cuda(dm.to_cells(p), True), cuda(dm.to_faces(phi), True),
         cuda(dm.to_bnd(Ub), True), cuda(dm.to_bnd(pb), True)]
    nu = torch.tensor([0.02], dtype=torch.float64, device="cuda", requires_grad=True)
    rng = np.random.default_rng(6)
    wU, wp, wphi = rng.normal(size=(3, m.n_cells)), rng.normal(size=m.n_cells), rng.normal(size=m.n_faces)
    U1, p1, phi1, _ = A.piso_step(h, *x, nu=nu)
    loss = (cuda(dm.to_cells(wU)) * U1).sum() + (cuda(dm.to_cells(wp)) * p1).sum() + \
        (cuda(dm.to_faces(wphi)) * phi1).sum()
    loss.backward()
    ref = O.piso_step_bwd(om, U, p, phi, Ub, pb, wU, wp, wphi, **kw)
    assert ref["status"] == 0
    assert nrel(dm.from_cells(host(x[0].grad)), ref["U"]) < 1e-8
    assert nrel(dm.from_cells(host(x[1].grad)), ref["p"]) < 1e-8
    assert nrel(dm.from_faces(host(x[2].grad)), ref["phi"]) < 1e-8
    assert nrel(dm.from_bnd(host(x[3].grad)), ref["Ub"]) < 1e-8
    assert abs(float(nu.grad[0]) - ref["nu"]) <= 1e-8 * abs(ref["nu"])
    # the inputs are left as they were
    assert np.array_equal(dm.from_cells(host(x[0])), U)
