"""GPU parity of the face operators against the CPU oracle (element by element).

Meshes are shuffled (random cell / face numbering) so that the library's RCM
renumbering, face re-orientation and sorting are exercised; every comparison
is made in the input numbering after mapping the GPU result back.  Sizes span
many 256-thread blocks with a ragged tail; the full 64^3 Kuhn mesh is checked
at the launch configuration the benchmark uses.
Tolerances: FP64 1e-12 and FP32 1e-5, normwise relative
||x_gpu - x_ref||_inf / ||x_ref||_inf.
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

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
DTYPES = [torch.float64, torch.float32]


def nrel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cuda(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda").contiguous()


MESHES = {
    "kuhn10": lambda: mg.shuffle(mg.kuhn_cube(10, 0.2, 3, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET)), 11),
    "channel": lambda: mg.channel_2d(32, 8, seed=4),
    "dbox": lambda: mg.shuffle(mg.distorted_box(9, 0.05, patch_types=dict(y1=mg.OUTLET)), 2),
    "pipe": lambda: mg.pipe_ohgrid(8, 4, 6),
}
_cache = {}


def get(name):
    if name not in _cache:
        m = MESHES[name]()
        _cache[name] = (m, O.OMesh.from_mesh(m), D.Mesh(m))
    return _cache[name]


def bc_table(om, cls):
    return {D.BC_VELOCITY: om.bc_U(), D.BC_PRESSURE: om.bc_p(),
            D.BC_ALL_FIXED: np.where(om.patch_type == O.PT_EMPTY, O.BC_EMPTY, O.BC_FIXED).astype(np.int32),
            D.BC_ALL_ZEROGRAD: np.where(om.patch_type == O.PT_EMPTY, O.BC_EMPTY, O.BC_ZEROGRAD).astype(np.int32)}[cls]


@pytest.mark.parametrize("name", list(MESHES))
def test_mesh_create_maps(name):
    m, om, dm = get(name)
    assert dm.nc == m.n_cells and dm.nf == m.n_faces
    assert sorted(dm.cell_new_of_old.tolist()) == list(range(m.n_cells))
    assert sorted(dm.face_old_of_new.tolist()) == list(range(m.n_faces))
    # boundary faces stay inside their patch
    for p in range(m.n_patches):
        s, z = int(m.patch_start[p]), int(m.patch_size[p])
        assert set(dm.face_old_of_new[s:s + z].tolist()) == set(range(s, s + z))
    assert dm.nnz == 2 * m.n_internal + m.n_boundary


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("cls", [D.BC_VELOCITY, D.BC_PRESSURE, D.BC_ALL_FIXED, D.BC_ALL_ZEROGRAD])
def test_grad_gauss(name, cls, dt):
    m, om, dm = get(name)
    f = mg.random_fields(m, 1)
    for nq in (1, 3):
        phi = f["U"][:nq]
        phib = f["U_b"][:nq]
        ref = O.grad_gauss(om, bc_table(om, cls), phi, phib)
        out = D.difvm_grad_gauss(dm, cls, cuda(dm.to_cells(phi), dt), cuda(dm.to_bnd(phib), dt))
        got = dm.from_cells(out.double().cpu().numpy())
        assert nrel(got, ref) < TOL[dt], (nq, nrel(got, ref))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("scheme", [D.DIV_UPWIND, D.DIV_LINEAR])
def test_div_flux(name, scheme, dt):
    m, om, dm = get(name)
    f = mg.random_fields(m, 2)
    mflux = f["m"].copy()
    mflux[::17] = 0.0                     # upwind tie: m = 0 takes the owner value
    for cls in (D.BC_VELOCITY, D.BC_PRESSURE):
        for nq in (1, 3):
            ref = O.div_flux(om, bc_table(om, cls), scheme, mflux, f["U"][:nq], f["U_b"][:nq])
            out = D.difvm_div_flux(dm, scheme, cls, cuda(dm.to_faces(mflux), dt),
                                   cuda(dm.to_cells(f["U"][:nq]), dt), cuda(dm.to_bnd(f["U_b"][:nq]), dt))
            got = dm.from_cells(out.double().cpu().numpy())
            assert nrel(got, ref) < TOL[dt], (cls, nq, nrel(got, ref))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("nonorth", [False, True])
def test_laplacian(name, nonorth, dt):
    m, om, dm = get(name)
    f = mg.random_fields(m, 3)
    rng = np.random.default_rng(5)
    for cls in (D.BC_VELOCITY, D.BC_PRESSURE, D.BC_ALL_FIXED):
        for nq in (1, 3):
            g = rng.standard_normal((nq, 3, m.n_cells)) if nonorth else None
            ref = O.laplacian(om, bc_table(om, cls), 0.37, f["U"][:nq], f["U_b"][:nq], g)
            out = D.difvm_laplacian(dm, cls, 0.37, cuda(dm.to_cells(f["U"][:nq]), dt),
                                    cuda(dm.to_bnd(f["U_b"][:nq]), dt),
                                    None if g is None else cuda(dm.to_cells(g), dt))
            got = dm.from_cells(out.double().cpu().numpy())
            assert nrel(got, ref) < TOL[dt], (cls, nq, nrel(got, ref))


SPLITS = [(D.NONORTH_MINIMUM, O.NONORTH_MINIMUM), (D.NONORTH_ORTHOGONAL, O.NONORTH_ORTHOGONAL),
          (D.NONORTH_NONE, O.NONORTH_NONE)]


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("name", ["kuhn10", "dbox"])
@pytest.mark.parametrize("split", SPLITS, ids=["minimum", "orthogonal", "none"])
def test_laplacian_nonorth_splits(name, split, dt):
    # the other splits of Eq. nonortho_flux (mesh flag) against the oracle's
    m = get(name)[0]
    om, dm = O.OMesh.from_mesh(m, split[1]), D.Mesh(m, nonorth=split[0])
    f = mg.random_fields(m, 4)
    g = np.random.default_rng(6).standard_normal((3, 3, m.n_cells))
    for cls in (D.BC_VELOCITY, D.BC_ALL_FIXED):
        ref = O.laplacian(om, bc_table(om, cls), 0.37, f["U"], f["U_b"], g)
        out = D.difvm_laplacian(dm, cls, 0.37, cuda(dm.to_cells(f["U"]), dt), cuda(dm.to_bnd(f["U_b"]), dt),
                                cuda(dm.to_cells(g), dt))
        got = dm.from_cells(out.double().cpu().numpy())
        assert nrel(got, ref) < TOL[dt], (cls, nrel(got, ref))


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("name", list(MESHES))
def test_laplacian_apply(name, dt):
    m, om, dm = get(name)
    rng = np.random.default_rng(6)
    Dg, L, U = rng.standard_normal(m.n_cells), rng.standard_normal(m.n_internal), rng.standard_normal(m.n_internal)
    x = rng.standard_normal((3, m.n_cells))
    # internal numbering of face coefficients: lower/upper swap on flipped faces
    flip = dm.face_flip[:m.n_internal] != 0
    Li = np.where(flip, U[dm.face_old_of_new[:m.n_internal]], L[dm.face_old_of_new[:m.n_internal]])
    Ui = np.where(flip, L[dm.face_old_of_new[:m.n_internal]], U[dm.face_old_of_new[:m.n_internal]])
    for nq in (1, 2, 3):
        for tr in (False, True):
            ref = O.ldu_apply(om, Dg, U if tr else L, L if tr else U, x[:nq])
            out = D.difvm_laplacian_apply(dm, cuda(dm.to_cells(Dg), dt), cuda(Li, dt), cuda(Ui, dt),
                                          cuda(dm.to_cells(x[:nq]), dt), transpose=tr)
            got = dm.from_cells(out.double().cpu().numpy())
            assert nrel(got, ref) < TOL[dt], (nq, tr, nrel(got, ref))
        ref = O.ldu_apply(om, Dg, L, None, x[:nq])       # symmetric: one coefficient per face
        out = D.difvm_laplacian_apply(dm, cuda(dm.to_cells(Dg), dt), cuda(L[dm.face_old_of_new[:m.n_internal]], dt),
                                      None, cuda(dm.to_cells(x[:nq]), dt))
        assert nrel(dm.from_cells(out.double().cpu().numpy()), ref) < TOL[dt]


def test_operators_are_deterministic():
    m, om, dm = get("kuhn10")
    f = mg.random_fields(m, 7)
    phi = cuda(dm.to_cells(f["U"]), torch.float64)
    phib = cuda(dm.to_bnd(f["U_b"]), torch.float64)
    a = D.difvm_grad_gauss(dm, D.BC_VELOCITY, phi, phib)
    b = D.difvm_grad_gauss(dm, D.BC_VELOCITY, phi, phib)
    assert torch.equal(a, b)


def test_constant_field_conservation_bitwise_antisymmetry():
    # the owner and neighbour see bitwise the same face message: the sum of a
    # divergence over all cells equals the boundary flux up to summation rounding
    m, om, dm = get("kuhn10")
    f = mg.random_fields(m, 8)
    mf = cuda(dm.to_faces(f["m"]), torch.float64)
    phi = cuda(dm.to_cells(f["phi"]), torch.float64)
    out = D.difvm_div_flux(dm, D.DIV_LINEAR, D.BC_ALL_ZEROGRAD, mf, phi).cpu().numpy()
    ob = dm.to_cells(np.arange(m.n_cells))  # noqa: F841
    bflux = (f["m"][m.n_internal:] * f["phi"][m.owner[m.n_internal:]]).sum()
    assert abs(out.sum() - bflux) < 1e-11 * np.abs(out).sum()


def test_bad_arguments_raise():
    m, om, dm = get("channel")
    phi = torch.zeros(5, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(D.DifvmError) as e:     # unknown bc class
        D._check(D.lib().difvm_grad_gauss(dm.h, 1, 9, phi.data_ptr(), None, 1, phi.data_ptr(), None))
    assert e.value.status == D.EINVAL
    with pytest.raises(D.DifvmError):          # ncomp out of range
        D._check(D.lib().difvm_grad_gauss(dm.h, 1, 0, phi.data_ptr(), None, 4, phi.data_ptr(), None))
    with pytest.raises(D.DifvmError):          # bad precision
        D._check(D.lib().difvm_grad_gauss(dm.h, 7, 0, phi.data_ptr(), None, 1, phi.data_ptr(), None))


def test_mesh_create_rejects_unknown_flags():
    m = get("kuhn10")[0]
    with pytest.raises(D.DifvmError):
        D.Mesh(m, flags=D.RENUMBER_RCM | 32)


def test_mesh_create_rejects_bad_meshes():
    m = mg.kuhn_cube(2, 0.0, 0)
    bad = mg.Mesh(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.__dict__.items()})
    bad.neighbour[3] = m.n_cells + 5
    with pytest.raises(D.DifvmError, match="out of range"):
        D.Mesh(bad)
    bad = mg.Mesh(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.__dict__.items()})
    bad.Sf[7] *= -1.0                           # area vector pointing into the owner
    with pytest.raises(D.DifvmError, match="S.d"):
        D.Mesh(bad)
    bad = mg.Mesh(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.__dict__.items()})
    bad.V[0] = 0.0
    with pytest.raises(D.DifvmError, match="not positive"):
        D.Mesh(bad)


def test_single_cell_mesh():
    # no internal faces at all: every operator reduces boundary faces only
    m = mg.hex_box(1, 1, 1, (1.0, 2.0, 3.0))
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    phib = np.arange(6.0)[None]
    ref = O.grad_gauss(om, O.BC_FIXED, np.ones((1, 1)), phib)
    got = D.difvm_grad_gauss(dm, D.BC_ALL_FIXED, cuda(np.ones((1, 1)), torch.float64),
                             cuda(dm.to_bnd(phib), torch.float64)).cpu().numpy()
    assert nrel(got, ref) < 1e-14


# ------------------------------------------------------------------ adjoints
def _dense_T(apply, n_in, w):
    """Oracle J^T w for a linear map, built column by column from unit vectors."""
    out = np.zeros(n_in)
    for k in range(n_in):
        e = np.zeros(n_in); e[k] = 1.0
        out[k] = np.dot(apply(e).ravel(), w.ravel())
    return out


@pytest.fixture(scope="module")
def tiny():
    m = mg.shuffle(mg.kuhn_cube(3, 0.2, 9, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET)), 3)
    return m, O.OMesh.from_mesh(m), D.Mesh(m)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("cls", [D.BC_VELOCITY, D.BC_PRESSURE])
def test_grad_gauss_bwd_is_oracle_transpose(tiny, cls, dt):
    m, om, dm = tiny
    nc, nb = m.n_cells, m.n_boundary
    rng = np.random.default_rng(1)
    w = rng.standard_normal((1, 3, nc))
    bc = bc_table(om, cls)
    ref_phi = _dense_T(lambda e: O.grad_gauss(om, bc, e, np.zeros(nb)), nc, w)
    ref_pb = _dense_T(lambda e: O.grad_gauss(om, bc, np.zeros(nc), e), nb, w)
    pbar = torch.zeros(1, nc, dtype=dt, device="cuda")
    pbbar = torch.zeros(1, nb, dtype=dt, device="cuda")
    D.difvm_grad_gauss_bwd(dm, cls, cuda(dm.to_cells(w), dt), pbar, pbbar)
    e = nrel(dm.from_cells(pbar.double().cpu().numpy())[0], ref_phi)
    assert e < TOL[dt], e
    if np.abs(ref_pb).max() > 0:
        e = nrel(dm.from_bnd(pbbar.double().cpu().numpy())[0], ref_pb)
        assert e < TOL[dt], e


def _upwind_mflux_T(om, bc, mf, phi, pb, w):
    """Oracle d<div_flux(m), w>/dm_f for the upwind scheme.  The upwind face
    flux m_f phi_upwind(m_f) is positively homogeneous in m_f, so the
    derivative at m_f != 0 is the oracle's divergence of the one-face flux
    m_f e_f, divided by m_f (no finite-difference step)."""
    out = np.zeros(mf.shape[0])
    for k in range(mf.shape[0]):
        e = np.zeros_like(mf); e[k] = mf[k]
        out[k] = np.dot(O.div_flux(om, bc, O.DIV_UPWIND, e, phi, pb).ravel(), w.ravel()) / mf[k]
    return out


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("scheme", [D.DIV_UPWIND, D.DIV_LINEAR])
def test_div_flux_bwd_is_oracle_transpose(tiny, scheme, dt):
    m, om, dm = tiny
    nc, nb, nf = m.n_cells, m.n_boundary, m.n_faces
    rng = np.random.default_rng(2)
    mf = rng.standard_normal(nf); phi = rng.standard_normal(nc); pb = rng.standard_normal(nb)
    w = rng.standard_normal(nc)
    bc = om.bc_U()
    ref_phi = _dense_T(lambda e: O.div_flux(om, bc, scheme, mf, e, np.zeros(nb)), nc, w)
    ref_pb = _dense_T(lambda e: O.div_flux(om, bc, scheme, mf, np.zeros(nc), e), nb, w)
    if scheme == D.DIV_LINEAR:
        ref_m = _dense_T(lambda e: O.div_flux(om, bc, scheme, e * 1.0, phi, pb), nf, w)
    else:
        ref_m = _upwind_mflux_T(om, bc, mf, phi, pb, w)
    mbar = torch.zeros(nf, dtype=dt, device="cuda")
    pbar = torch.zeros(1, nc, dtype=dt, device="cuda")
    pbbar = torch.zeros(1, nb, dtype=dt, device="cuda")
    D.difvm_div_flux_bwd(dm, scheme, D.BC_VELOCITY, cuda(dm.to_faces(mf), dt), cuda(dm.to_cells(phi)[None], dt),
                         cuda(dm.to_bnd(pb)[None], dt), cuda(dm.to_cells(w)[None], dt), mbar, pbar, pbbar)
    errs = (nrel(dm.from_cells(pbar.double().cpu().numpy())[0], ref_phi),
            nrel(dm.from_bnd(pbbar.double().cpu().numpy())[0], ref_pb),
            nrel(dm.from_faces(mbar.double().cpu().numpy()), ref_m))
    assert max(errs) < TOL[dt], errs


@pytest.mark.parametrize("dt", DTYPES)
def test_laplacian_bwd_is_oracle_transpose(tiny, dt):
    m, om, dm = tiny
    nc, nb = m.n_cells, m.n_boundary
    rng = np.random.default_rng(3)
    w = rng.standard_normal(nc)
    bc = om.bc_U()
    g0 = np.zeros((1, 3, nc))
    ref_phi = _dense_T(lambda e: O.laplacian(om, bc, 0.7, e, np.zeros(nb), g0), nc, w)
    ref_pb = _dense_T(lambda e: O.laplacian(om, bc, 0.7, np.zeros(nc), e, g0), nb, w)
    ref_g = _dense_T(lambda e: O.laplacian(om, bc, 0.7, np.zeros(nc), np.zeros(nb), e.reshape(1, 3, nc)), 3 * nc, w)
    pbar = torch.zeros(1, nc, dtype=dt, device="cuda")
    pbbar = torch.zeros(1, nb, dtype=dt, device="cuda")
    gbar = torch.zeros(1, 3, nc, dtype=dt, device="cuda")
    D.difvm_laplacian_bwd(dm, D.BC_VELOCITY, 0.7, cuda(dm.to_cells(w)[None], dt), pbar, pbbar, gbar)
    errs = (nrel(dm.from_cells(pbar.double().cpu().numpy())[0], ref_phi),
            nrel(dm.from_bnd(pbbar.double().cpu().numpy())[0], ref_pb),
            nrel(dm.from_cells(gbar.double().cpu().numpy()).ravel(), ref_g))
    assert max(errs) < TOL[dt], errs


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("sym", [False, True])
def test_laplacian_apply_bwd_is_oracle_transpose(tiny, sym, dt):
    m, om, dm = tiny
    rng = np.random.default_rng(4)
    nc, ni = m.n_cells, m.n_internal
    fo, flip = dm.face_old_of_new[:ni], dm.face_flip[:ni] != 0
    # coefficients in the input numbering; internally L and U swap on flipped faces
    Dg = rng.standard_normal(nc)
    L = rng.standard_normal(ni)
    U = L if sym else rng.standard_normal(ni)
    x, ybar = rng.standard_normal((2, nc)), rng.standard_normal((2, nc))
    Li, Ui = np.where(flip, U[fo], L[fo]), np.where(flip, L[fo], U[fo])
    xg, yg = cuda(dm.to_cells(x), dt), cuda(dm.to_cells(ybar), dt)
    Dgg, Lg, Ug = cuda(dm.to_cells(Dg), dt), cuda(Li, dt), None if sym else cuda(Ui, dt)
    xbar = torch.zeros_like(xg)
    Dbar, Lbar = torch.zeros_like(Dgg), torch.zeros_like(Lg)
    Ubar = None if sym else torch.zeros_like(Lg)
    D.difvm_laplacian_apply_bwd(dm, Dgg, Lg, Ug, xg, yg, xbar, Dbar, Lbar, Ubar)
    # x_bar = A^T y_bar: the oracle's apply with L and U swapped
    ref_x = O.ldu_apply(om, Dg, U, L, ybar)
    e = nrel(dm.from_cells(xbar.double().cpu().numpy()), ref_x)
    assert e < TOL[dt], e
    # coefficient gradients: the oracle's y = A x is linear in D, L and U
    z = np.zeros(ni)
    ref_D = _dense_T(lambda e_: O.ldu_apply(om, e_, z, z, x), nc, ybar)
    e = nrel(dm.from_cells(Dbar.double().cpu().numpy()), ref_D)
    assert e < TOL[dt], e
    lb, ub = Lbar.double().cpu().numpy(), None if sym else Ubar.double().cpu().numpy()
    if sym:
        ref_L = _dense_T(lambda e_: O.ldu_apply(om, np.zeros(nc), e_, None, x), ni, ybar)
        got_L = np.empty(ni); got_L[fo] = lb
        e = nrel(got_L, ref_L)
        assert e < TOL[dt], e
    else:
        ref_L = _dense_T(lambda e_: O.ldu_apply(om, np.zeros(nc), e_, z, x), ni, ybar)
        ref_U = _dense_T(lambda e_: O.ldu_apply(om, np.zeros(nc), z, e_, x), ni, ybar)
        got_L, got_U = np.empty(ni), np.empty(ni)
        got_L[fo], got_U[fo] = np.where(flip, ub, lb), np.where(flip, lb, ub)
        errs = nrel(got_L, ref_L), nrel(got_U, ref_U)
        assert max(errs) < TOL[dt], errs
    # and the dot-product identity <A x, y_bar> = <x, A^T y_bar>, within the
    # rounding bound TOL * sum of |terms|
    y = D.difvm_laplacian_apply(dm, Dgg, Lg, Ug, xg).double()
    lhs = (y * yg.double()).sum().item()
    rhs = (xg.double() * xbar.double()).sum().item()
    scale = (y.abs() * yg.double().abs()).sum().item() + (xg.double() * xbar.double()).abs().sum().item()
    assert abs(lhs - rhs) < TOL[dt] * scale, (lhs, rhs, scale)


# ---------------------------------------------------------- full-size (64^3)
@pytest.fixture(scope="module")
def kuhn64():
    m = mg.kuhn_cube(64, 0.2, 0)
    return m, O.OMesh.from_mesh(m), D.Mesh(m)


@pytest.mark.parametrize("dt", DTYPES)
def test_full_size_operators(kuhn64, dt):
    # every face operator on the 1.6M-cell mesh, launched as the benchmark launches it
    m, om, dm = kuhn64
    f = mg.random_fields(m, 0)
    phi, phib = f["phi"], f["phi_b"]
    errs = {}

    def check(name, got, ref):
        errs[name] = nrel(got, ref)

    ref = O.grad_gauss(om, om.bc_p(), phi, phib)
    check("grad_gauss_scalar", dm.from_cells(D.difvm_grad_gauss(
        dm, D.BC_PRESSURE, cuda(dm.to_cells(phi), dt), cuda(dm.to_bnd(phib), dt)).double().cpu().numpy()), ref)
    ref = O.grad_gauss(om, om.bc_U(), f["U"], f["U_b"])
    check("grad_gauss_vector", dm.from_cells(D.difvm_grad_gauss(
        dm, D.BC_VELOCITY, cuda(dm.to_cells(f["U"]), dt), cuda(dm.to_bnd(f["U_b"]), dt)).double().cpu().numpy()), ref)
    for scheme, nm in ((O.DIV_UPWIND, "upwind"), (O.DIV_LINEAR, "linear")):
        ref = O.div_flux(om, om.bc_U(), scheme, f["m"], f["U"], f["U_b"])
        check("div_flux_" + nm, dm.from_cells(D.difvm_div_flux(
            dm, scheme, D.BC_VELOCITY, cuda(dm.to_faces(f["m"]), dt), cuda(dm.to_cells(f["U"]), dt),
            cuda(dm.to_bnd(f["U_b"]), dt)).double().cpu().numpy()), ref)
    fix = bc_table(om, D.BC_ALL_FIXED)
    g = O.grad_gauss(om, fix, phi, phib)
    ref = O.laplacian(om, fix, 1.0, phi, phib, g)
    check("laplacian_nonorth", dm.from_cells(D.difvm_laplacian(
        dm, D.BC_ALL_FIXED, 1.0, cuda(dm.to_cells(phi), dt), cuda(dm.to_bnd(phib), dt),
        cuda(dm.to_cells(g), dt)).double().cpu().numpy()), ref)
    rng = np.random.default_rng(8)
    ni, fo, flip = m.n_internal, dm.face_old_of_new[:m.n_internal], dm.face_flip[:m.n_internal] != 0
    Dg, L, U = rng.standard_normal(m.n_cells) + 10.0, rng.standard_normal(ni), rng.standard_normal(ni)
    x = rng.standard_normal((3, m.n_cells))
    ref = O.ldu_apply(om, Dg, L, None, x[:1])
    check("laplacian_apply_sym_1", dm.from_cells(D.difvm_laplacian_apply(
        dm, cuda(dm.to_cells(Dg), dt), cuda(L[fo], dt), None,
        cuda(dm.to_cells(x[:1]), dt)).double().cpu().numpy()), ref)
    ref = O.ldu_apply(om, Dg, L, U, x)
    check("laplacian_apply_asym_3", dm.from_cells(D.difvm_laplacian_apply(
        dm, cuda(dm.to_cells(Dg), dt), cuda(np.where(flip, U[fo], L[fo]), dt),
        cuda(np.where(flip, L[fo], U[fo]), dt), cuda(dm.to_cells(x), dt)).double().cpu().numpy()), ref)
    assert max(errs.values()) < TOL[dt], errs


# ------------------------------------------------------------- autotuning
def test_autotuned_variants_agree_and_are_kept():
    # the F32 face operators of a tetrahedral mesh time their launch variants on
    # first use; every variant computes the same sums in the same order
    m = get("kuhn10")[0]
    dm = D.Mesh(m)
    D.difvm_mesh_autotune(dm, 0)
    f = mg.random_fields(m, 9)
    dt = torch.float32
    phi, U = cuda(dm.to_cells(f["U"][:1]), dt), cuda(dm.to_cells(f["U"]), dt)
    phib, Ub = cuda(dm.to_bnd(f["U_b"][:1]), dt), cuda(dm.to_bnd(f["U_b"]), dt)
    mf = cuda(dm.to_faces(f["m"]), dt)
    g = D.difvm_grad_gauss(dm, D.BC_ALL_FIXED, phi, phib)
    rng = np.random.default_rng(3)
    Dg, L = cuda(rng.standard_normal(dm.nc) + 5.0, dt), cuda(rng.standard_normal(dm.ni), dt)
    ops = {
        (1, 0, 1): lambda: D.difvm_grad_gauss(dm, D.BC_VELOCITY, phi, phib),
        (1, 0, 3): lambda: D.difvm_grad_gauss(dm, D.BC_VELOCITY, U, Ub),
        (2, 1, 3): lambda: D.difvm_div_flux(dm, D.DIV_UPWIND, D.BC_VELOCITY, mf, U, Ub),
        (2, 0, 3): lambda: D.difvm_div_flux(dm, D.DIV_LINEAR, D.BC_PRESSURE, mf, U, Ub),
        (3, 1, 1): lambda: D.difvm_laplacian(dm, D.BC_ALL_FIXED, 0.3, phi, phib, g),
        (3, 0, 3): lambda: D.difvm_laplacian(dm, D.BC_VELOCITY, 0.3, U, Ub),
        (4, 0, 3): lambda: D.difvm_laplacian_apply(dm, Dg, L, None, U),
    }
    ref = {k: fn().clone() for k, fn in ops.items()}
    assert D.difvm_mesh_tuning(dm) == {}
    D.difvm_mesh_autotune(dm, 2)
    for k, fn in ops.items():
        first, second = fn().clone(), fn().clone()
        assert torch.equal(first, ref[k]) and torch.equal(second, ref[k]), k
    kept = D.difvm_mesh_tuning(dm)
    assert set(kept) >= set(ops) and all(0 <= v <= 2 for v in kept.values()), kept
    with pytest.raises(D.DifvmError):
        D.difvm_mesh_autotune(dm, 3)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("name", ["kuhn10", "pipe"])
def test_wide_index_layouts_give_bitwise_the_same_operators(name, dt):
    # compact 4-byte slot words (other cell and face id as offsets) against the
    # 8-byte (word, face id) slots that DIFVM_WIDE_INDICES selects (and that large
    # meshes use): the same faces in the same order, so bitwise the same sums
    m = get(name)[0]
    f = mg.random_fields(m, 11)
    res = []
    for flags in (D.RENUMBER_RCM | D.SORT_FACES, D.RENUMBER_RCM | D.SORT_FACES | D.WIDE_INDICES):
        dm = D.Mesh(m, flags=flags)
        assert D.difvm_mesh_layout(dm)[0] == (not flags & D.WIDE_INDICES)
        phi, U = cuda(dm.to_cells(f["U"][:1]), dt), cuda(dm.to_cells(f["U"]), dt)
        phib, Ub = cuda(dm.to_bnd(f["U_b"][:1]), dt), cuda(dm.to_bnd(f["U_b"]), dt)
        mf = cuda(dm.to_faces(f["m"]), dt)
        g = D.difvm_grad_gauss(dm, D.BC_ALL_FIXED, phi, phib)
        rng = np.random.default_rng(5)
        Dg, L, Uu = (cuda(rng.standard_normal(dm.nc) + 5.0, dt), cuda(rng.standard_normal(dm.ni), dt),
                     cuda(rng.standard_normal(dm.ni), dt))
        outs = [g,
                D.difvm_grad_gauss(dm, D.BC_VELOCITY, U, Ub),
                D.difvm_grad_gauss(dm, D.BC_PRESSURE, phi, phib),
                D.difvm_div_flux(dm, D.DIV_UPWIND, D.BC_VELOCITY, mf, U, Ub),
                D.difvm_div_flux(dm, D.DIV_LINEAR, D.BC_PRESSURE, mf, U, Ub),
                D.difvm_laplacian(dm, D.BC_ALL_FIXED, 0.3, phi, phib, g),
                D.difvm_laplacian(dm, D.BC_VELOCITY, 0.3, U, Ub),
                D.difvm_laplacian_apply(dm, Dg, L, None, phi),
                D.difvm_laplacian_apply(dm, Dg, L, Uu, U)]
        res.append([dm.from_cells(o.cpu().numpy()) for o in outs])
    for k, (a, b) in enumerate(zip(*res)):
        assert np.array_equal(a, b), k
