"""The allocation-free LDU-apply adjoint against the regular one and the oracle.

difvm_laplacian_apply_bwd_noalloc serves callers that cannot allocate device
memory (their memory belongs to another runtime's pool, or they run a loop
where cudaMalloc's device-wide synchronisation is not acceptable): it forms
A^T y_bar in a scratch array built into the library instead of a buffer the
caller passes.  Its outputs must equal those of difvm_laplacian_apply_bwd,
on two calls in a row (the second call reuses the scratch the first one left
behind): bitwise, since both run the same transposed apply and the same
accumulation.  The FP64 x_bar increment is also checked against the oracle's
LDU apply with L and U swapped, and the call must leave the device's free
memory and torch's allocator untouched.  This file is collected last on
purpose.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2603_15920_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_15920_b300 import difvm as D  # noqa: E402

# the built-in scratch: 16 MiB
LIMIT_BYTES = 16 << 20


def nrel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def mesh():
    m = mg.shuffle(mg.kuhn_cube(8, 0.2, 4), 6)
    return m, O.OMesh.from_mesh(m), D.Mesh(m)


def _call_noalloc(dm, prec, Dg, L, U, x, ybar, xbar, Dbar, Lbar, Ubar):
    p = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    return D.lib().difvm_laplacian_apply_bwd_noalloc(
        dm.h, prec, p(Dg), p(L), p(U), p(x), p(ybar), x.shape[0], p(xbar), p(Dbar), p(Lbar), p(Ubar),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("sym", [False, True])
def test_noalloc_matches_regular_adjoint_twice(mesh, dt, sym):
    m, om, dm = mesh
    prec = D.F64 if dt == torch.float64 else D.F32
    rng = np.random.default_rng(11)
    ni, fo = m.n_internal, dm.face_old_of_new[:m.n_internal]
    flip = dm.face_flip[:ni] != 0
    for call in range(2):                   # two calls in a row, different inputs
        cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda").contiguous()
        # coefficients and fields in the input numbering, mapped to the library's
        Dg_in = rng.standard_normal(m.n_cells)
        L_in = rng.standard_normal(ni)
        U_in = L_in if sym else rng.standard_normal(ni)
        ybar_in = rng.standard_normal((3, m.n_cells))
        Li = np.where(flip, U_in[fo], L_in[fo])
        Ui = np.where(flip, L_in[fo], U_in[fo])
        Dg, L, U = cu(dm.to_cells(Dg_in)), cu(Li), None if sym else cu(Ui)
        x = cu(dm.to_cells(rng.standard_normal((3, m.n_cells))))
        ybar = cu(dm.to_cells(ybar_in))
        start = cu(rng.standard_normal((3, m.n_cells)))      # outputs accumulate
        ref = [start.clone(), torch.zeros_like(Dg), torch.zeros_like(L),
               None if sym else torch.zeros_like(L)]
        got = [start.clone(), torch.zeros_like(Dg), torch.zeros_like(L),
               None if sym else torch.zeros_like(L)]
        D.difvm_laplacian_apply_bwd(dm, Dg, L, U, x, ybar, *ref)
        st = _call_noalloc(dm, prec, Dg, L, U, x, ybar, *got)
        assert st == D.OK, D.lib().difvm_last_error()
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            if r is not None:
                assert torch.equal(g, r), call
        if dt == torch.float64:
            # x_bar - start = A^T y_bar: the oracle's apply with L and U swapped
            inc = dm.from_cells((got[0] - start).cpu().numpy())
            want = O.ldu_apply(om, Dg_in, U_in, L_in, ybar_in)
            assert nrel(inc, want) < 1e-12, (call, nrel(inc, want))


def test_noalloc_allocates_nothing(mesh):
    m, om, dm = mesh
    rng = np.random.default_rng(12)
    cu = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()
    Dg, L = cu(rng.standard_normal(dm.nc)), cu(rng.standard_normal(dm.ni))
    x, ybar = cu(rng.standard_normal((3, dm.nc))), cu(rng.standard_normal((3, dm.nc)))
    xbar, Dbar, Lbar = torch.zeros_like(x), torch.zeros_like(Dg), torch.zeros_like(L)
    # warm-up: loads the kernels' code and looks up the scratch's address
    assert _call_noalloc(dm, D.F64, Dg, L, None, x, ybar, xbar, Dbar, Lbar, None) == D.OK
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert _call_noalloc(dm, D.F64, Dg, L, None, x, ybar, xbar, Dbar, Lbar, None) == D.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


@pytest.fixture(scope="module")
def at_limit():
    # 128^3 hexes: 2,097,152 cells = the FP64 one-component limit and the FP32
    # two-component limit exactly; one extra cell puts both one element over
    m = mg.hex_box(128, 128, 128)
    over, _ = mg.batch([m, mg.hex_box(1, 1, 1)])
    return D.Mesh(m), D.Mesh(over)


def _limit_call(dm, dt, nq, with_xbar=True, coeff=False):
    x = torch.ones(nq, dm.nc, dtype=dt, device="cuda")
    L = torch.full((dm.ni,), -0.1, dtype=dt, device="cuda")
    Dg = torch.ones(dm.nc, dtype=dt, device="cuda")
    xbar = torch.zeros_like(x) if with_xbar else None
    Dbar = torch.zeros_like(Dg) if coeff else None
    Lbar = torch.zeros_like(L) if coeff else None
    st = _call_noalloc(dm, D.F64 if dt == torch.float64 else D.F32, Dg, L, None, x, x, xbar, Dbar,
                       Lbar, None)
    torch.cuda.synchronize()
    return st, xbar, Dbar


@pytest.mark.parametrize("dt,nq", [(torch.float64, 1), (torch.float32, 2)])
def test_noalloc_size_limit_is_exact(at_limit, dt, nq):
    exact, over = at_limit
    elt = 8 if dt == torch.float64 else 4
    assert exact.nc * nq * elt == LIMIT_BYTES and over.nc * nq * elt == LIMIT_BYTES + nq * elt
    st, xbar, _ = _limit_call(exact, dt, nq)
    assert st == D.OK, D.lib().difvm_last_error()
    # A^T 1 with D = 1, L = U = -0.1: 1 - 0.1 x (number of internal faces of the cell)
    assert float(xbar.max()) == pytest.approx(1.0 - 0.1 * 3)
    st, _, _ = _limit_call(over, dt, nq)
    assert st == D.EINVAL
    assert b"maximum" in D.lib().difvm_last_error()


def test_noalloc_fp32_three_components_rejected(at_limit):
    exact, _ = at_limit
    st, _, _ = _limit_call(exact, torch.float32, 3)   # 25,165,824 bytes
    assert st == D.EINVAL
    st, _, _ = _limit_call(exact, torch.float32, 1)   # 8 MiB fits
    assert st == D.OK


def test_noalloc_coefficient_gradients_need_no_scratch(at_limit):
    _, over = at_limit
    # x_bar = NULL: no scratch is used, so a mesh over the limit is accepted
    st, _, Dbar = _limit_call(over, torch.float64, 3, with_xbar=False, coeff=True)
    assert st == D.OK, D.lib().difvm_last_error()
    assert float(Dbar.min()) == 3.0          # sum_c ybar_i x_i with x = ybar = 1


def test_noalloc_rejects_too_large_a_problem():
    # 750,000 cells x 3 components in FP64 need 18 MB of scratch: over the 16 MiB limit
    m = mg.kuhn_cube(50, 0.0, 0)
    dm = D.Mesh(m)
    x = torch.zeros(3, dm.nc, dtype=torch.float64, device="cuda")
    L = torch.zeros(dm.ni, dtype=torch.float64, device="cuda")
    Dg = torch.ones(dm.nc, dtype=torch.float64, device="cuda")
    xbar = torch.zeros_like(x)
    st = _call_noalloc(dm, D.F64, Dg, L, None, x, x, xbar, None, None, None)
    assert st == D.EINVAL
    assert b"maximum" in D.lib().difvm_last_error()
    # one component (6 MB) fits
    st = _call_noalloc(dm, D.F64, Dg, L, None, x[:1].contiguous(), x[:1].contiguous(),
                       xbar[:1].contiguous(), None, None, None)
    assert st == D.OK
