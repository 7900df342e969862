"""The allocation-free LDU-apply adjoint against the regular one.

difvm_laplacian_apply_bwd_noalloc serves callers that cannot allocate device
memory (their memory belongs to another runtime's pool, or they run a loop
where cudaMalloc's device-wide synchronisation is not acceptable): it forms
A^T y_bar in a scratch array built into the library instead of a buffer the
caller passes.  Its outputs must equal those of difvm_laplacian_apply_bwd,
on two calls in a row (the second call reuses the scratch the first one left
behind).  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2603_15920_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_15920_b300 import difvm as D  # noqa: E402

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def nrel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def mesh():
    return D.Mesh(mg.shuffle(mg.kuhn_cube(8, 0.2, 4), 6))


def _call_noalloc(dm, prec, Dg, L, U, x, ybar, xbar, Dbar, Lbar, Ubar):
    p = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    return D.lib().difvm_laplacian_apply_bwd_noalloc(
        dm.h, prec, p(Dg), p(L), p(U), p(x), p(ybar), x.shape[0], p(xbar), p(Dbar), p(Lbar), p(Ubar),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("sym", [False, True])
def test_noalloc_matches_regular_adjoint_twice(mesh, dt, sym):
    dm = mesh
    prec = D.F64 if dt == torch.float64 else D.F32
    rng = np.random.default_rng(11)
    for call in range(2):                   # two calls in a row, different inputs
        cu = lambda a: torch.as_tensor(a, dtype=dt, device="cuda").contiguous()
        Dg = cu(rng.standard_normal(dm.nc))
        L = cu(rng.standard_normal(dm.ni))
        U = None if sym else cu(rng.standard_normal(dm.ni))
        x = cu(rng.standard_normal((3, dm.nc)))
        ybar = cu(rng.standard_normal((3, dm.nc)))
        start = cu(rng.standard_normal((3, dm.nc)))      # outputs accumulate
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
                assert nrel(g, r) < TOL[dt], (call, nrel(g, r))


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
