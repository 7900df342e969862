"""A mesh read from polyMesh files (geometry from the library's
``difvm_polymesh_geometry``) runs the PISO step on the GPU with the oracle's
step on the same mesh: a prism channel with inlet and outlet, 1e-9 per step."""
import numpy as np
import pytest

import oracle as O
from paper_2603_15920_b300 import meshgen as mg
from paper_2603_15920_b300 import polymesh as pm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_15920_b300 import difvm as D  # noqa: E402


def nrel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda").contiguous()


def host(t):
    return t.double().cpu().numpy()


def test_polymesh_case_piso_steps_match_oracle(tmp_path):
    src = mg.distorted_box(8, 0.05, 4, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET))
    d = str(tmp_path / "polyMesh")
    pm.write_polymesh(d, src)
    m = pm.load_mesh(d, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET))
    om, dm = O.OMesh.from_mesh(m), D.Mesh(m)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("x0") - m.n_internal] = 1.0
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    o = D.piso_opts(0.05, 0.02, 2, 3, solve_U=D.solve_opts(D.BICGSTAB, 1e-12, max_iter=2000),
                    solve_p=D.solve_opts(D.PCG, 1e-12, max_iter=20000), pref_cell=int(dm.cell_new_of_old[0]))
    h = D.Piso(dm, D.F64, o)
    worst = 0.0
    for _ in range(3):
        g = (cuda(dm.to_cells(U)), cuda(dm.to_cells(p)), cuda(dm.to_faces(phi)), cuda(dm.to_bnd(Ub)),
             cuda(dm.to_bnd(pb)))
        assert h.step(*g)[0] == D.OK
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, nu=0.05, dt=0.02, tolU=1e-12, tolp=1e-12)
        worst = max(worst, nrel(dm.from_cells(host(g[0])), U), nrel(dm.from_cells(host(g[1])), p),
                    nrel(dm.from_faces(host(g[2])), phi))
    assert worst < 1e-9, worst
