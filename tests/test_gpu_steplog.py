"""The per-step metrics log on the GPU: a few PISO steps of a small cavity, the
continuity error the log computes on the device against the same sum taken on
the host from the face flux, and the step records themselves."""
import io
import json

import numpy as np
import pytest

from paper_2603_15920_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_15920_b300 import difvm as D  # noqa: E402


def test_steplog_records_and_continuity():
    m = mg.shuffle(mg.kuhn_cube(8, 0.2, 61), 62)
    dm = D.Mesh(m)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    o = D.piso_opts(0.02, 0.05, 2, 3, solve_U=D.solve_opts(D.BICGSTAB, 1e-12, max_iter=2000),
                    solve_p=D.solve_opts(D.PCG, 1e-12, max_iter=2000, precond=D.PRECOND_AMG),
                    pref_cell=int(dm.cell_new_of_old[5]), nonorth_limit=0.5)
    pg = D.Piso(dm, D.F64, o)
    dt = torch.float64
    U = torch.zeros((3, dm.nc), dtype=dt, device="cuda")
    p = torch.zeros(dm.nc, dtype=dt, device="cuda")
    ub = torch.as_tensor(dm.to_bnd(Ub), dtype=dt, device="cuda").contiguous()
    pb = torch.zeros(dm.nb, dtype=dt, device="cuda")
    phi = D.difvm_flux_from_U(dm, U, ub)
    info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")
    buf = io.StringIO()
    log = D.StepLog(buf, mesh=dm, n_corr=2)
    recs = []
    for k in range(3):
        assert pg.step(U, p, phi, ub, pb, info=info)[0] == D.OK
        recs.append(log.log(k, info, phi=phi, t=0.05 * (k + 1)))
    assert [json.loads(x) for x in buf.getvalue().splitlines()] == recs
    for r in recs:
        assert r["status"] == D.OK and len(r["itU"]) == 3 and len(r["itp"]) == 2 and min(r["itp"]) > 0
    # the device sum against the host sum of the same flux (input numbering)
    f = dm.from_faces(phi.cpu().numpy())
    ni = m.n_internal
    div = (np.bincount(m.owner, f, m.n_cells) - np.bincount(m.neighbour, f[:ni], m.n_cells))
    empty = np.zeros(m.n_faces, bool)
    for pt, (s0, sz) in enumerate(zip(m.patch_start, m.patch_size)):
        if m.patch_type[pt] == mg.EMPTY:
            empty[s0:s0 + sz] = True
    assert not empty.any()
    a = np.abs(div).sum()
    assert abs(recs[-1]["continuity_abs"] - a) <= 1e-9 * np.abs(f).sum()
    # after the last corrector the flux is divergence-free to the solver tolerance
    assert recs[-1]["continuity_rel"] < 1e-8
