"""Parity at full size, in the configuration the benchmark times.

* The 64^3 Kuhn lid cavity (1,572,864 cells): one PISO step from rest with F32
  fields, the float-float multigrid pressure CG and the step captured as one
  CUDA graph, against one FP64 oracle step with tight solver tolerances (the
  1e-4 field bar of the mixed-precision path).
* The batched workload (64 lid cavities, n ~ U{8..48}, 15.8M cells, each
  side other than the lid a wall or, with probability 0.2, an opening): one
  graph-launched F32 step of the whole batch; the three smallest cases, the
  smallest case with an opening and the smallest closed one (pressure pinned),
  which the oracle steps in seconds, are checked one by one against the oracle
  run on each case alone (a case's result depends only on its own cells).

The oracle steps take about a minute on one host core.
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

NU, DT = 0.01, 0.002
NONORTH = 1            # explicit non-orthogonal correction in the momentum equation
FIELD_TOL = 1e-4       # mixed precision against the FP64 oracle (fields)


def nrel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def f32(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda").contiguous()


def host(t):
    return t.double().cpu().numpy()


def _oracle_step(m, Ub, pin):
    om = O.OMesh.from_mesh(m)
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    U, p, phi, _, _, info = O.piso_step(om, U, p, phi, Ub, pb, nu=NU, dt=DT, nonorth=NONORTH,
                                        tolU=1e-12, tolp=1e-12, pref_cell=pin)
    assert info["status"] == 0
    return U, p, phi


def test_kuhn64_cavity_graph_step_f32_matches_oracle():
    m = mg.kuhn_cube(64, 0.2, 0)
    dm = D.Mesh(m)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    pref = int(dm.cell_new_of_old[0])      # pressure pinned at input cell 0
    h = D.Piso(dm, D.F32, D.piso_opts(
        NU, DT, 2, NONORTH, solve_U=D.solve_opts(D.BICGSTAB, 1e-6, max_iter=1000, check_every=4),
        solve_p=D.solve_opts(D.PCG, 1e-10, max_iter=20000, check_every=4, refine_max=20, inner_tol=1e-4,
                             precond=D.PRECOND_AMG),
        pref_cell=pref))
    U = torch.zeros((3, dm.nc), dtype=torch.float32, device="cuda")
    p = torch.zeros(dm.nc, dtype=torch.float32, device="cuda")
    ub = f32(dm.to_bnd(Ub))
    pb = torch.zeros(dm.nb, dtype=torch.float32, device="cuda")
    phi = D.difvm_flux_from_U(dm, U, ub)
    gi = D.decode_piso_info(h.step_graph(U, p, phi, ub, pb))
    assert gi["status"] == D.OK and max(gi["itp"][:2]) <= 40
    Ur, pr, phir = _oracle_step(m, Ub, 0)
    assert nrel(dm.from_cells(host(U)), Ur) < FIELD_TOL
    assert nrel(dm.from_cells(host(p)), pr) < FIELD_TOL
    assert nrel(dm.from_faces(host(phi)), phir) < FIELD_TOL


def test_batched_64_cavities_graph_step_f32_sampled_cases_match_oracle():
    # the benchmark's batch: walls and openings drawn per case, lid U = (1, 0, 0)
    ms, u, cs, Ub_u, opens = mg.cavity_batch(64, 4, 0.2)
    assert 0 < opens.any(axis=1).sum() < 64          # both kinds of case occur
    dmu = D.Mesh(u, case_cell_start=cs)
    h = D.Piso(dmu, D.F32, D.piso_opts(
        NU, DT, 2, NONORTH, solve_U=D.solve_opts(D.BICGSTAB, 1e-6, max_iter=1000, check_every=4),
        solve_p=D.solve_opts(D.PCG, 1e-8, max_iter=20000, check_every=32, precond=D.PRECOND_AMG),
        pref_cell=0))
    U = torch.zeros((3, dmu.nc), dtype=torch.float32, device="cuda")
    p = torch.zeros(dmu.nc, dtype=torch.float32, device="cuda")
    ub = f32(dmu.to_bnd(Ub_u))
    pb = torch.zeros(dmu.nb, dtype=torch.float32, device="cuda")
    phi = D.difvm_flux_from_U(dmu, U, ub)
    gi = D.decode_piso_info(h.step_graph(U, p, phi, ub, pb))
    assert gi["status"] == D.OK
    Uu, pu = dmu.from_cells(host(U)), dmu.from_cells(host(p))
    order = np.argsort([m.n_cells for m in ms], kind="stable")
    sample = list(order[:3])
    sample += [k for k in order if opens[k].any() and k not in sample][:1]     # the smallest with an opening
    sample += [k for k in order if not opens[k].any() and k not in sample][:1]  # the smallest closed one
    for k in sample:
        m = ms[k]
        Ub = np.zeros((3, m.n_boundary))
        Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
        # the case's pinned cell (closed cases): its first cell in the internal numbering
        rel = dmu.cell_new_of_old[cs[k]:cs[k + 1]] - cs[k]
        pin = int(np.where(rel == 0)[0][0])
        Ur, pr, _ = _oracle_step(m, Ub, pin)
        e = nrel(Uu[:, cs[k]:cs[k + 1]], Ur), nrel(pu[cs[k]:cs[k + 1]], pr)
        assert max(e) < FIELD_TOL, (k, e)
