"""The differentiable pulsatile pipe with an RCR Windkessel outlet (Sec. 2.6.3,
Sec. 3.2.2), at full size on the GPU.

Mesh: straight cylinder R = 1, L = 10, O-H grid (16 x 16 core block, four outer
blocks of 16 x 8), 200 layers: 153,600 cells.  Inlet: parabolic profile scaled
so that the flux is Q(t) = 1 + 0.5 sin 2 pi t + 0.2 sin 4 pi t at t^{n+1};
outlet: RCR Windkessel (exact update); nu = 0.035; dt = 0.0025; 400 PISO steps
in FP64.  Loss: mean squared pressure misfit at 8 seeded probe cells over all
400 steps, against the trajectory of (R_p, C, R_d) = (0.15, 0.7, 1.3).  The
gradient at (0.1, 1, 1) comes from the hand-written step adjoints chained in
reverse over the trajectory with the state kept every 20 steps; it must equal
central differences of the GPU forward to 1e-4 (relative).  The same chain is
pinned against the oracle's forward on a small pipe in
tests/test_oracle_adjoint.py.
"""
import time

import numpy as np
import pytest

from paper_2603_15920_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2603_15920_b300 import difvm as D  # noqa: E402

STEPS, DT, NU, CKPT = 400, 0.0025, 0.035, 20


class Pipe:
    def __init__(self, n_core=16, n_outer=8, n_layers=200, L=10.0, n_probes=8):
        m = mg.pipe_ohgrid(n_core, n_outer, n_layers, L=L)
        self.m, self.dm = m, D.Mesh(m)
        dm = self.dm
        ub = mg.pipe_inflow(m)          # parabolic, along +z, unit flux
        self.shape = torch.as_tensor(dm.to_bnd(ub), dtype=torch.float64, device="cuda").contiguous()
        probes = np.random.default_rng(11).choice(m.n_cells, size=n_probes, replace=False)
        self.probes = torch.as_tensor(dm.cell_new_of_old[probes], dtype=torch.long, device="cuda")
        self.out = m.patch_index("outlet")
        tol = 1e-12
        self.h = D.Piso(dm, D.F64, D.piso_opts(
            NU, DT, 2, 1, solve_U=D.solve_opts(D.BICGSTAB, tol, max_iter=2000, check_every=4),
            solve_p=D.solve_opts(D.PCG, tol, max_iter=5000, check_every=4, precond=D.PRECOND_AMG),
            wk_scheme=D.WK_EXACT, wk_patch=[self.out]))

    def boundary(self, j, Ub):
        torch.mul(self.shape, mg.pulsatile_flow((j + 1) * DT), out=Ub)   # values at t^{n+1}

    def state(self, theta):
        dm = self.dm
        U = torch.zeros(3, dm.nc, dtype=torch.float64, device="cuda")
        p = torch.zeros(dm.nc, dtype=torch.float64, device="cuda")
        Ub = self.shape.clone()
        self.boundary(-1, Ub)
        phi = D.difvm_flux_from_U(dm, U, Ub)
        pb = torch.zeros(dm.nb, dtype=torch.float64, device="cuda")
        wk = torch.tensor([theta[0], theta[1], theta[2], 0.0], dtype=torch.float64, device="cuda")
        return [U, p, phi, Ub, pb], wk

    def forward(self, theta):
        """Probe pressures of every step [STEPS, probes] (graph-launched steps)."""
        (U, p, phi, Ub, pb), wk = self.state(theta)
        info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")
        P = torch.empty(STEPS, self.probes.numel(), dtype=torch.float64, device="cuda")
        for j in range(STEPS):
            self.boundary(j, Ub)
            self.h.step_graph(U, p, phi, Ub, pb, wk, info=info)
            P[j] = p[self.probes]
        assert D.decode_piso_info(info)["status"] == D.OK
        return P

    def loss(self, theta, target):
        return float(((self.forward(theta) - target) ** 2).mean())

    def gradient(self, theta, target):
        st, wk = self.state(theta)
        N = float(target.numel())

        def seeds(j, U, p, phi, pb, w):
            g = torch.zeros_like(p)
            g[self.probes] = 2.0 * (p[self.probes] - target[j]) / N
            return None, g, None, None, None
        r = D.trajectory_adjoint(self.h, st, STEPS, self.boundary, seeds, wk=wk, checkpoint_every=CKPT)
        assert r["status"] == D.OK
        return np.array([float(r["Rp"][0]), float(r["C"][0]), float(r["Rd"][0])])


@pytest.fixture(scope="module")
def pipe():
    return Pipe()


def test_pipe_mesh_is_the_survey_size(pipe):
    assert pipe.dm.nc == 153600


def test_pulsatile_pipe_windkessel_gradient_matches_central_differences(pipe):
    target = pipe.forward((0.15, 0.7, 1.3))
    theta = np.array([0.1, 1.0, 1.0])
    t0 = time.perf_counter()
    g = pipe.gradient(theta, target)
    t_adj = time.perf_counter() - t0
    for i in range(3):
        h = 1e-5 * theta[i]
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (pipe.loss(tp, target) - pipe.loss(tm, target)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-4 * abs(fd), (i, g[i], fd, t_adj)
