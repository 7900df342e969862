#!/usr/bin/env python3
"""Benchmark: PISO steps/s on the 1.6M-cell Kuhn-tet lid-driven cavity.

Workload (one "step" = one PISO time step, i.e. one pass of the whole hot
path: Gauss gradients, momentum assembly with upwind convection and
over-relaxed diffusion, BiCGStab momentum solve on the matrix-free LDU
operator, two pressure correctors with the graph-Laplacian assembly, PCG with
FP64 iterative refinement, Rhie-Chow flux and velocity correction):
  mesh   Kuhn tetrahedra of a 64^3 hex grid of the unit cube, interior vertices
         jittered by U(-0.2h, 0.2h) (seed 0), RCM-renumbered: 1,572,864 cells,
         3,170,304 faces (synthetic; no dataset exists for it)
  flow   lid-driven cavity, lid u = (1,0,0) on y = 1, Re = 100 (nu = 0.01),
         dt = 0.002, two correctors, pressure pinned at one cell, explicit
         over-relaxed non-orthogonal correction in the momentum equation, the
         pressure Laplacian orthogonal (its lagged correction diverges on these
         jittered tetrahedra; at dt = 0.004 two correctors do not contain the
         PISO splitting error on this mesh)
  solve  pressure PCG to ||r|| <= 1e-10 ||b|| in FP64 refinement residuals;
         momentum BiCGStab to 1e-6 (F32) / 1e-10 (F64)
  prec   headline: FP32 fields and operators, FP64 dots + pressure refinement;
         the plain FP64 run is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun, one process per GPU): every rank runs its own replica of the
cavity ("replicas only": the path has no exchange step); value = steps of all
ranks / max-over-ranks time.  The working set (about 0.9 GB in F32) is far
larger than the 126 MB L2, so no L2 flush is needed between steps.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PISO steps/s & fwd+adjoint/fwd time at 1.6M-cell tet mesh; face-op HBM GB/s %"
WORKLOAD = "kuhn64_cavity_re100"
N_KUHN, JITTER, SEED = 64, 0.2, 0
NU, DT = 0.01, 0.002
# the batched cavities (64 cases, n ~ U{8..48}) keep these whatever --mesh is
BATCH_JITTER, BATCH_NU = JITTER, NU
# --mesh 128: the large mixed-precision cavity (12.6M cells, jitter 0.15h, Re 400).
# At jitter 0.2h and Re 100 the 128^3 cavity diverges within a few steps in FP32 and
# FP64 alike (nu dt / h^2 = 0.33 against 0.08 at 64^3: the explicit non-orthogonal
# momentum correction is unstable there); at Re 400 nu dt / h^2 is 0.08 again.
LARGE = {128: ("kuhn128_cavity_re400", 0.15, 0.0025)}
# Explicit over-relaxed non-orthogonal correction in the momentum equation only
# (bit 0); the lagged correction of the pressure Laplacian (bit 1) diverges on
# these jittered tetrahedra for every setting tried.  dt = 0.002: with two
# correctors the PISO splitting error grows at dt = 0.004 on this mesh.
NONORTH = 1
CKPT = 5          # checkpoint interval of the checkpointed forward + adjoint run
BINOM_SLOTS = 4   # stored states besides the initial one in the binomial-schedule run


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of x over the ranks (x itself on one rank): N independent
    replicas are timed to the slowest one."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ms_per_step, world):
    """Whole-job steps/s of `world` replicas, each taking ms_per_step (the
    slowest rank's time)."""
    return world * 1e3 / ms_per_step


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def make_mesh(n=None):
    from paper_2603_15920_b300 import meshgen as mg
    return mg.kuhn_cube(n or N_KUHN, JITTER, SEED)


def lid_bc(m):
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    return Ub


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------- CPU baseline
def run_batched(D, torch, K=20, W=3, n_cases=64, seed=4, precond=None, f64=True, adjoint=True):
    """Batched form: the meshgen.cavity_batch cavities as one disjoint-union mesh, Re =
    100 (nu = 0.01), dt = 0.002 for every case, FP32 fields with FP64 dots
    (pressure CG per case to 1e-8), per-case solver scalars, every step one CUDA
    graph; beside it the same batch in plain FP64 (pressure to 1e-10) and the
    FP32 fields' difference from it after the same steps; and forward + adjoint
    of the total kinetic energy over the K steps.  Pressure: CG with one
    multigrid V-cycle over the union per iteration (default) or Jacobi."""
    from paper_2603_15920_b300 import meshgen as mg
    precond = D.PRECOND_AMG if precond is None else precond
    ms, u, cs, Ub_h, opens = mg.cavity_batch(n_cases, seed, BATCH_JITTER)
    dm = D.Mesh(u, case_cell_start=cs)
    ce = 32 if precond == D.PRECOND_JACOBI else 4

    def handle(prec):
        tolp = 1e-8 if prec == D.F32 else 1e-10
        o = D.piso_opts(BATCH_NU, DT, 2, NONORTH,
                        solve_U=D.solve_opts(D.BICGSTAB, 1e-6 if prec == D.F32 else 1e-10, max_iter=1000,
                                             check_every=4),
                        solve_p=D.solve_opts(D.PCG, tolp, max_iter=20000, check_every=ce, precond=precond),
                        pref_cell=0)
        return D.Piso(dm, prec, o)

    def state(dt_):
        U = torch.zeros((3, dm.nc), dtype=dt_, device="cuda")
        p = torch.zeros(dm.nc, dtype=dt_, device="cuda")
        ub = torch.as_tensor(dm.to_bnd(Ub_h), dtype=dt_, device="cuda").contiguous()
        pb = torch.zeros(dm.nb, dtype=dt_, device="cuda")
        return [U, p, D.difvm_flux_from_U(dm, U, ub), ub, pb]

    info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")

    def timed(prec):
        h, st = handle(prec), state(torch.float32 if prec == D.F32 else torch.float64)
        for _ in range(W):
            h.step_graph(*st, info=info)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            h.step_graph(*st, info=info)
        e1.record()
        torch.cuda.synchronize()
        return h, st, e0.elapsed_time(e1) / K, D.decode_piso_info(info)

    h, s32, ms32, gi = timed(D.F32)
    out = {"workload": f"{n_cases} Kuhn lid cavities (lid U = (1,0,0)), n ~ U{{8..48}}, jitter {BATCH_JITTER}, "
                       f"each other side a wall with probability 0.8, else an opening (p = 0), seed {seed}",
           "cells": int(dm.nc), "cases": n_cases, "cases_with_opening": int(opens.any(axis=1).sum()),
           "value": 1e3 / ms32, "unit": "steps/s", "ms_per_step": ms32, "cell_steps_per_s": dm.nc * 1e3 / ms32,
           "steps": K, "warmup": W,
           "api": "difvm_piso_step_graph on a batched mesh (per-case Krylov scalars)",
           "pressure_solver": ("CG + one multigrid V-cycle over the union per iteration"
                               if precond == D.PRECOND_AMG else "CG + Jacobi"),
           "precision": "f32 fields, f64 dots, pressure tol 1e-8 per case",
           "status": int(gi["status"]), "pressure_iters_max_over_cases": gi["itp"][:2]}
    if f64:
        h64, s64, ms64, gi64 = timed(D.F64)

        def nrel(a, b):
            a, b = a.double(), b.double()
            return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))
        out["f64"] = {"value": 1e3 / ms64, "unit": "steps/s", "ms_per_step": ms64, "status": int(gi64["status"]),
                      "pressure_iters_max_over_cases": gi64["itp"][:2],
                      "f32_field_err_vs_f64": {"steps": W + K, "U": nrel(s32[0], s64[0]),
                                               "p": nrel(s32[1], s64[1]), "phi": nrel(s32[2], s64[2])},
                      "f32_over_f64_speed": ms64 / ms32}
        del h64, s64
    # the multigrid launch shapes first-use timing picked, and the same batch with the
    # default shapes (difvm_mesh_autotune mode 0 restores them; a new handle captures
    # a new graph)
    out["tuned_launch_shapes"] = {f"{k[0]}.{k[1]}.{k[2]}": v for k, v in D.difvm_mesh_tuning(dm).items()
                                  if k[0] in (5, 6)}
    if f64 and adjoint:
        D.difvm_mesh_autotune(dm, 0)
        hf, sf, msf, gif = timed(D.F32)
        out["default_launch_shapes"] = {"value": 1e3 / msf, "unit": "steps/s", "ms_per_step": msf,
                                        "status": int(gif["status"]),
                                        "tuned_over_default_speed": msf / ms32}
        D.difvm_mesh_autotune(dm, 2)     # tuned again for the runs that follow
        del hf, sf
    if adjoint:
        # forward + adjoint of the total kinetic energy after K steps (every step taped)
        V = torch.as_tensor(dm.to_cells(u.V), dtype=torch.float32, device="cuda")

        def ke_grad(U_, p_, phi_, pb_, wk_):
            return (V * U_).contiguous(), torch.zeros_like(p_), torch.zeros_like(phi_), None, None
        tapes = [h.new_tape("cuda") for _ in range(K)]
        base = [t.clone() for t in s32]
        D.simulate_adjoint(h, [t.clone() for t in base], 1, ke_grad, tapes=tapes)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        adj = D.simulate_adjoint(h, [t.clone() for t in base], K, ke_grad, tapes=tapes)
        a1.record()
        torch.cuda.synchronize()
        fa = a0.elapsed_time(a1) / K
        out.update({"fwd_adj_ms_per_step": fa, "fwd_adjoint_over_fwd": fa / ms32,
                    "fwd_adjoint_note": "forward steps of the adjoint run are recorded host-loop steps; "
                                        f"{K} steps taped", "adjoint_status": int(adj["status"])})
        del tapes
    return out


def run_large(D, torch, K=10, W=3, n=128):
    """The large mixed-precision case: lid-driven cavity on Kuhn tetrahedra of a
    128^3 hex grid (12,582,912 cells), jitter 0.15h, Re 400 (nu = 0.0025), dt
    0.002, two correctors; the FP32 step (FP64 dots, float-float pressure CG to
    1e-10 around the FP32 V-cycle) and the plain FP64 step, each K graph steps
    after W from rest; the FP32 fields against the FP64 ones after the same
    steps; and forward + adjoint of the kinetic energy over K steps with the
    state kept every 5 steps (segments re-run with tapes)."""
    name, jitter, nu = LARGE[n]
    from paper_2603_15920_b300 import meshgen as mg
    m = mg.kuhn_cube(n, jitter, SEED)
    dm = D.Mesh(m)
    Ub_h = lid_bc(m)
    pref = int(dm.cell_new_of_old[0])
    info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")

    def handle(prec):
        if prec == D.F32:
            sp = D.solve_opts(D.PCG, 1e-10, max_iter=20000, check_every=4, refine_max=20, inner_tol=1e-4,
                              precond=D.PRECOND_AMG)
        else:
            sp = D.solve_opts(D.PCG, 1e-10, max_iter=20000, check_every=4, precond=D.PRECOND_AMG)
        return D.Piso(dm, prec, D.piso_opts(
            nu, DT, 2, NONORTH, solve_U=D.solve_opts(D.BICGSTAB, 1e-6 if prec == D.F32 else 1e-10,
                                                     max_iter=1000, check_every=4),
            solve_p=sp, pref_cell=pref))

    def state(dt_):
        U = torch.zeros(3, dm.nc, dtype=dt_, device="cuda")
        p = torch.zeros(dm.nc, dtype=dt_, device="cuda")
        Ub = torch.as_tensor(dm.to_bnd(Ub_h), dtype=dt_, device="cuda").contiguous()
        pb = torch.zeros(dm.nb, dtype=dt_, device="cuda")
        return [U, p, D.difvm_flux_from_U(dm, U, Ub), Ub, pb]

    def run(prec):
        h, st = handle(prec), state(torch.float32 if prec == D.F32 else torch.float64)
        for _ in range(W):
            h.step_graph(*st, info=info)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            h.step_graph(*st, info=info)
        e1.record()
        torch.cuda.synchronize()
        return h, st, e0.elapsed_time(e1) / K, D.decode_piso_info(info)

    h32, s32, ms32, gi32 = run(D.F32)
    h64, s64, ms64, gi64 = run(D.F64)

    def nrel(a, b):
        a, b = a.double(), b.double()
        return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))
    err = {"steps": W + K, "U": nrel(s32[0], s64[0]), "p": nrel(s32[1], s64[1]), "phi": nrel(s32[2], s64[2])}
    del h64, s64
    V = torch.as_tensor(dm.to_cells(m.V), dtype=torch.float32, device="cuda")

    def ke_grad(U, p, phi, pb, wk):
        return (V * U).contiguous(), torch.zeros_like(p), torch.zeros_like(phi), None, None
    ck = 5
    tapes = [h32.new_tape("cuda") for _ in range(ck)]
    base = [t.clone() for t in s32]
    D.simulate_adjoint(h32, [t.clone() for t in base], 1, ke_grad, tapes=tapes)
    s1 = [t.clone() for t in base]
    torch.cuda.synchronize()
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    a.record()
    for _ in range(K):
        h32.step(*s1, info=info)
    b.record()
    adj = D.simulate_adjoint(h32, [t.clone() for t in base], K, ke_grad, checkpoint_every=ck, tapes=tapes)
    c.record()
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info()
    fwd, fa = a.elapsed_time(b), b.elapsed_time(c)
    return {"workload": name, "mesh": f"kuhn{n}^3 jitter {jitter} seed {SEED} RCM", "cells": dm.nc,
            "faces": dm.nf, "nu": nu, "dt": DT,
            "value": 1e3 / ms32, "unit": "steps/s", "ms_per_step": ms32, "steps": K, "warmup": W,
            "status": int(gi32["status"]), "pressure_iters_last_step": gi32["itp"][:2],
            "f64": {"value": 1e3 / ms64, "ms_per_step": ms64, "status": int(gi64["status"]),
                    "pressure_iters_last_step": gi64["itp"][:2]},
            "f32_field_err_vs_f64": err, "f32_over_f64_speed": ms64 / ms32,
            "fwd_adjoint_over_fwd": {"value": fa / fwd, "steps": K, "checkpoint_every": ck,
                                     "fwd_ms_per_step": fwd / K, "fwd_adj_ms_per_step": fa / K,
                                     "status": int(adj["status"]),
                                     "forward": "host-loop steps (difvm_piso_step) in both"},
            "device_memory_in_use_GB": round((total - free) / 1e9, 1)}


def run_pipe(D, torch, steps=400, ckpt=20):
    """The differentiable pulsatile pipe (the survey's config 3): O-H pipe R = 1,
    L = 10, 153,600 cells; parabolic inflow Q(t) = 1 + 0.5 sin 2 pi t + 0.2 sin
    4 pi t; RCR Windkessel outlet (R_p, C, R_d) = (0.1, 1, 1), exact update; nu
    0.035, dt 0.0025, FP64, 400 steps.  Loss: pressure misfit at 8 probes over
    all steps against the (0.15, 0.7, 1.3) trajectory; its gradient by the
    step adjoints chained over the trajectory, the state kept every 20 steps
    (tests/test_gpu_pipe.py checks it against central differences at 1e-4)."""
    from paper_2603_15920_b300 import meshgen as mg
    dt, nu = 0.0025, 0.035
    m = mg.pipe_ohgrid(16, 8, 200, L=10.0)
    dm = D.Mesh(m)
    shape = torch.as_tensor(dm.to_bnd(mg.pipe_inflow(m)), dtype=torch.float64, device="cuda").contiguous()
    probes = np.random.default_rng(11).choice(m.n_cells, size=8, replace=False)
    probes = torch.as_tensor(dm.cell_new_of_old[probes], dtype=torch.long, device="cuda")
    h = D.Piso(dm, D.F64, D.piso_opts(
        nu, dt, 2, 1, solve_U=D.solve_opts(D.BICGSTAB, 1e-12, max_iter=2000, check_every=4),
        solve_p=D.solve_opts(D.PCG, 1e-12, max_iter=5000, check_every=4, precond=D.PRECOND_AMG),
        wk_scheme=D.WK_EXACT, wk_patch=[m.patch_index("outlet")]))
    info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")

    def boundary(j, Ub):
        torch.mul(shape, mg.pulsatile_flow((j + 1) * dt), out=Ub)

    def state(theta):
        U = torch.zeros(3, dm.nc, dtype=torch.float64, device="cuda")
        p = torch.zeros(dm.nc, dtype=torch.float64, device="cuda")
        Ub = shape.clone()
        boundary(-1, Ub)
        pb = torch.zeros(dm.nb, dtype=torch.float64, device="cuda")
        wk = torch.tensor(list(theta) + [0.0], dtype=torch.float64, device="cuda")
        return [U, p, D.difvm_flux_from_U(dm, U, Ub), Ub, pb], wk

    def forward(theta):
        (U, p, phi, Ub, pb), wk = state(theta)
        P = torch.empty(steps, 8, dtype=torch.float64, device="cuda")
        for j in range(steps):
            boundary(j, Ub)
            h.step_graph(U, p, phi, Ub, pb, wk, info=info)
            P[j] = p[probes]
        return P

    target = forward((0.15, 0.7, 1.3))
    torch.cuda.synchronize()
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    a.record()
    P = forward((0.1, 1.0, 1.0))
    b.record()
    torch.cuda.synchronize()
    loss = float(((P - target) ** 2).mean())
    st, wk = state((0.1, 1.0, 1.0))
    N = float(target.numel())

    def seeds(j, U, p, phi, pb, w):
        g = torch.zeros_like(p)
        g[probes] = 2.0 * (p[probes] - target[j]) / N
        return None, g, None, None, None
    torch.cuda.synchronize()
    b2 = torch.cuda.Event(enable_timing=True)
    b2.record()
    r = D.trajectory_adjoint(h, st, steps, boundary, seeds, wk=wk, checkpoint_every=ckpt)
    c.record()
    torch.cuda.synchronize()
    fwd, fa = a.elapsed_time(b), b2.elapsed_time(c)
    return {"workload": "pulsatile O-H pipe with an RCR Windkessel outlet, 400 steps", "cells": dm.nc,
            "precision": "f64", "value": steps * 1e3 / fwd, "unit": "steps/s", "ms_per_step": fwd / steps,
            "api": "difvm_piso_step_graph per step, inlet values updated in place",
            "loss": loss, "dL_dRp_C_Rd": [float(r["Rp"][0]), float(r["C"][0]), float(r["Rd"][0])],
            "fwd_adjoint_over_fwd": {"value": fa / fwd, "checkpoint_every": ckpt, "fwd_adj_ms": fa,
                                     "forward": "host-loop steps in the adjoint run"},
            "status": int(r["status"])}


def run_face_ops(D, torch, m, dm, peak, reps=20, copies=4):
    """The face operators on the bench mesh in FP32 and FP64 (Sec. 2.3-2.4: Gauss
    gradient, convective divergence, diffusive flux, LDU apply).  `copies`
    device copies of the mesh, each with its own inputs, are used in turn by
    `reps` back-to-back launches between two CUDA events, so every launch finds
    its geometry and fields out of L2 (the other copies' 3 x 100-250 MB passed
    through it since) and the launch latency overlaps the previous kernel.
    Algorithmic bytes: each face array read once (int32 owner/neighbour + the
    geometry the operator needs), each input cell array read once, each output
    written once; gathers hit cache."""
    nc, ni, nf, nb = dm.nc, dm.ni, dm.nf, dm.nb
    nhf = 2 * ni + nb          # half-faces: every internal face seen from both cells
    # FP64 work per launch: FP64 add / mul / fma instructions of each kernel, per
    # internal half-face (boundary half-faces are ~1% of the total and counted
    # alike) and per cell, read off the kernels' arithmetic
    fp64_ops = {"grad_gauss_scalar": (7, 3), "grad_gauss_vector": (19, 9), "div_flux_upwind_3": (6, 0),
                "div_flux_linear_3": (13, 0), "laplacian_apply_sym_1": (1, 1),
                "laplacian_apply_asym_3": (3, 3), "laplacian_nonorth_1": (15, 0)}
    dms = [dm] + [D.Mesh(m, device=torch.cuda.current_device()) for _ in range(copies - 1)]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    res = {}
    for prec, dt, v in ((D.F32, torch.float32, 4), (D.F64, torch.float64, 8)):
        def rn(*shape):
            return torch.randn(*shape, generator=gen, device="cuda", dtype=dt)

        def ops_of(d):
            phi, phib, U, Ub, mf = rn(1, nc), rn(1, nb), rn(3, nc), rn(3, nb), rn(nf)
            Dg, L, Uu, x1, x3 = rn(nc).abs() + 10.0, rn(ni), rn(ni), rn(1, nc), rn(3, nc)
            g1 = torch.empty(1, 3, nc, dtype=dt, device="cuda")
            g3 = torch.empty(3, 3, nc, dtype=dt, device="cuda")
            o1, o3 = torch.empty(1, nc, dtype=dt, device="cuda"), torch.empty(3, nc, dtype=dt, device="cuda")
            gp = D.difvm_grad_gauss(d, D.BC_ALL_FIXED, phi, phib)
            return {
                "grad_gauss_scalar": (lambda: D.difvm_grad_gauss(d, D.BC_PRESSURE, phi, phib, grad=g1),
                                      nf * (8 + 4 * v) + nc * 5 * v),
                "grad_gauss_vector": (lambda: D.difvm_grad_gauss(d, D.BC_VELOCITY, U, Ub, grad=g3),
                                      nf * (8 + 4 * v) + nc * 13 * v),
                "div_flux_upwind_3": (lambda: D.difvm_div_flux(d, D.DIV_UPWIND, D.BC_VELOCITY, mf, U, Ub, out=o3),
                                      nf * (8 + v) + nc * 6 * v),
                "div_flux_linear_3": (lambda: D.difvm_div_flux(d, D.DIV_LINEAR, D.BC_VELOCITY, mf, U, Ub, out=o3),
                                      nf * (8 + 2 * v) + nc * 6 * v),
                "laplacian_apply_sym_1": (lambda: D.difvm_laplacian_apply(d, Dg, L, None, x1, y=o1),
                                          nf * (8 + v) + nc * 3 * v),
                "laplacian_apply_asym_3": (lambda: D.difvm_laplacian_apply(d, Dg, L, Uu, x3, y=o3),
                                           nf * (8 + 2 * v) + nc * 7 * v),
                "laplacian_nonorth_1": (lambda: D.difvm_laplacian(d, D.BC_ALL_FIXED, 1.0, phi, phib, grad=gp,
                                                                  out=o1),
                                        nf * (8 + 5 * v) + nc * 5 * v),
            }
        per_copy = [ops_of(d) for d in dms]
        key = "f32" if prec == D.F32 else "f64"

        def time_op(fns):
            for f in fns:
                f()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for r in range(reps):
                fns[r % copies]()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        for name in per_copy[0]:
            fns = [oc[name][0] for oc in per_copy]
            nbytes = per_copy[0][name][1]
            t_default = None
            if prec == D.F32:
                # the default launch variant, then the one first-use timing keeps
                for d in dms:
                    D.difvm_mesh_autotune(d, 0)
                t_default = time_op(fns)
                for d in dms:
                    D.difvm_mesh_autotune(d, 1)
            t = time_op(fns)
            gbs = nbytes / (t * 1e-3) / 1e9
            e = {"us": round(t * 1e3, 2), "alg_MB": round(nbytes / 1e6, 1),
                 "GB/s": round(gbs, 1), "frac": round(gbs / peak, 3),
                 "frac_of_8TBs": round(gbs / 8000.0, 3)}
            if t_default is not None:
                e["us_default_variant"] = round(t_default * 1e3, 2)
            else:
                # FP64: the roofline is the slower of HBM and the FP64 pipe
                # (1.25 TFLOP/s dense = 0.625e12 fma instructions/s, every FP64
                # add / mul / fma taking one issue slot)
                ph, pc = fp64_ops[name]
                ops = ph * nhf + pc * nc
                t_alu, t_hbm = ops / 0.625e12, nbytes / (peak * 1e9)
                e.update({"fp64_ops": int(ops), "t_alu_us": round(t_alu * 1e6, 2),
                          "t_hbm_us": round(t_hbm * 1e6, 2), "bound": "alu" if t_alu > t_hbm else "hbm",
                          "frac_of_bound": round(max(t_alu, t_hbm) / (t * 1e-3), 3)})
            res.setdefault(name, {})[key] = e
        if prec == D.F32:
            res["_tuned_variants"] = {f"{k[0]}.{k[1]}.{k[2]}": v for k, v in D.difvm_mesh_tuning(dms[0]).items()}
        del per_copy
    del dms[1:]
    fr = [res[k]["f32"]["frac"] for k in res if not k.startswith("_")]
    return {"unit": "GB/s (algorithmic)", "peak": peak, "reps": reps, "ops": res,
            "f32_frac_median": float(np.median(fr)), "f32_frac_min": float(min(fr)),
            "method": f"{reps} back-to-back launches rotating over {copies} device copies of the mesh and "
                      "its inputs (each launch L2-cold), between two CUDA events"}


def cpu_oracle_step_rate(m, steps=1, warm_steps=0):
    """The FP64 CPU oracle (single thread, as it stands) on the same cavity.
    Returns (steps/s, seconds, sample description)."""
    import oracle as O
    om = O.OMesh.from_mesh(m)
    Ub = lid_bc(m)
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    kw = dict(nu=NU, dt=DT, tolU=1e-10, tolp=1e-10, pref_cell=0, nonorth=NONORTH)
    for _ in range(warm_steps):
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, **kw)
    t = time.perf_counter()
    for _ in range(steps):
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, **kw)
    dt = time.perf_counter() - t
    return steps / dt, dt


def reference_arm(args):
    """--impl reference: the oracle timed on the host cores, same metric/unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    m = make_mesh()
    # each step of this arm is one full oracle PISO step of the cavity
    import oracle as O
    om = O.OMesh.from_mesh(m)
    Ub = lid_bc(m)
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    phi = O.flux_from_U(om, U, Ub)
    kw = dict(nu=NU, dt=DT, tolU=1e-10, tolp=1e-10, pref_cell=0, nonorth=NONORTH)
    W, K = min(args.warmup, 1), min(args.steps, 2)
    for _ in range(W):
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, **kw)
    t = time.perf_counter()
    for _ in range(K):
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, **kw)
    el = time.perf_counter() - t
    v = K / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": 1e3 * el / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mesh": f"kuhn{N_KUHN}^3 jitter {JITTER} seed {SEED}",
                   "cells": m.n_cells, "faces": m.n_faces, "nu": NU, "dt": DT},
        "cpu_baseline": {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{K} full oracle PISO steps of the cavity after {W} warm-up step(s) "
                                   f"(requested --steps {args.steps} --warmup {args.warmup}, capped "
                                   "to keep the run within minutes)"},
        "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2603_15920_b300 import difvm as D
    global WORKLOAD, JITTER, NU
    if args.mesh in LARGE:
        WORKLOAD, JITTER, NU = LARGE[args.mesh]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    m = make_mesh(args.mesh)
    dm = D.Mesh(m, device=local)
    if args.no_autotune:     # profiling runs: the default launch shapes, no first-use timing launches
        D.difvm_mesh_autotune(dm, 0)
    if args.face_ops_only:   # profiling runs of the face operators alone
        print(json.dumps(run_face_ops(D, torch, m, dm, measured_peaks()[0])), flush=True)
        return 0
    if args.face_ops_launches:
        # a fixed launch sequence for ncu captures: the default launch variants (no
        # first-use timing), one gradient of the pressure-class field, then each F32
        # operator 5 times in the order of the face-op table
        D.difvm_mesh_autotune(dm, 0)
        g = torch.Generator(device="cuda")
        g.manual_seed(7)
        rn = lambda *sh: torch.randn(*sh, generator=g, device="cuda")
        nc, ni, nf, nb = dm.nc, dm.ni, dm.nf, dm.nb
        phi, phib, U, Ub, mf = rn(1, nc), rn(1, nb), rn(3, nc), rn(3, nb), rn(nf)
        Dg, L, Uu, x1, x3 = rn(nc).abs() + 10.0, rn(ni), rn(ni), rn(1, nc), rn(3, nc)
        gp = D.difvm_grad_gauss(dm, D.BC_ALL_FIXED, phi, phib)
        ops = [lambda: D.difvm_grad_gauss(dm, D.BC_PRESSURE, phi, phib),
               lambda: D.difvm_grad_gauss(dm, D.BC_VELOCITY, U, Ub),
               lambda: D.difvm_div_flux(dm, D.DIV_UPWIND, D.BC_VELOCITY, mf, U, Ub),
               lambda: D.difvm_div_flux(dm, D.DIV_LINEAR, D.BC_VELOCITY, mf, U, Ub),
               lambda: D.difvm_laplacian_apply(dm, Dg, L, None, x1),
               lambda: D.difvm_laplacian_apply(dm, Dg, L, Uu, x3),
               lambda: D.difvm_laplacian(dm, D.BC_ALL_FIXED, 1.0, phi, phib, grad=gp)]
        for f in ops:
            for _ in range(5):
                f()
        torch.cuda.synchronize()
        print(json.dumps({"face_op_launches": 5 * len(ops) + 1}), flush=True)
        return 0
    if args.batch_only:      # the batched 64-case form alone
        print(json.dumps(run_batched(D, torch, K=args.steps,
                                     precond=D.PRECOND_JACOBI if args.batch_jacobi else None)), flush=True)
        return 0
    # the face operators first, each timed on a fresh mesh before any solver runs
    face_ops = None if args.only_f32 else run_face_ops(D, torch, m, dm, measured_peaks()[0])
    if args.no_autotune:
        D.difvm_mesh_autotune(dm, 0)
    Ub_h = lid_bc(m)
    pref = int(dm.cell_new_of_old[0])

    def new_state(dt_):
        U = torch.zeros(3, dm.nc, dtype=dt_, device="cuda")
        p = torch.zeros(dm.nc, dtype=dt_, device="cuda")
        Ub = torch.as_tensor(dm.to_bnd(Ub_h), dtype=dt_, device="cuda").contiguous()
        pb = torch.zeros(dm.nb, dtype=dt_, device="cuda")
        phi = D.difvm_flux_from_U(dm, U, Ub)
        return [U, p, phi, Ub, pb]

    def piso(prec, precond=D.PRECOND_AMG, conv=D.CONV_UPWIND, time_scheme=D.TIME_BE, check_every=None,
             precond_U=D.PRECOND_JACOBI):
        # pressure: CG preconditioned by one multigrid V-cycle (or Jacobi); the
        # Jacobi form polls less often since it runs ~50x more iterations
        ce = check_every or (32 if precond == D.PRECOND_JACOBI else 4)
        if prec == D.F32:
            return D.Piso(dm, D.F32, D.piso_opts(
                NU, DT, 2, NONORTH, solve_U=D.solve_opts(D.BICGSTAB, 1e-6, max_iter=1000,
                                                         check_every=check_every or 4),
                solve_p=D.solve_opts(D.PCG, 1e-10, max_iter=20000, check_every=ce, refine_max=20,
                                     inner_tol=1e-4, precond=precond),
                pref_cell=pref, conv=conv, time_scheme=time_scheme))
        return D.Piso(dm, D.F64, D.piso_opts(
            NU, DT, 2, NONORTH, solve_U=D.solve_opts(D.BICGSTAB, 1e-10, max_iter=1000, check_every=4,
                                                     precond=precond_U),
            solve_p=D.solve_opts(D.PCG, 1e-10, max_iter=20000, check_every=ce, precond=precond),
            pref_cell=pref))

    info = torch.zeros(D.PISO_INFO_NBYTES, dtype=torch.uint8, device="cuda")

    def timed(prec, W, K, prof_tag=None, graph=False, precond=D.PRECOND_AMG, conv=D.CONV_UPWIND,
              time_scheme=D.TIME_BE, precond_U=D.PRECOND_JACOBI):
        dt_ = torch.float32 if prec == D.F32 else torch.float64
        h = piso(prec, precond, conv, time_scheme, precond_U=precond_U)
        s = new_state(dt_)

        def one():
            if graph:
                h.step_graph(*s, info=info)
                return 0
            return h.step(*s, info=info)[0]
        for _ in range(W):
            one()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        if prof_tag:
            D.difvm_prof_start(prof_tag, 200000)
        l0 = D.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        worst = 0
        for _ in range(K):
            worst = max(worst, one())
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        launches = D.launch_count() - l0
        prof = D.difvm_prof_stop() if prof_tag else None
        gi = D.decode_piso_info(info)
        if graph:
            worst = gi["status"]
        return dict(ms=ms, launches=launches, status=worst, prof=prof, info=gi, state=s, handle=h)

    # profiling runs (--only-f32) may skip the warm-up; timed runs keep W >= 3
    W, K = (args.warmup if args.only_f32 else max(args.warmup, 3)), args.steps
    # headline: the F32 step through difvm_piso_step_graph (the step captured once
    # as a CUDA graph, every solve a device-side loop; replayed each step)
    graph = not args.only_f32
    clocks = Clocks(local)
    clocks.start()
    rg = timed(D.F32, W, K, graph=graph)
    ck = clocks.stop()
    # the same step through difvm_piso_step (host-driven solver loops): secondary
    # line, launch count, and the state the roofline pass continues from
    r32 = timed(D.F32, W, K) if graph else rg
    # roofline passes: the same handle and state continue for K more steps, with
    # CUDA events recorded around every launch of one kernel (kept out of the
    # headline timed region, whose launches they would slow): the kernel with the
    # largest share of the step's time, the coarse-level corrected smoothing
    # sweep k_amg_post1<float, 8> (levels 2-5), and the mesh-level residual
    h32, s32 = r32["handle"], r32["state"]
    prof = {}
    for tag in (D.PROF_AMG_POST1C, D.PROF_AMG_RESID):
        torch.cuda.synchronize()
        D.difvm_prof_start(tag, 200000)
        for _ in range(K):
            h32.step(*s32, info=info)
        torch.cuda.synchronize()
        nbytes = D.prof_bytes()
        ms_tot, n_l = D.difvm_prof_stop()
        prof[tag] = (ms_tot, n_l, nbytes)
    # the split of a host-loop step into its phases (events at phase boundaries)
    torch.cuda.synchronize()
    D.difvm_phase_prof_start(100000)
    for _ in range(K):
        h32.step(*s32, info=info)
    torch.cuda.synchronize()
    ph_ms, ph_steps = D.difvm_phase_prof_stop()
    phases = {k: v / max(ph_steps, 1) for k, v in ph_ms.items()}
    ms_local = rg["ms"] / K
    ms_step = max_over_ranks(ms_local, dist if world > 1 else None, "cuda")
    value = job_rate(ms_step, world)

    # algorithmic bytes of one step: the same settings with the solvers' convergence
    # checked after every iteration (no iterations past convergence), W steps from
    # rest, then the bytes of K steps counted (the Krylov and multigrid kernels)
    hb, sb = piso(D.F32, check_every=1), new_state(torch.float32)
    for _ in range(W):
        hb.step(*sb, info=info)
    torch.cuda.synchronize()
    b0 = D.alg_bytes()
    for _ in range(K):
        hb.step(*sb, info=info)
    torch.cuda.synchronize()
    step_bytes = (D.alg_bytes() - b0) / K
    del hb, sb

    peak, peak_kind = measured_peaks()

    def kernel_roofline(tag):
        ms_tot, n_l, nbytes = prof[tag]
        avg_ms = ms_tot / max(n_l, 1)
        per_launch = nbytes / max(n_l, 1)
        ach = per_launch / (avg_ms * 1e-3) / 1e9 if n_l else None
        return ach, per_launch, avg_ms, n_l
    achieved, alg_bytes, avg_ms, n_post1 = kernel_roofline(D.PROF_AMG_POST1C)
    ach_res, alg_res, avg_res, n_res = kernel_roofline(D.PROF_AMG_RESID)

    def traffic_of(name):
        path = os.path.join(ROOT, "profiles", name)
        if not (os.path.exists(path) and args.mesh == N_KUHN):   # captured on the 64^3 mesh
            return None
        try:
            return json.load(open(path)).get("dram_bytes_per_launch")
        except Exception:
            return None

    if args.only_f32:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "steps/s", "ms_per_step": ms_step,
                              "mesh": args.mesh, "status": int(r32["status"]),
                              "amg_post1c_avg_us": avg_ms * 1e3, "amg_resid_avg_us": avg_res * 1e3,
                              "step_alg_bytes": step_bytes, "phases_ms_per_step": phases,
                              "info": r32["info"]}), flush=True)
        return 0
    rj = timed(D.F32, W, K, graph=True, precond=D.PRECOND_JACOBI)
    jacobi = {"value": 1e3 * K / rj["ms"], "unit": "steps/s", "ms_per_step": rj["ms"] / K,
              "status": int(rj["status"]), "pressure_iters_last_step": rj["info"]["itp"][:2],
              "api": "difvm_piso_step_graph, pressure CG with Jacobi preconditioning"}
    # the paper's preconditioner (diagonal incomplete Cholesky, level-scheduled): FP64, one
    # step (its sweeps advance one dependency level per launch: minutes per step above 64^3)
    if args.mesh <= N_KUHN:
        rd = timed(D.F64, 1, 1, precond=D.PRECOND_DIC)
        dic = {"value": 1e3 / rd["ms"], "unit": "steps/s", "ms_per_step": rd["ms"], "steps": 1,
               "status": int(rd["status"]), "pressure_iters_last_step": rd["info"]["itp"][:2],
               "launches_per_step": int(rd["launches"]),
               "api": "difvm_piso_step, FP64, pressure CG with DIC (factor and each sweep one launch, rows "
                      "waiting on the rows they depend on)"}
        # the paper's preconditioning of both solves: DILU momentum BiCGStab, DIC pressure CG
        ri = timed(D.F64, 1, 1, precond=D.PRECOND_DIC, precond_U=D.PRECOND_DIC)
        dic["with_dilu_momentum"] = {"value": 1e3 / ri["ms"], "unit": "steps/s", "ms_per_step": ri["ms"],
                                     "status": int(ri["status"]),
                                     "pressure_iters_last_step": ri["info"]["itp"][:2],
                                     "momentum_iters_last_step": ri["info"]["itU"],
                                     "launches_per_step": int(ri["launches"])}
    else:
        dic = {"skipped": f"not timed above {N_KUHN}^3 (a chain of dependency levels per sweep)"}
    rs = timed(D.F32, W, K, graph=True, conv=D.CONV_SOU)
    sou = {"value": 1e3 * K / rs["ms"], "unit": "steps/s", "ms_per_step": rs["ms"] / K,
           "status": int(rs["status"]), "pressure_iters_last_step": rs["info"]["itp"][:2],
           "momentum_iters_last_step": rs["info"]["itU"],
           "api": "difvm_piso_step_graph, momentum convection by second-order upwind deferred correction"}
    rc = timed(D.F32, W, K, graph=True, time_scheme=D.TIME_CN)
    cn = {"value": 1e3 * K / rc["ms"], "unit": "steps/s", "ms_per_step": rc["ms"] / K,
          "status": int(rc["status"]), "pressure_iters_last_step": rc["info"]["itp"][:2],
          "momentum_iters_last_step": rc["info"]["itU"],
          "api": "difvm_piso_step_graph, Crank-Nicolson momentum predictor"}
    host_loop = {"value": 1e3 * K / r32["ms"], "unit": "steps/s", "ms_per_step": r32["ms"] / K,
                 "status": int(r32["status"]), "pressure_iters_last_step": r32["info"]["itp"][:2],
                 "api": "difvm_piso_step (host polls the solver flags every check_every iterations)"}
    # plain FP64 form, same workload (fewer steps: it is the slow form)
    r64 = timed(D.F64, 3, max(2, min(K, 5)))
    ms64 = r64["ms"] / max(2, min(K, 5))
    # accuracy of the mixed-precision step: the F32 form (graph) stepped from rest
    # as many times as the FP64 run, fields compared (normwise max relative)
    n64 = 3 + max(2, min(K, 5))
    hq, sq = piso(D.F32), new_state(torch.float32)
    for _ in range(n64):
        hq.step_graph(*sq, info=info)
    torch.cuda.synchronize()

    def nrel(a, b):
        a, b = a.double(), b.double()
        return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))
    f32_err = {"steps": n64, "U": nrel(sq[0], r64["state"][0]), "p": nrel(sq[1], r64["state"][1]),
               "phi": nrel(sq[2], r64["state"][2])}
    del hq, sq

    # end to end through the public API, like the headline from rest (W warm-up
    # steps, then K timed steps): per step the boundary values go host -> device
    # from pinned memory, the step runs (difvm_piso_step_graph), and its result
    # (U, p, phi) comes back to pinned host buffers before the next step starts
    dt_ = torch.float32
    he, se = piso(D.F32), new_state(dt_)
    Ub_pin = torch.as_tensor(dm.to_bnd(Ub_h), dtype=dt_).contiguous().pin_memory()
    pb_pin = torch.zeros(dm.nb, dtype=dt_).pin_memory()
    out_pin = [torch.empty(se[k].shape, dtype=dt_).pin_memory() for k in range(3)]

    def e2e_step():
        se[3].copy_(Ub_pin, non_blocking=True)
        se[4].copy_(pb_pin, non_blocking=True)
        he.step_graph(*se, info=info)
        for k in range(3):
            out_pin[k].copy_(se[k], non_blocking=True)
        torch.cuda.current_stream().synchronize()
    for _ in range(W):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / K, dist if world > 1 else None, "cuda")
    h2d = (Ub_pin.numel() + pb_pin.numel()) * 4
    d2h = sum(t.numel() for t in out_pin) * 4
    e2e_same = bool(torch.equal(out_pin[0], se[0].cpu()) and torch.equal(out_pin[0], rg["state"][0].cpu()))
    del he, se

    h, s = r32["handle"], r32["state"]
    # forward + adjoint against forward alone, from one state of the same run:
    # loss = kinetic energy after K steps, its adjoint back to the state K steps
    # earlier and to U_b and nu (every step recorded; and with the state kept
    # every CKPT steps and the segments re-run with tapes)
    V32 = torch.as_tensor(dm.to_cells(m.V), dtype=dt_, device="cuda")

    def ke_grad(U, p, phi, pb, wk):
        return (V32 * U).contiguous(), torch.zeros_like(p), torch.zeros_like(phi), None, None

    base = [t.clone() for t in s]

    def fresh():
        return [t.clone() for t in base]

    def ev_time(fn):
        torch.cuda.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    # tapes and the handle's adjoint workspace are allocated before timing
    tapes = [h.new_tape("cuda") for _ in range(K)]
    D.simulate_adjoint(h, fresh(), 1, ke_grad, tapes=tapes)
    s1 = fresh()
    fwd_ms, _ = ev_time(lambda: [h.step(*s1, info=info) for _ in range(K)])
    s2 = fresh()
    fa_ms, adj = ev_time(lambda: D.simulate_adjoint(h, s2, K, ke_grad, tapes=tapes))
    s3 = fresh()
    fc_ms, adjc = ev_time(lambda: D.simulate_adjoint(h, s3, K, ke_grad, checkpoint_every=CKPT,
                                                     tapes=tapes))
    same = bool(torch.equal(adj["U"], adjc["U"]) and torch.equal(adj["nu"], adjc["nu"]))
    s4 = fresh()
    fb_ms, adjb = ev_time(lambda: D.simulate_adjoint(h, s4, K, ke_grad, checkpoints=BINOM_SLOTS, tapes=tapes))
    same_b = bool(torch.equal(adj["U"], adjb["U"]) and torch.equal(adj["nu"], adjb["nu"]))
    fwd_adj = {"value": fa_ms / fwd_ms, "unit": "time ratio", "steps": K,
               "fwd_ms_per_step": fwd_ms / K, "fwd_adj_ms_per_step": fa_ms / K,
               "over_headline_graph_step": (fa_ms / K) / ms_local,
               "over_headline_note": "fwd+adjoint (host-loop forward steps with tapes, then the reverse "
                                     "sweep) per step over the headline's graph-launched forward step",
               "taping": "every step recorded (tapes resident in HBM)",
               "tape_bytes_per_step": h.tape_bytes(),
               "checkpointed": {"every": CKPT, "value": fc_ms / fwd_ms,
                                "fwd_adj_ms_per_step": fc_ms / K, "bitwise_equal": same},
               "binomial": {"states": BINOM_SLOTS + 1, "tapes": 1, "value": fb_ms / fwd_ms,
                            "fwd_adj_ms_per_step": fb_ms / K, "bitwise_equal": same_b,
                            "plain_steps": D.binomial_cost(K, BINOM_SLOTS) + 1,
                            "schedule": "optimal binomial (Griewank), Sec. 2.5"},
               "loss": "kinetic energy after the K steps",
               "status": int(max(adj["status"], adjc["status"], adjb["status"])),
               "dL_dnu": float(adj["nu"][0]),
               "adjoint_iters_first_step": {k_: D.decode_piso_info(adj["info"])[k_][:n_]
                                            for k_, n_ in (("itU", 3), ("itp", 2))}}

    large = pipe = None
    if args.mesh == N_KUHN and not args.no_large:
        large = run_large(D, torch)
        pipe = run_pipe(D, torch)
    batched = None
    if not args.no_batch:
        batched = run_batched(D, torch)
        bj = run_batched(D, torch, K=3, precond=D.PRECOND_JACOBI, f64=False, adjoint=False)
        batched["jacobi_pressure"] = {k: bj[k] for k in ("value", "unit", "ms_per_step", "status",
                                                         "pressure_iters_max_over_cases", "steps")}

    if rank != 0:
        return 0
    # CPU baseline: one full oracle PISO step of the same cavity (single thread)
    cpu = None
    if not args.no_cpu:
        import oracle as O
        rate, secs = cpu_oracle_step_rate(m, steps=1)
        cpu = {"value": rate, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"1 full FP64 oracle PISO step of the same cavity from rest ({secs:.1f} s)"}
        # the same oracle built with OpenMP over cells (cell-CSR LDU apply, fixed-block
        # dot products: deterministic) on every host core
        try:
            threads = O.use_multicore(True)
            rate_mc, secs_mc = cpu_oracle_step_rate(m, steps=1)
        finally:
            O.use_multicore(False)
        cpu["all_cores"] = {"value": rate_mc, "unit": "steps/s", "cores": threads, "nproc": os.cpu_count(),
                            "kind": "oracle, OpenMP build",
                            "sample": f"1 full FP64 oracle PISO step of the same cavity from rest "
                                      f"({secs_mc:.1f} s)"}
    gi = rg["info"]
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.mesh in (N_KUHN, *LARGE) else f"kuhn{args.mesh}_cavity_re100",
                   "mesh": f"kuhn{args.mesh}^3 jitter {JITTER} seed {SEED} RCM",
                   "cells": dm.nc, "faces": dm.nf, "nu": NU, "dt": DT, "n_corr": 2,
                   "nonorth": "momentum (the lagged pressure correction diverges on these tets)",
                   "precision": "f32 fields/operators, f64 dots; pressure: f64 CG to 1e-10 around an "
                                "f32 multigrid V-cycle",
                   "pressure_solver": "CG + one aggregation-multigrid V-cycle per iteration",
                   "parallelism": f"replicas x{world}",
                   "api": "difvm_piso_step_graph (one CUDA graph per step, solver loops on the device)",
                   "l2": f"working set (~{0.9 * (args.mesh / 64) ** 3:.1f} GB) > 126 MB L2; no flush needed"},
        "gpu_launches": int(r32["launches"]),
        "tuned_launch_shapes": {f"{k[0]}.{k[1]}.{k[2]}": v for k, v in D.difvm_mesh_tuning(dm).items()},
        "gpu_launches_note": "counted on the host-loop run of the same K steps; the graph replays "
                             "the same kernels plus at most 3 early-exit iterations and one "
                             "loop-condition kernel per pass of each solver loop",
        "status": int(rg["status"]),
        "pressure_iters_last_step": gi["itp"][:2], "momentum_iters_last_step": gi["itU"],
        "host_loop": host_loop,
        "phases_ms_per_step": {"host_loop_step": phases,
                               "note": "CUDA events at the phase boundaries of difvm_piso_step (F32, "
                                       "same run as the roofline passes); the graph step runs the same "
                                       "kernels"},
        "jacobi_pressure": jacobi,
        "dic_pressure": dic,
        "sou_convection": sou,
        "crank_nicolson": cn,
        "f64": {"value": 1e3 / ms64, "unit": "steps/s", "ms_per_step": ms64,
                "pressure_iters_last_step": r64["info"]["itp"][:2],
                "momentum_iters_last_step": r64["info"]["itU"],
                "f32_field_err_vs_f64": f32_err},
        "fwd_adjoint_over_fwd": fwd_adj,
        "face_ops": face_ops,
        "batched": batched,
        "large": large,
        "pulsatile_pipe": pipe,
        "roofline": {"kernel": "k_amg_post1<float, 8> (coarse-level multigrid corrected smoothing "
                               "sweep, levels 2-5; the largest share of the step's kernel time)",
                     "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic_of("traffic_amg_post1c_f32_kuhn64.json"),
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_us": avg_ms * 1e3,
                     "launches_timed": n_post1, "peak_kind": peak_kind,
                     "step_alg_bytes": step_bytes,
                     "step_frac": step_bytes / (ms_step * 1e-3) / (peak * 1e9),
                     "step_frac_note": "algorithmic bytes of the Krylov and multigrid kernels of one step "
                                       "(about 93% of the step's kernel time) / ms_per_step / peak; the "
                                       "assembly, gradient and flux kernels are not counted, so this is a "
                                       "lower bound",
                     "mesh_level_residual": {"kernel": "k_amg_resid<float, 1>", "achieved": ach_res,
                                             "frac": (ach_res / peak) if ach_res else None,
                                             "alg_bytes_per_launch": alg_res,
                                             "avg_launch_us": avg_res * 1e3, "launches_timed": n_res,
                                             "traffic": traffic_of("traffic_amg_resid_f32_kuhn64.json")}},
        "e2e": {"value": job_rate(e2e_ms, world), "unit": "steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "returned": "U, p, phi to pinned host memory every step",
                "same_final_U_as_headline": e2e_same},
        "clocks": ck,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-case line")
    ap.add_argument("--no-large", action="store_true", help="skip the 128^3 Re 400 and pulsatile-pipe lines")
    ap.add_argument("--batch-only", action="store_true", help="time only the batched 64-case form")
    ap.add_argument("--batch-jacobi", action="store_true",
                    help="with --batch-only: Jacobi instead of multigrid for the pressure CG")
    ap.add_argument("--mesh", type=int, default=N_KUHN, help="Kuhn hex grid size n (n^3 hexes)")
    ap.add_argument("--face-ops-only", action="store_true",
                    help="run only the face-operator timings (for profiling runs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default launch shapes and no first-use timing on the bench mesh (for launch lists)")
    ap.add_argument("--face-ops-launches", action="store_true",
                    help="launch each F32 face operator 5 times with the default variants (for ncu captures)")
    ap.add_argument("--only-f32", action="store_true",
                    help="time only the F32 form (no F64 or end-to-end legs; for profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
