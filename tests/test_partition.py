"""A mesh cut into per-rank subdomains (partition.py): host logic, and two gloo
ranks on the CPU.

Each rank's local mesh holds its owned cells, their ghosts and every face of an
owned cell in the global face order, so a face-loop operator gives every owned
cell its whole-mesh value bit for bit once the ghosts hold their owners' values.
The oracle's operators stand in for a rank's kernels here (the CPU has no GPU):
the LDU apply and the Gauss gradient on the local meshes, the halo exchange and
the FP64 dot products over ranks, and ten Jacobi-CG iterations on the
partitioned system, all against the single-domain results, bitwise.
"""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2603_15920_b300 import meshgen as mg
from paper_2603_15920_b300 import partition as P

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _mesh():
    return mg.shuffle(mg.kuhn_cube(6, 0.2, 3, patch_types=dict(x1=mg.OUTLET)), 4)


def _system(m, seed=1):
    om = O.OMesh.from_mesh(m)
    w, c, k = O.face_coeffs(om)
    rng = np.random.default_rng(seed)
    a = c[:m.n_internal] * rng.uniform(0.5, 2.0, m.n_internal)
    Dg = np.bincount(m.owner[:m.n_internal], a, m.n_cells) + np.bincount(m.neighbour, a, m.n_cells) + 0.1 * m.V
    return om, Dg, -a


@pytest.mark.parametrize("nparts", [2, 3])
def test_subdomains_cover_the_mesh_once(nparts):
    m = _mesh()
    part = P.partition_cells(m, nparts)
    assert set(np.bincount(part)) <= {m.n_cells // nparts, m.n_cells // nparts + 1}
    subs = P.build_subdomains(m, part)
    owned = np.concatenate([s.cells[:s.n_owned] for s in subs])
    assert np.array_equal(np.sort(owned), np.arange(m.n_cells))
    # every face is held by exactly one rank
    held = np.concatenate([s.faces[s.face_owned] for s in subs])
    assert np.array_equal(np.sort(held), np.arange(m.n_faces))
    deg = np.bincount(np.r_[m.owner, m.neighbour], minlength=m.n_cells)
    for s in subs:
        lm = s.mesh
        ldeg = np.bincount(np.r_[lm.owner, lm.neighbour], minlength=lm.n_cells)
        assert np.array_equal(ldeg[:s.n_owned], deg[s.cells[:s.n_owned]])   # owned cells see all their faces
        assert np.all(np.diff(s.faces[:lm.n_internal]) > 0)                 # global order kept
        for q, idx in s.recv.items():
            assert np.array_equal(subs[q].cells[subs[q].send[s.rank]], s.cells[idx])
        assert all(part[s.cells[s.n_owned:]] != s.rank)


def test_local_operators_give_the_whole_mesh_rows_bitwise():
    m = _mesh()
    om, Dg, L = _system(m)
    U = L * np.random.default_rng(2).uniform(0.5, 1.5, L.shape[0])
    rng = np.random.default_rng(3)
    x, phib = rng.normal(size=(3, m.n_cells)), rng.normal(size=(3, m.n_boundary))
    y = O.ldu_apply(om, Dg, L, U, x)
    g = O.grad_gauss(om, om.bc_U(), x, phib)
    for s in P.build_subdomains(m, P.partition_cells(m, 3)):
        lm, n, ni = s.mesh, s.n_owned, s.mesh.n_internal
        lom = O.OMesh.from_mesh(lm)
        fi = s.faces[:ni]
        yl = O.ldu_apply(lom, Dg[s.cells], L[fi], U[fi], x[:, s.cells])
        assert np.array_equal(yl[:, :n], y[:, s.cells[:n]])
        gl = O.grad_gauss(lom, lom.bc_U(), x[:, s.cells], phib[:, s.faces[ni:] - m.n_internal])
        assert np.array_equal(gl[:, :, :n], g[:, :, s.cells[:n]])


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _cg(apply, dot, Dg, b, iters):
    x = torch.zeros_like(b)
    r = b - apply(x)
    z = r / Dg
    p = z.clone()
    rz = dot(r, z)
    for _ in range(iters):
        q = apply(p)
        alpha = rz / dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        z = r / Dg
        rz1 = dot(r, z)
        p = z + (rz1 / rz) * p
        rz = rz1
    return x


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = _mesh()
        om, Dg, L = _system(m)
        part = P.partition_cells(m, world)
        subs = P.build_subdomains(m, part)
        s = subs[rank]
        lom = O.OMesh.from_mesh(s.mesh)
        n, fi = s.n_owned, s.faces[:s.mesh.n_internal]
        xg = np.random.default_rng(5).normal(size=(2, m.n_cells))
        # halo exchange: ghosts get their owners' values
        xl = torch.as_tensor(xg[:, s.cells]).clone()
        xl[:, n:] = -7.0
        P.exchange(s, xl, dist)
        res = {"halo": bool(np.array_equal(xl.numpy(), xg[:, s.cells]))}
        # the partitioned apply: owned rows
        res["apply"] = O.ldu_apply(lom, Dg[s.cells], L[fi], None, xl.numpy())[:, :n]
        res["owned"] = s.cells[:n]
        # dot products over ranks
        res["dot"] = P.dot(s, xl, xl, dist).numpy()
        # ten Jacobi-CG iterations on the partitioned system

        def apply(v):
            v = v.clone()
            P.exchange(s, v, dist)
            return torch.as_tensor(O.ldu_apply(lom, Dg[s.cells], L[fi], None, v.numpy()[None])[0])
        b = torch.as_tensor(np.random.default_rng(6).normal(size=m.n_cells)[s.cells])
        res["cg"] = _cg(apply, lambda a, c: P.dot(s, a, c, dist), torch.as_tensor(Dg[s.cells]), b, 10)[:n].numpy()
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_the_single_domain_bitwise():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    m = _mesh()
    om, Dg, L = _system(m)
    part = P.partition_cells(m, world)
    owned = [np.flatnonzero(part == r) for r in range(world)]
    xg = np.random.default_rng(5).normal(size=(2, m.n_cells))
    y = O.ldu_apply(om, Dg, L, None, xg)

    def dot_ref(a, c):   # the ranks' partial sums, added across ranks
        return sum((a[..., o].double() * c[..., o].double()).sum(dim=-1) for o in owned)
    x_ref = _cg(lambda v: torch.as_tensor(O.ldu_apply(om, Dg, L, None, v.numpy()[None])[0]), dot_ref,
                torch.as_tensor(Dg), torch.as_tensor(np.random.default_rng(6).normal(size=m.n_cells)), 10)
    for r in range(world):
        got = res[r]
        assert got["halo"]
        assert np.array_equal(got["apply"], y[:, got["owned"]])
        assert np.array_equal(got["dot"], dot_ref(torch.as_tensor(xg), torch.as_tensor(xg)).numpy())
        assert np.array_equal(got["cg"], x_ref[got["owned"]].numpy())


def test_three_gloo_ranks_exchange_and_apply_bitwise():
    # a middle slab has two neighbour ranks; the halo exchange and the partitioned
    # apply stay bitwise (only the FP64 sums over three ranks depend on the
    # reduction order, so the dot products and CG are checked to rounding)
    world, port = 3, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    m = _mesh()
    om, Dg, L = _system(m)
    part = P.partition_cells(m, world)
    subs = P.build_subdomains(m, part)
    assert max(len(s.recv) for s in subs) == 2
    owned = [np.flatnonzero(part == r) for r in range(world)]
    xg = np.random.default_rng(5).normal(size=(2, m.n_cells))
    y = O.ldu_apply(om, Dg, L, None, xg)
    dot = (xg * xg).sum(axis=-1)

    def dot_ref(a, c):
        return sum((a[..., o].double() * c[..., o].double()).sum(dim=-1) for o in owned)
    x_ref = _cg(lambda v: torch.as_tensor(O.ldu_apply(om, Dg, L, None, v.numpy()[None])[0]), dot_ref,
                torch.as_tensor(Dg), torch.as_tensor(np.random.default_rng(6).normal(size=m.n_cells)), 10)
    for r in range(world):
        got = res[r]
        assert got["halo"]
        assert np.array_equal(got["apply"], y[:, got["owned"]])
        np.testing.assert_allclose(got["dot"], dot, rtol=1e-14)
        np.testing.assert_allclose(got["cg"], x_ref[got["owned"]].numpy(), rtol=1e-10,
                                   atol=1e-12 * float(x_ref.abs().max()))
