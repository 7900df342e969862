"""A mesh cut into per-rank subdomains for one process per GPU (Sec. 4.2 names
graph partitioning with halo exchange as the way past one GPU).

Host-side logic only; the operators and solvers on each rank are the library's,
run on the rank's local mesh.  The pieces:

* ``partition_cells``: cells split into ``nparts`` balanced slabs of a
  reverse Cuthill-McKee order of the cell graph (each cut is a front of the
  ordering, so a subdomain touches at most two others on band-like meshes).
  No METIS is available here; any other cell -> rank map can be passed in.
* ``Subdomain``: the local mesh of one rank.  Its cells are the rank's own cells
  (ascending global id) followed by its ghosts (cells of other ranks that share
  a face with an owned cell, ascending global id); its faces are every global
  face that touches an owned cell, in ascending global face id (internal faces
  first, then boundary faces by patch), with their global orientation.  An
  owned cell therefore sees exactly its global faces in the global order, so a
  cell-centric operator (every face message summed in ascending face id) gives
  an owned cell the value it has on the whole mesh, bit for bit, once the
  ghosts hold their owners' values; ghost rows are incomplete and ignored.
  Each cut face appears on both of its ranks; ``face_owned`` marks the copy
  that counts (the rank of the face's global owner), for face fields and sums.
* ``Subdomain.send`` / ``Subdomain.recv`` and ``exchange``: per neighbour rank,
  the owned cells it needs (send, ascending global id) and where its cells land
  among the ghosts (receive, same order); ``exchange`` moves the values with
  point-to-point ``torch.distributed`` messages (gloo on host tensors, NCCL on
  device tensors), once before every pass that gathers neighbour values.
* ``dot``: the inner product over owned cells, summed on each rank and then
  across ranks with ``all_reduce`` in FP64 (2 ranks: the sum of two partials is
  the same double in either order).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import meshgen as mg


def partition_cells(mesh, nparts: int) -> np.ndarray:
    """Rank of every cell: nparts slabs of equal size (to one cell) of a reverse
    Cuthill-McKee order of the cell graph."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    nc, ni = mesh.n_cells, mesh.n_internal
    o, n = mesh.owner[:ni], mesh.neighbour
    A = sp.coo_matrix((np.ones(2 * ni), (np.r_[o, n], np.r_[n, o])), shape=(nc, nc)).tocsr()
    order = reverse_cuthill_mckee(A, symmetric_mode=True)
    part = np.empty(nc, np.int32)
    bounds = np.linspace(0, nc, nparts + 1).round().astype(np.int64)
    for r in range(nparts):
        part[order[bounds[r]:bounds[r + 1]]] = r
    return part


@dataclass
class Subdomain:
    rank: int
    mesh: mg.Mesh                 # local mesh: owned cells, then ghosts
    cells: np.ndarray             # global id of every local cell
    n_owned: int
    faces: np.ndarray             # global id of every local face
    face_owned: np.ndarray        # bool: this rank holds the face (its global owner is owned here)
    send: dict = field(default_factory=dict)   # rank -> local ids of owned cells it needs
    recv: dict = field(default_factory=dict)   # rank -> local ids of the ghosts it provides

    @property
    def n_ghost(self) -> int:
        return int(self.cells.shape[0]) - self.n_owned


def build_subdomains(mesh, part: np.ndarray) -> list:
    """The local mesh and halo lists of every rank of the cell -> rank map part."""
    nparts = int(part.max()) + 1
    nc, ni = mesh.n_cells, mesh.n_internal
    own_i, nei = mesh.owner[:ni], mesh.neighbour
    bpatch = mesh.boundary_patch_id()
    subs = []
    for r in range(nparts):
        owned = np.flatnonzero(part == r)
        touch = (part[own_i] == r) | (part[nei] == r)
        ifaces = np.flatnonzero(touch)                               # ascending global id
        other = np.r_[own_i[ifaces], nei[ifaces]]
        ghosts = np.unique(other[part[other] != r])
        cells = np.r_[owned, ghosts].astype(np.int64)
        loc = np.full(nc, -1, np.int64)
        loc[cells] = np.arange(cells.shape[0])
        bfaces = ni + np.flatnonzero(part[mesh.owner[ni:]] == r)     # grouped by patch, global order
        groups = []
        for p in range(mesh.n_patches):
            f = bfaces[bpatch[bfaces - ni] == p]
            groups.append((loc[mesh.owner[f]].astype(np.int64), mesh.Sf[f], mesh.Cf[f]))
        local = mg._finish(cells.shape[0], loc[own_i[ifaces]], loc[nei[ifaces]], mesh.Sf[ifaces],
                           mesh.Cf[ifaces], mesh.V[cells], mesh.C[cells], groups, mesh.patch_names,
                           list(mesh.patch_type))
        faces = np.r_[ifaces, bfaces]
        face_owned = part[mesh.owner[faces]] == r
        subs.append(Subdomain(r, local, cells, int(owned.shape[0]), faces, face_owned))
    # halo lists: what each rank's ghosts need from their owners, in ascending global id
    for s in subs:
        ghosts = s.cells[s.n_owned:]
        for q in np.unique(part[ghosts]):
            q = int(q)
            g = ghosts[part[ghosts] == q]                  # ascending (ghosts are sorted)
            s.recv[q] = s.n_owned + np.flatnonzero(part[ghosts] == q)
            t = subs[q]
            pos = np.searchsorted(t.cells[:t.n_owned], g)
            assert np.array_equal(t.cells[pos], g)
            t.send[s.rank] = pos
    return subs


def exchange(sub: Subdomain, x, dist):
    """Fill the ghost entries of x ([..., n_local] tensor of this rank) with
    their owners' values.  Every rank must call it (collective over the
    neighbour pairs)."""
    import torch
    reqs, bufs = [], {}
    for q in sorted(sub.recv):
        bufs[q] = torch.empty(x.shape[:-1] + (len(sub.recv[q]),), dtype=x.dtype, device=x.device)
        reqs.append(dist.irecv(bufs[q], src=q))
    for q in sorted(sub.send):
        idx = torch.as_tensor(sub.send[q], dtype=torch.long, device=x.device)
        reqs.append(dist.isend(x[..., idx].contiguous(), dst=q))
    for rq in reqs:
        rq.wait()
    for q, b in bufs.items():
        x[..., torch.as_tensor(sub.recv[q], dtype=torch.long, device=x.device)] = b
    return x


def dot(sub: Subdomain, x, y, dist):
    """sum over owned cells of x y (last axis), across every rank, in FP64."""
    n = sub.n_owned
    # contiguous operands: the reduction order of a sum depends on the layout
    xo, yo = x[..., :n].double().contiguous(), y[..., :n].double().contiguous()
    part = (xo * yo).sum(dim=-1, keepdim=True)
    dist.all_reduce(part, op=dist.ReduceOp.SUM)
    return part[..., 0]
