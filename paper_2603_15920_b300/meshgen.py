"""Seeded synthetic meshes and fields for the face-operator / PISO path.

This module only *generates inputs*.  It produces the static arrays that the
method takes as given (Sec. 2.4.1, static graph construction): owner and
neighbour cell indices per face, face area vectors S_f (pointing out of the
owner), face centroids x_f, cell volumes V and cell centroids C, and the
boundary patches (faces grouped by patch, after all internal faces).  It holds
none of the finite-volume arithmetic (face interpolation, gradients, fluxes,
matrices, solvers): that lives in the CUDA library and, independently, in the
CPU oracle.  Both sides are fed from here.

Mesh families (all synthetic, all seeded):
  * ``hex_box``   -- uniform axis-aligned hexahedra (the 2D channel of the
                     Poiseuille run is a one-cell-thick box with empty z sides),
  * ``kuhn_cube`` -- a unit cube cut into n^3 hexes, each split into the six
                     Kuhn tetrahedra around its v000-v111 diagonal, interior
                     vertices jittered uniformly by +-jitter*h,
  * ``pipe_ohgrid`` -- a straight cylinder meshed by an O-H grid (square core
                     block plus four outer blocks) extruded in uniform layers.

Patch type codes (an input convention shared with the C ABI header):
  WALL   fixed velocity (value supplied per face), zero-gradient pressure
  INLET  fixed velocity, zero-gradient pressure
  OUTLET zero-gradient velocity, fixed pressure
  EMPTY  excluded from every face sum (2D runs)
"""
from __future__ import annotations

from dataclasses import dataclass, field
import itertools

import numpy as np

WALL, INLET, OUTLET, EMPTY = 0, 1, 2, 3


@dataclass
class Mesh:
    n_cells: int
    n_internal: int
    owner: np.ndarray        # int32 [nf]
    neighbour: np.ndarray    # int32 [nint]
    Sf: np.ndarray           # float64 [nf, 3], out of the owner
    Cf: np.ndarray           # float64 [nf, 3], face centroids
    V: np.ndarray            # float64 [nc]
    C: np.ndarray            # float64 [nc, 3]
    patch_names: list = field(default_factory=list)
    patch_start: np.ndarray = None   # int32 [np], absolute face index
    patch_size: np.ndarray = None    # int32 [np]
    patch_type: np.ndarray = None    # int32 [np]
    # vertex topology (polyMesh form), when the generator keeps it: points [np, 3];
    # the vertices of face f are face_pts[face_ptr[f]:face_ptr[f + 1]], ordered so that
    # their right-hand normal points out of the owner
    points: np.ndarray = None
    face_ptr: np.ndarray = None
    face_pts: np.ndarray = None

    @property
    def n_faces(self) -> int:
        return int(self.owner.shape[0])

    @property
    def n_boundary(self) -> int:
        return self.n_faces - self.n_internal

    @property
    def n_patches(self) -> int:
        return len(self.patch_names)

    def patch_index(self, name: str) -> int:
        return self.patch_names.index(name)

    def patch_faces(self, name: str) -> np.ndarray:
        p = self.patch_index(name)
        s = int(self.patch_start[p])
        return np.arange(s, s + int(self.patch_size[p]))

    def boundary_patch_id(self) -> np.ndarray:
        """Patch id of every boundary face, [nb]."""
        out = np.empty(self.n_boundary, np.int32)
        for p in range(self.n_patches):
            s = int(self.patch_start[p]) - self.n_internal
            out[s:s + int(self.patch_size[p])] = p
        return out

    def check(self):
        nc, ni, nf = self.n_cells, self.n_internal, self.n_faces
        assert self.owner.dtype == np.int32 and self.neighbour.dtype == np.int32
        assert self.neighbour.shape == (ni,)
        assert self.Sf.shape == (nf, 3) and self.Cf.shape == (nf, 3)
        assert self.V.shape == (nc,) and self.C.shape == (nc, 3)
        assert self.owner.min() >= 0 and self.owner.max() < nc
        if ni > 0:
            assert self.neighbour.min() >= 0 and self.neighbour.max() < nc
        assert np.all(self.V > 0)
        assert int(self.patch_start[0]) == ni
        assert int(self.patch_start[-1] + self.patch_size[-1]) == nf
        assert np.all(self.patch_start[1:] == self.patch_start[:-1] + self.patch_size[:-1])
        return self


def _finish(nc, owner, neighbour, Sf, Cf, V, C, bnd_groups, names, types, topo=None):
    """Assemble a Mesh from internal faces plus boundary face groups.  topo:
    (points, internal face vertices [ni, k], [group face vertices [n_g, k]])."""
    o_i, S_i, X_i = owner, Sf, Cf
    o_b = [g[0] for g in bnd_groups]
    S_b = [g[1] for g in bnd_groups]
    X_b = [g[2] for g in bnd_groups]
    ni = o_i.shape[0]
    sizes = np.array([o.shape[0] for o in o_b], np.int32)
    starts = (ni + np.concatenate([[0], np.cumsum(sizes)[:-1]])).astype(np.int32)
    m = Mesh(
        n_cells=int(nc), n_internal=int(ni),
        owner=np.ascontiguousarray(np.concatenate([o_i] + o_b).astype(np.int32)),
        neighbour=np.ascontiguousarray(neighbour.astype(np.int32)),
        Sf=np.ascontiguousarray(np.concatenate([S_i] + S_b).astype(np.float64)),
        Cf=np.ascontiguousarray(np.concatenate([X_i] + X_b).astype(np.float64)),
        V=np.ascontiguousarray(V.astype(np.float64)),
        C=np.ascontiguousarray(C.astype(np.float64)),
        patch_names=list(names), patch_start=starts, patch_size=sizes,
        patch_type=np.array(types, np.int32),
    )
    if topo is not None:
        pts, fv_i, fv_b = topo
        fv = [np.asarray(a, np.int64) for a in [fv_i] + list(fv_b)]
        counts = np.concatenate([np.full(a.shape[0], a.shape[1]) for a in fv])
        m.points = np.ascontiguousarray(pts, np.float64)
        m.face_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        m.face_pts = np.ascontiguousarray(np.concatenate([a.ravel() for a in fv]).astype(np.int32))
        assert m.face_ptr[-1] == m.face_pts.shape[0] and m.face_ptr.shape[0] == m.n_faces + 1
    return m.check()


def shuffle(mesh: Mesh, seed: int) -> Mesh:
    """Randomly renumber cells, internal faces and faces inside each patch.

    Face orientation is kept (S_f still points out of the same physical cell),
    so an internal face may end up with owner id > neighbour id.  This is the
    'cell ids randomly permuted by seed' input of the channel run; the loader
    must undo the locality loss.  The vertex topology is not carried over.
    """
    rng = np.random.default_rng(seed)
    nc, ni, nf = mesh.n_cells, mesh.n_internal, mesh.n_faces
    new_of_old = rng.permutation(nc).astype(np.int32)
    old_of_new = np.empty(nc, np.int64)
    old_of_new[new_of_old] = np.arange(nc)
    fperm = [rng.permutation(ni)]
    for p in range(mesh.n_patches):
        s, n = int(mesh.patch_start[p]), int(mesh.patch_size[p])
        fperm.append(s + rng.permutation(n))
    fperm = np.concatenate(fperm)
    return Mesh(
        n_cells=nc, n_internal=ni,
        owner=np.ascontiguousarray(new_of_old[mesh.owner[fperm]]),
        neighbour=np.ascontiguousarray(new_of_old[mesh.neighbour[fperm[:ni]]]),
        Sf=np.ascontiguousarray(mesh.Sf[fperm]), Cf=np.ascontiguousarray(mesh.Cf[fperm]),
        V=np.ascontiguousarray(mesh.V[old_of_new]), C=np.ascontiguousarray(mesh.C[old_of_new]),
        patch_names=list(mesh.patch_names), patch_start=mesh.patch_start.copy(),
        patch_size=mesh.patch_size.copy(), patch_type=mesh.patch_type.copy(),
    ).check()


def batch(meshes):
    """Disjoint union of independent meshes (the batched input of Sec. 2.4:
    many cases in one launch).  Cells and internal faces are concatenated in
    case order; boundary patches are listed case by case and named
    "c<k>/<name>".  Returns (mesh, case_cell_start[n_cases + 1])."""
    cs = np.concatenate([[0], np.cumsum([m.n_cells for m in meshes])]).astype(np.int32)
    owner_i, nei, S_i, X_i = [], [], [], []
    for k, m in enumerate(meshes):
        ni = m.n_internal
        owner_i.append(m.owner[:ni] + cs[k])
        nei.append(m.neighbour + cs[k])
        S_i.append(m.Sf[:ni])
        X_i.append(m.Cf[:ni])
    groups, names, types = [], [], []
    for k, m in enumerate(meshes):
        for p, nm in enumerate(m.patch_names):
            f = m.patch_faces(nm)
            groups.append((m.owner[f] + cs[k], m.Sf[f], m.Cf[f]))
            names.append(f"c{k}/{nm}")
            types.append(int(m.patch_type[p]))
    u = _finish(int(cs[-1]), np.concatenate(owner_i), np.concatenate(nei),
                np.concatenate(S_i), np.concatenate(X_i),
                np.concatenate([m.V for m in meshes]), np.concatenate([m.C for m in meshes]),
                groups, names, types)
    return u, cs


def cavity_batch(n_cases: int = 64, seed: int = 4, jitter: float = 0.2):
    """The batched benchmark input: n_cases lid-driven cavities, each a Kuhn
    cube of n^3 hexes with n ~ U{8..48} and the given jitter (case k seeded
    100 + k).  The lid (patch y1) is a wall moving with U = (1, 0, 0); each of
    the other five sides is a fixed wall with probability 0.8, else an opening
    (OUTLET: zero-gradient velocity, fixed pressure), drawn by seed.  Returns
    (cases, union mesh, case_cell_start, lid boundary values of the union
    [3, n_boundary], opening table [n_cases, 5] for x0, x1, y0, z0, z1)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(8, 49, size=n_cases)
    sides = ("x0", "x1", "y0", "z0", "z1")
    opens = rng.uniform(size=(n_cases, len(sides))) >= 0.8
    ms = [kuhn_cube(int(n), jitter, 100 + k,
                    patch_types={sd: (OUTLET if opens[k, q] else WALL) for q, sd in enumerate(sides)})
          for k, n in enumerate(ns)]
    u, cs = batch(ms)
    Ub = np.zeros((3, u.n_boundary))
    for k in range(n_cases):
        Ub[0, u.patch_faces(f"c{k}/y1") - u.n_internal] = 1.0
    return ms, u, cs, Ub, opens


# ---------------------------------------------------------------------------
# uniform hex box
# ---------------------------------------------------------------------------
def hex_box(nx, ny, nz, lengths=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0),
            patch_types=None) -> Mesh:
    """Uniform box of nx*ny*nz hexahedra.  Patches x0,x1,y0,y1,z0,z1."""
    Lx, Ly, Lz = lengths
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    ox, oy, oz = origin
    types = dict(x0=WALL, x1=WALL, y0=WALL, y1=WALL, z0=WALL, z1=WALL)
    if patch_types:
        types.update(patch_types)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    cid = lambda i, j, k: i + nx * (j + ny * k)
    nc = nx * ny * nz
    C = np.stack([ox + (i + 0.5) * hx, oy + (j + 0.5) * hy, oz + (k + 0.5) * hz], 1)
    V = np.full(nc, hx * hy * hz)
    own, nei, S, X = [], [], [], []
    area = np.array([hy * hz, hx * hz, hx * hy])
    for ax, (ii, jj, kk) in enumerate([(i, j, k)] * 3):
        step = [0, 0, 0]
        step[ax] = 1
        lim = [nx, ny, nz][ax]
        idx = [ii, jj, kk][ax]
        m = idx < lim - 1
        o = cid(ii[m], jj[m], kk[m])
        n = cid(ii[m] + step[0], jj[m] + step[1], kk[m] + step[2])
        Sv = np.zeros((m.sum(), 3)); Sv[:, ax] = area[ax]
        Xv = C[o].copy(); Xv[:, ax] += 0.5 * [hx, hy, hz][ax]
        own.append(o); nei.append(n); S.append(Sv); X.append(Xv)
    groups, names = [], []
    for ax, (lo, hi) in enumerate([("x0", "x1"), ("y0", "y1"), ("z0", "z1")]):
        idx = [i, j, k][ax]
        lim = [nx, ny, nz][ax]
        h = [hx, hy, hz][ax]
        for name, sel, sgn in ((lo, idx == 0, -1.0), (hi, idx == lim - 1, 1.0)):
            o = cid(i[sel], j[sel], k[sel])
            Sv = np.zeros((o.shape[0], 3)); Sv[:, ax] = sgn * area[ax]
            Xv = C[o].copy(); Xv[:, ax] += sgn * 0.5 * h
            groups.append((o, Sv, Xv)); names.append(name)
    return _finish(nc, np.concatenate(own), np.concatenate(nei), np.concatenate(S),
                   np.concatenate(X), V, C, groups, names, [types[n] for n in names])


def channel_2d(nx=64, ny=16, lengths=(4.0, 1.0, 0.0625), seed=None) -> Mesh:
    """The Poiseuille channel: inlet x0, outlet x1, walls y0/y1, empty z sides."""
    m = hex_box(nx, ny, 1, lengths, patch_types=dict(
        x0=INLET, x1=OUTLET, y0=WALL, y1=WALL, z0=EMPTY, z1=EMPTY))
    m.patch_names = ["inlet", "outlet", "wall_lo", "wall_hi", "front", "back"]
    if seed is not None:
        m = shuffle(m, seed)
    return m


# ---------------------------------------------------------------------------
# Kuhn-split tetrahedral cube
# ---------------------------------------------------------------------------
_KUHN_PERMS = list(itertools.permutations(range(3)))
_TET_FACES = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))


def kuhn_cube(n: int, jitter: float = 0.0, seed: int = 0, patch_types=None) -> Mesh:
    """Unit cube, n^3 hexes, 6 Kuhn tets each (6 n^3 cells, 12 n^2 boundary faces).

    Interior vertices are moved by U(-jitter*h, +jitter*h) per coordinate
    (seeded); boundary vertices stay on the cube, so every boundary face lies
    exactly in its side plane.  Internal faces come in vertex-key order (not
    sorted by cell), boundary faces grouped by side x0,x1,y0,y1,z0,z1.
    """
    h = 1.0 / n
    n1 = n + 1
    g = np.arange(n1, dtype=np.float64) * h
    vz, vy, vx = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([vx.ravel(), vy.ravel(), vz.ravel()], 1)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=P.shape)
        ii = np.rint(P / h).astype(np.int64)
        interior = np.all((ii > 0) & (ii < n), axis=1)
        P[interior] += d[interior]
    vid = lambda i, j, k: i + n1 * (j + n1 * k)
    hk, hj, hi = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    nhex = n ** 3
    tets = np.empty((nhex, 6, 4), np.int64)
    for t, perm in enumerate(_KUHN_PERMS):
        cur = np.zeros((3, nhex), np.int64)
        base = np.stack([hi, hj, hk])
        tets[:, t, 0] = vid(*base)
        for s in range(3):
            cur[perm[s]] += 1
            b = base + cur
            tets[:, t, s + 1] = vid(*b)
    tets = tets.reshape(-1, 4)
    nc = tets.shape[0]
    X = P[tets]                                   # [nc,4,3]
    C = X.mean(axis=1)
    e1, e2, e3 = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]
    V = np.abs(np.einsum("ij,ij->i", e1, np.cross(e2, e3))) / 6.0
    assert np.all(V > 0), "inverted tetrahedron"
    # face slots: 4 per tet
    fv = np.sort(tets[:, _TET_FACES], axis=2).reshape(-1, 3)   # [4nc,3]
    cell_of_slot = np.repeat(np.arange(nc), 4)
    nv = P.shape[0]
    key = (fv[:, 0] * nv + fv[:, 1]) * nv + fv[:, 2]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    first = np.ones(ks.shape[0], bool)
    first[1:] = ks[1:] != ks[:-1]
    starts = np.flatnonzero(first)
    counts = np.diff(np.append(starts, ks.shape[0]))
    assert counts.max() <= 2
    pair = starts[counts == 2]
    single = starts[counts == 1]
    ca, cb = cell_of_slot[order[pair]], cell_of_slot[order[pair + 1]]
    own_i, nei_i = np.minimum(ca, cb), np.maximum(ca, cb)
    fvi = fv[order[pair]]
    own_b = cell_of_slot[order[single]]
    fvb = fv[order[single]]

    def geom(fverts, own):
        A, B, Cc = P[fverts[:, 0]], P[fverts[:, 1]], P[fverts[:, 2]]
        S = 0.5 * np.cross(B - A, Cc - A)
        Xf = (A + B + Cc) / 3.0
        sgn = np.sign(np.einsum("ij,ij->i", S, Xf - C[own]))
        assert np.all(sgn != 0)
        oriented = np.where(sgn[:, None] > 0, fverts, fverts[:, ::-1])
        return S * sgn[:, None], Xf, oriented

    S_i, X_i, fvi_o = geom(fvi, own_i)
    S_b, X_b, fvb_o = geom(fvb, own_b)
    types = dict(x0=WALL, x1=WALL, y0=WALL, y1=WALL, z0=WALL, z1=WALL)
    if patch_types:
        types.update(patch_types)
    groups, names, gfv = [], [], []
    tol = 1e-9
    for ax, (lo, hi) in enumerate([("x0", "x1"), ("y0", "y1"), ("z0", "z1")]):
        for name, val in ((lo, 0.0), (hi, 1.0)):
            sel = np.abs(X_b[:, ax] - val) < tol
            groups.append((own_b[sel], S_b[sel], X_b[sel])); names.append(name)
            gfv.append(fvb_o[sel])
    assert sum(g[0].shape[0] for g in groups) == own_b.shape[0] == 12 * n * n
    return _finish(nc, own_i, nei_i, S_i, X_i, V, C, groups, names,
                   [types[nm] for nm in names], topo=(P, fvi_o, gfv))


# ---------------------------------------------------------------------------
# extruded quad meshes: O-H grid pipe, smoothly distorted box
# ---------------------------------------------------------------------------
def extrude_quads(xy, quads, n_layers, Lz, edge_patch, edge_patch_names, edge_patch_types,
                  bottom=("z0", WALL), top=("z1", WALL)) -> Mesh:
    """Extrude a planar quad mesh (counter-clockwise quads) in uniform z layers.

    Cells are prisms over the quads, so every face is planar (horizontal quads
    and vertical trapezoids) and its area vector and centroid are exact.
    ``edge_patch(mid_xy) -> int`` assigns each 2D boundary edge (by its
    midpoint) to one of the side patches.  Patch order: side patches, bottom, top.
    """
    quads = np.asarray(quads, np.int64)
    nq2 = quads.shape[0]
    Q = xy[quads]
    x0, y0 = Q[..., 0], Q[..., 1]
    x1, y1 = np.roll(x0, -1, 1), np.roll(y0, -1, 1)
    cr = x0 * y1 - x1 * y0
    A2 = 0.5 * cr.sum(1)
    assert np.all(A2 > 0), "quads must be counter-clockwise and non-degenerate"
    cxq = ((x0 + x1) * cr).sum(1) / (6 * A2)
    cyq = ((y0 + y1) * cr).sum(1) / (6 * A2)
    ed = np.stack([quads, np.roll(quads, -1, 1)], 2).reshape(-1, 2)
    eq = np.repeat(np.arange(nq2), 4)
    es = np.sort(ed, 1)
    nv2 = xy.shape[0]
    key = es[:, 0] * nv2 + es[:, 1]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    first = np.ones(ks.shape[0], bool); first[1:] = ks[1:] != ks[:-1]
    st = np.flatnonzero(first)
    cnt = np.diff(np.append(st, ks.shape[0]))
    assert cnt.max() <= 2
    pair, single = st[cnt == 2], st[cnt == 1]
    dz = Lz / n_layers
    nc = nq2 * n_layers
    cell = lambda q, l: q + nq2 * l
    lay = np.repeat(np.arange(n_layers), nq2)
    C = np.stack([np.tile(cxq, n_layers), np.tile(cyq, n_layers), (lay + 0.5) * dz], 1)
    V = np.tile(A2, n_layers) * dz

    P3 = np.concatenate([np.concatenate([xy, np.full((nv2, 1), l * dz)], 1) for l in range(n_layers + 1)])
    vtx = lambda v, l: v + nv2 * l    # vertex v of the 2D mesh on plane z = l dz

    def side_v(slot, l):                 # (a, l) (b, l) (b, l+1) (a, l+1): normal out of the first quad
        e = ed[order[slot]]
        return np.stack([vtx(e[:, 0], l), vtx(e[:, 1], l), vtx(e[:, 1], l + 1), vtx(e[:, 0], l + 1)], 1)

    def side(slot, l):
        e = ed[order[slot]]              # directed edge as seen from its first quad
        pa, pb = xy[e[:, 0]], xy[e[:, 1]]
        t2 = pb - pa
        S = np.stack([t2[:, 1] * dz, -t2[:, 0] * dz, np.zeros(len(e))], 1)   # outward of a CCW polygon
        X = np.stack([0.5 * (pa[:, 0] + pb[:, 0]), 0.5 * (pa[:, 1] + pb[:, 1]),
                      np.full(len(e), (l + 0.5) * dz)], 1)
        return S, X

    own, nei, S, X, FV = [], [], [], [], []
    qa, qb = eq[order[pair]], eq[order[pair + 1]]
    for l in range(n_layers):
        Sl, Xl = side(pair, l)
        own.append(cell(qa, l)); nei.append(cell(qb, l)); S.append(Sl); X.append(Xl)
        FV.append(side_v(pair, l))
    zero = np.zeros(nq2)
    for l in range(n_layers - 1):
        own.append(cell(np.arange(nq2), l)); nei.append(cell(np.arange(nq2), l + 1))
        S.append(np.stack([zero, zero, A2], 1))
        X.append(np.stack([cxq, cyq, np.full(nq2, (l + 1) * dz)], 1))
        FV.append(vtx(quads, l + 1))     # counter-clockwise: normal +z, out of the lower cell
    own_i, nei_i = np.concatenate(own), np.concatenate(nei)
    S_i, X_i = np.concatenate(S), np.concatenate(X)
    FV_i = np.concatenate(FV)
    flip = own_i > nei_i
    own_i, nei_i = np.where(flip, nei_i, own_i), np.where(flip, own_i, nei_i)
    S_i[flip] *= -1
    FV_i[flip] = FV_i[flip][:, ::-1]
    wq = eq[order[single]]
    e_single = ed[order[single]]
    mids = 0.5 * (xy[e_single[:, 0]] + xy[e_single[:, 1]])
    pid = np.array([edge_patch(mid) for mid in mids], np.int64)
    groups, names, types, gfv = [], [], [], []
    for p, (nm, tp) in enumerate(zip(edge_patch_names, edge_patch_types)):
        sel = pid == p
        wo, wS, wX, wv = [], [], [], []
        for l in range(n_layers):
            Sl, Xl = side(single[sel], l)
            wo.append(cell(wq[sel], l)); wS.append(Sl); wX.append(Xl); wv.append(side_v(single[sel], l))
        groups.append((np.concatenate(wo), np.concatenate(wS), np.concatenate(wX)))
        names.append(nm); types.append(tp)
        gfv.append(np.concatenate(wv) if wv else np.zeros((0, 4), np.int64))
    groups.append((cell(np.arange(nq2), 0), np.stack([zero, zero, -A2], 1),
                   np.stack([cxq, cyq, np.zeros(nq2)], 1)))
    groups.append((cell(np.arange(nq2), n_layers - 1), np.stack([zero, zero, A2], 1),
                   np.stack([cxq, cyq, np.full(nq2, Lz)], 1)))
    gfv += [vtx(quads, 0)[:, ::-1], vtx(quads, n_layers)]
    names += [bottom[0], top[0]]; types += [bottom[1], top[1]]
    return _finish(nc, own_i, nei_i, S_i, X_i, V, C, groups, names, types, topo=(P3, FV_i, gfv))


def pipe_ohgrid(n_core=16, n_outer=8, n_layers=200, R=1.0, L=10.0, core_frac=0.5,
                outlet_type=OUTLET) -> Mesh:
    """Straight cylinder of radius R and length L along z (O-H grid).

    Cross-section: an n_core x n_core square core of half-width core_frac*R
    and four outer blocks of n_core x n_outer quads that map each square edge
    linearly onto a quarter of the circle (4*n_core boundary points), extruded
    in n_layers uniform layers.  Patches: wall, inlet (z=0), outlet (z=L).
    """
    a = core_frac * R
    nq = 4 * n_core
    t = np.linspace(-a, a, n_core + 1)
    cx, cy = np.meshgrid(t, t, indexing="xy")
    core_xy = np.stack([cx.ravel(), cy.ravel()], 1)
    cidx = lambda i, j: i + (n_core + 1) * j
    per = ([(n_core, s) for s in range(n_core)] + [(n_core - s, n_core) for s in range(n_core)]
           + [(0, n_core - s) for s in range(n_core)] + [(s, 0) for s in range(n_core)])
    per_idx = np.array([cidx(i, j) for i, j in per])     # counter-clockwise from (a,-a)
    sq = core_xy[per_idx]
    k = np.arange(nq)
    theta = np.deg2rad(-45.0 + 90.0 * (k // n_core) + 90.0 * (k % n_core) / n_core)
    circ = R * np.stack([np.cos(theta), np.sin(theta)], 1)
    ncore_v = core_xy.shape[0]
    xy = np.concatenate([core_xy] + [(1 - r / n_outer) * sq + (r / n_outer) * circ
                                     for r in range(1, n_outer + 1)])
    rid = lambda r, k: per_idx[k % nq] if r == 0 else ncore_v + (r - 1) * nq + (k % nq)
    quads = [[cidx(i, j), cidx(i + 1, j), cidx(i + 1, j + 1), cidx(i, j + 1)]
             for j in range(n_core) for i in range(n_core)]
    quads += [[rid(r, kk), rid(r + 1, kk), rid(r + 1, kk + 1), rid(r, kk + 1)]
              for r in range(n_outer) for kk in range(nq)]
    return extrude_quads(xy, quads, n_layers, L, lambda mid: 0, ["wall"], [WALL],
                         bottom=("inlet", INLET), top=("outlet", outlet_type))


def pipe_inflow(mesh: Mesh):
    """Inlet boundary velocities of unit flux for an O-H pipe: a parabolic
    profile in the face-centre radius (kept positive on every inlet face),
    along +z, scaled so that sum_f u_f |S_f| = 1 over the inlet.  Returns
    [3, n_boundary] (zero off the inlet); multiply by Q(t) for the flow Q."""
    fin = mesh.patch_faces("inlet")
    r2 = mesh.Cf[fin, 0] ** 2 + mesh.Cf[fin, 1] ** 2
    shape = 1.0 - r2 / r2.max() * 0.999
    area = np.linalg.norm(mesh.Sf[fin], axis=1)
    ub = np.zeros((3, mesh.n_boundary))
    ub[2, fin - mesh.n_internal] = shape / (shape * area).sum()
    return ub


def pulsatile_flow(t: float) -> float:
    """Inlet flow of the pulsatile pipe: Q(t) = 1 + 0.5 sin 2 pi t + 0.2 sin 4 pi t."""
    return 1.0 + 0.5 * np.sin(2 * np.pi * t) + 0.2 * np.sin(4 * np.pi * t)


def distorted_box(n: int, eps: float = 0.05, nz: int = None, patch_types=None) -> Mesh:
    """Unit cube of n x n x nz prisms whose x-y grid is smoothly distorted.

    Vertex map (x, y) -> (x + eps sin(2 pi x) sin(2 pi y), y + eps sin(2 pi x) sin(2 pi y)):
    a fixed smooth map, so refinement converges to it; boundary vertices stay on
    the square.  Faces are planar and non-orthogonal in x-y.  Patches
    x0,x1,y0,y1,z0,z1 as in ``hex_box``.
    """
    nz = n if nz is None else nz
    g = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")
    s = eps * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    xy = np.stack([(X + s).ravel(), (Y + s).ravel()], 1)
    vid = lambda i, j: i + (n + 1) * j
    quads = [[vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)]
             for j in range(n) for i in range(n)]
    types = dict(x0=WALL, x1=WALL, y0=WALL, y1=WALL, z0=WALL, z1=WALL)
    if patch_types:
        types.update(patch_types)

    def side(mid):
        if abs(mid[0]) < 1e-12: return 0
        if abs(mid[0] - 1) < 1e-12: return 1
        if abs(mid[1]) < 1e-12: return 2
        return 3
    return extrude_quads(xy, quads, nz, 1.0, side, ["x0", "x1", "y0", "y1"],
                         [types[k] for k in ("x0", "x1", "y0", "y1")],
                         bottom=("z0", types["z0"]), top=("z1", types["z1"]))


# ---------------------------------------------------------------------------
# seeded fields
# ---------------------------------------------------------------------------
def random_fields(mesh: Mesh, seed: int = 0):
    """phi [nc], U [3,nc], m [nf], phi_b [nb], U_b [3,nb], all ~N(0,1)."""
    rng = np.random.default_rng(seed)
    nc, nf, nb = mesh.n_cells, mesh.n_faces, mesh.n_boundary
    return dict(
        phi=rng.standard_normal(nc), U=rng.standard_normal((3, nc)),
        m=rng.standard_normal(nf), phi_b=rng.standard_normal(nb),
        U_b=rng.standard_normal((3, nb)),
    )
