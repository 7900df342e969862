"""OpenFOAM polyMesh input and output (ASCII), so that meshes made elsewhere can
be run (the paper's meshes are OpenFOAM cases, Sec. 3; every element type of
Sec. 1: tetrahedra, hexahedra, prisms, pyramids, polyhedra).

A polyMesh directory holds ``points`` (vectorField), ``faces`` (faceList),
``owner`` and ``neighbour`` (labelList) and ``boundary`` (patch dictionary).
Internal faces come first (owner < neighbour, the face's right-hand normal
pointing from owner to neighbour), then each patch's faces in one contiguous
range.  ``read_polymesh`` parses that layout; ``load_mesh`` adds the geometry
(``difvm_polymesh_geometry`` of the library) and returns a ``meshgen.Mesh``
ready for ``difvm.Mesh``; ``write_polymesh`` writes a mesh that carries its
vertex topology.

Patch types: ``empty`` -> EMPTY; any other patch takes the solver type given
for its name in ``patch_types`` (WALL, INLET, OUTLET or EMPTY), WALL when not
given (a polyMesh names the patch kind, the boundary conditions live
elsewhere in an OpenFOAM case).
"""
from __future__ import annotations

import os
import re

import numpy as np

from . import meshgen as mg

_HEADER = """FoamFile
{{
    version     2.0;
    format      ascii;
    class       {cls};
    location    "constant/polyMesh";
    object      {obj};
}}
"""


def _strip(text: str) -> str:
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    m = re.search(r"FoamFile\s*\{", text)
    if m:   # drop the header dictionary
        depth, i = 1, m.end()
        while depth:
            depth += {"{": 1, "}": -1}.get(text[i], 0)
            i += 1
        text = text[i:]
    return text


def _list_body(text: str, what: str):
    """(count, body between the outermost parentheses) of an ASCII list."""
    m = re.search(r"(\d+)\s*\(", text)
    if not m:
        raise ValueError(f"{what}: no list found")
    n, start = int(m.group(1)), m.end()
    depth, i = 1, start
    while depth:
        if i >= len(text):
            raise ValueError(f"{what}: unbalanced parentheses")
        c = text[i]
        depth += 1 if c == "(" else (-1 if c == ")" else 0)
        i += 1
    return n, text[start:i - 1]


def _read(path):
    with open(path) as f:
        return _strip(f.read())


def read_polymesh(directory: str) -> dict:
    """Topology of a polyMesh directory: points [np,3], face_ptr [nf+1],
    face_pts, owner [nf], neighbour [ni], n_cells and the patches as
    (name, type, start_face, n_faces)."""
    n, body = _list_body(_read(os.path.join(directory, "points")), "points")
    pts = np.array(body.replace("(", " ").replace(")", " ").split(), np.float64)
    if pts.shape[0] != 3 * n:
        raise ValueError(f"points: {pts.shape[0]} numbers for {n} points")
    points = pts.reshape(n, 3)

    nf, body = _list_body(_read(os.path.join(directory, "faces")), "faces")
    tok = np.array(body.replace("(", " ").replace(")", " ").split(), np.int64)
    # each face: its vertex count, then the vertices; walk the counts (a plain
    # list is several times faster to step through than the array)
    tl = tok.tolist()
    cpos = np.empty(nf, np.int64)
    pos = 0
    for f in range(nf):
        if pos >= len(tl):
            raise ValueError("faces: vertex counts do not match the list")
        cpos[f] = pos
        pos += 1 + tl[pos]
    if pos != len(tl):
        raise ValueError("faces: vertex counts do not match the list")
    counts = tok[cpos]
    keep = np.ones(tok.shape[0], bool)
    keep[cpos] = False                 # drop the count tokens: the rest are the loops in order
    face_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    face_pts = tok[keep].astype(np.int32)

    no, body = _list_body(_read(os.path.join(directory, "owner")), "owner")
    owner = np.array(body.split(), np.int32)
    nn, body = _list_body(_read(os.path.join(directory, "neighbour")), "neighbour")
    neighbour = np.array(body.split(), np.int32) if nn else np.zeros(0, np.int32)
    if owner.shape[0] != nf or no != nf or neighbour.shape[0] != nn:
        raise ValueError("owner / neighbour sizes do not match the faces")

    _, body = _list_body(_read(os.path.join(directory, "boundary")), "boundary")
    patches = []
    for name, d in re.findall(r"([A-Za-z0-9_.:\-]+)\s*\{([^{}]*)\}", body):
        kv = dict(re.findall(r"(\w+)\s+([^;]+);", d))
        patches.append((name, kv.get("type", "patch").strip(), int(kv["startFace"]), int(kv["nFaces"])))
    patches.sort(key=lambda p: p[2])
    n_cells = int(max(owner.max(), neighbour.max() if nn else -1)) + 1
    return dict(points=points, face_ptr=face_ptr, face_pts=face_pts, owner=owner, neighbour=neighbour,
                n_cells=n_cells, patches=patches)


def load_mesh(directory: str, patch_types: dict | None = None) -> mg.Mesh:
    """A polyMesh directory as a ``meshgen.Mesh`` with its geometry computed by
    the library (``difvm_polymesh_geometry``) and its vertex topology kept."""
    from . import difvm as D   # the geometry is native code
    t = read_polymesh(directory)
    ni = int(t["neighbour"].shape[0])
    nf = int(t["owner"].shape[0])
    expect = ni
    for name, _, start, size in t["patches"]:
        if start != expect:
            raise ValueError(f"patch {name} starts at face {start}, expected {expect}")
        expect += size
    if expect != nf:
        raise ValueError(f"patches cover faces up to {expect} of {nf}")
    Sf, Cf, V, C = D.difvm_polymesh_geometry(t["points"], t["face_ptr"], t["face_pts"], t["owner"],
                                             t["neighbour"], t["n_cells"])
    types = [mg.EMPTY if ftype == "empty" else (patch_types or {}).get(name, mg.WALL)
             for name, ftype, _, _ in t["patches"]]
    m = mg.Mesh(n_cells=t["n_cells"], n_internal=ni, owner=t["owner"], neighbour=t["neighbour"],
                Sf=Sf, Cf=Cf, V=V, C=C, patch_names=[p[0] for p in t["patches"]],
                patch_start=np.array([p[2] for p in t["patches"]], np.int32),
                patch_size=np.array([p[3] for p in t["patches"]], np.int32),
                patch_type=np.array(types, np.int32), points=t["points"], face_ptr=t["face_ptr"],
                face_pts=t["face_pts"])
    return m.check()


_TYPE_NAME = {mg.WALL: "wall", mg.INLET: "patch", mg.OUTLET: "patch", mg.EMPTY: "empty"}


def write_polymesh(directory: str, m: mg.Mesh) -> None:
    """Write a mesh that carries its vertex topology (``points``, ``face_ptr``,
    ``face_pts``) as an ASCII polyMesh.  Internal faces must have owner <
    neighbour (re-oriented otherwise, with their vertex loops reversed)."""
    if m.points is None:
        raise ValueError("the mesh has no vertex topology")
    os.makedirs(directory, exist_ok=True)
    ni, nf = m.n_internal, m.n_faces
    own, nei = m.owner.astype(np.int64).copy(), m.neighbour.astype(np.int64).copy()
    loops = [m.face_pts[m.face_ptr[f]:m.face_ptr[f + 1]] for f in range(nf)]
    for f in np.flatnonzero(own[:ni] > nei):
        own[f], nei[f] = nei[f], own[f]
        loops[f] = loops[f][::-1]
    # OpenFOAM orders internal faces by owner (upper-triangular order)
    order = np.lexsort((nei, own[:ni]))
    perm = np.concatenate([order, np.arange(ni, nf)])

    def write(name, cls, lines, n):
        with open(os.path.join(directory, name), "w") as f:
            f.write(_HEADER.format(cls=cls, obj=name))
            f.write(f"\n{n}\n(\n")
            f.write("\n".join(lines))
            f.write("\n)\n")

    write("points", "vectorField", [f"({float(x)!r} {float(y)!r} {float(z)!r})" for x, y, z in m.points],
          m.points.shape[0])
    write("faces", "faceList", [f"{len(loops[f])}({' '.join(str(int(v)) for v in loops[f])})" for f in perm], nf)
    write("owner", "labelList", [str(int(own[f])) for f in perm], nf)
    write("neighbour", "labelList", [str(int(nei[f])) for f in order], ni)
    entries = []
    for p, name in enumerate(m.patch_names):
        entries.append(f"    {name}\n    {{\n        type            {_TYPE_NAME[int(m.patch_type[p])]};\n"
                       f"        nFaces          {int(m.patch_size[p])};\n"
                       f"        startFace       {int(m.patch_start[p])};\n    }}")
    write("boundary", "polyBoundaryMesh", entries, len(entries))
