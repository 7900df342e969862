"""Polyhedral geometry and the OpenFOAM polyMesh reader / writer.

The oracle's geometry (divergence theorem and polygon fans, ``oracle.polymesh_geometry``)
is pinned against closed forms (a unit cube, a tetrahedron, a prism over a
non-convex L-shaped base) and against the exact geometry that the mesh
generators compute from their own formulas; the library's geometry
(``difvm_polymesh_geometry``: triangles around the face's vertex average,
pyramids around the cell's face-centroid average; host code) is compared with
the oracle's (1e-13, relative).  Files written by ``write_polymesh`` read back
to the same topology; a hand-written polyMesh in OpenFOAM syntax parses.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2603_15920_b300 import meshgen as mg
from paper_2603_15920_b300 import polymesh as pm


def nrel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _single_cell(points, faces):
    """One closed cell: faces as vertex loops with outward right-hand normals."""
    fp = np.concatenate([[0], np.cumsum([len(f) for f in faces])]).astype(np.int32)
    fv = np.concatenate(faces).astype(np.int32)
    own = np.zeros(len(faces), np.int32)
    return np.asarray(points, np.float64), fp, fv, own, np.zeros(0, np.int32)


def _cube():
    P = [(x, y, z) for z in (0, 1) for y in (0, 1) for x in (0, 1)]
    faces = [[0, 2, 3, 1], [4, 5, 7, 6], [0, 1, 5, 4], [2, 6, 7, 3], [0, 4, 6, 2], [1, 3, 7, 5]]
    return _single_cell(P, faces)


def _l_prism(h=0.7):
    # L-shaped base (a 2x2 square minus its upper-right unit square), extruded to height h
    base = [(0, 0), (2, 0), (2, 1), (1, 1), (1, 2), (0, 2)]
    P = [(x, y, 0.0) for x, y in base] + [(x, y, h) for x, y in base]
    n = len(base)
    faces = [list(range(n))[::-1], list(range(n, 2 * n))]
    faces += [[k, (k + 1) % n, n + (k + 1) % n, n + k] for k in range(n)]
    return _single_cell(P, faces)


def test_oracle_geometry_closed_forms():
    S, X, V, C = O.polymesh_geometry(*_cube()[:3], *_cube()[3:], 1)
    np.testing.assert_allclose(V, [1.0], rtol=1e-15)
    np.testing.assert_allclose(C, [[0.5, 0.5, 0.5]], atol=1e-15)
    np.testing.assert_allclose(np.abs(S).sum(axis=1), 1.0, rtol=1e-15)
    assert np.abs(S.sum(axis=0)).max() < 1e-15          # a closed surface
    # tetrahedron: V = |det| / 6, centroid = vertex mean
    P = np.array([[0.1, 0.2, 0.0], [1.3, 0.1, 0.2], [0.4, 1.1, 0.1], [0.3, 0.5, 0.9]])
    faces = [[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]]
    S, X, V, C = O.polymesh_geometry(*_single_cell(P, faces)[:3], *_single_cell(P, faces)[3:], 1)
    np.testing.assert_allclose(V, [abs(np.linalg.det(P[1:] - P[0])) / 6], rtol=1e-14)
    np.testing.assert_allclose(C[0], P.mean(axis=0), rtol=1e-14)
    # prism over a non-convex L: volume = 3 h; base centroid (5/6, 5/6), mid-height
    h = 0.7
    S, X, V, C = O.polymesh_geometry(*_l_prism(h)[:3], *_l_prism(h)[3:], 1)
    np.testing.assert_allclose(V, [3 * h], rtol=1e-14)
    np.testing.assert_allclose(C[0], [5 / 6, 5 / 6, h / 2], rtol=1e-14)
    np.testing.assert_allclose(X[0], [5 / 6, 5 / 6, 0.0], atol=1e-15)


GENERATED = {
    "kuhn_jittered": lambda: mg.kuhn_cube(4, 0.25, 3),
    "distorted_prisms": lambda: mg.distorted_box(5, 0.05, 3),
    "pipe_ohgrid": lambda: mg.pipe_ohgrid(6, 3, 4),
}


@pytest.mark.parametrize("name", list(GENERATED))
def test_oracle_geometry_matches_generated_meshes(name):
    m = GENERATED[name]()
    S, X, V, C = O.polymesh_geometry(m.points, m.face_ptr, m.face_pts, m.owner, m.neighbour, m.n_cells)
    for got, ref in ((S, m.Sf), (X, m.Cf), (V, m.V), (C, m.C)):
        assert nrel(got, ref) < 1e-13


def _lib_geometry(*a):
    from paper_2603_15920_b300 import difvm as D   # host code of the library
    return D.difvm_polymesh_geometry(*a)


@pytest.mark.parametrize("name", list(GENERATED))
def test_library_geometry_matches_oracle(name):
    m = GENERATED[name]()
    args = (m.points, m.face_ptr, m.face_pts, m.owner, m.neighbour, m.n_cells)
    for got, ref in zip(_lib_geometry(*args), O.polymesh_geometry(*args)):
        assert nrel(got, ref) < 1e-13


def test_library_geometry_closed_forms_and_errors():
    for cell, V0, C0 in ((_cube(), 1.0, [0.5, 0.5, 0.5]), (_l_prism(0.7), 2.1, [5 / 6, 5 / 6, 0.35])):
        S, X, V, C = _lib_geometry(*cell[:3], cell[3], cell[4], 1)
        np.testing.assert_allclose(V, [V0], rtol=1e-14)
        np.testing.assert_allclose(C[0], C0, rtol=1e-14)
    from paper_2603_15920_b300 import difvm as D
    P, fp, fv, own, nei = _cube()
    with pytest.raises(D.DifvmError):       # inward faces: negative volume
        _lib_geometry(P, fp, fv[::-1].copy(), own, nei, 1)
    bad = fv.copy(); bad[0] = 99
    with pytest.raises(D.DifvmError):       # vertex out of range
        _lib_geometry(P, fp, bad, own, nei, 1)


def test_polymesh_roundtrip(tmp_path):
    m = mg.kuhn_cube(3, 0.2, 5, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET))
    d = str(tmp_path / "polyMesh")
    pm.write_polymesh(d, m)
    t = pm.read_polymesh(d)
    assert t["n_cells"] == m.n_cells and t["neighbour"].shape[0] == m.n_internal
    np.testing.assert_array_equal(t["points"], m.points)
    assert [(p[0], p[2], p[3]) for p in t["patches"]] == [
        (nm, int(s), int(z)) for nm, s, z in zip(m.patch_names, m.patch_start, m.patch_size)]
    # the same faces (as vertex loops with owner / neighbour), internal ones sorted by owner
    loops = lambda fp, fv, f: tuple(fv[fp[f]:fp[f + 1]])
    ref = {(loops(m.face_ptr, m.face_pts, f), int(m.owner[f]), int(m.neighbour[f]) if f < m.n_internal else -1)
           for f in range(m.n_faces)}
    got = {(loops(t["face_ptr"], t["face_pts"], f), int(t["owner"][f]),
            int(t["neighbour"][f]) if f < m.n_internal else -1) for f in range(m.n_faces)}
    assert got == ref
    assert np.all(np.diff(t["owner"][:m.n_internal]) >= 0)


def test_load_mesh_geometry_and_patch_types(tmp_path):
    m = mg.distorted_box(4, 0.05, 3, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET))
    d = str(tmp_path / "polyMesh")
    pm.write_polymesh(d, m)
    lm = pm.load_mesh(d, patch_types=dict(x0=mg.INLET, x1=mg.OUTLET))
    assert list(lm.patch_type) == list(m.patch_type)
    # face order: internal faces sorted by owner; compare through the (owner, neighbour) key
    key = lambda mm: np.lexsort((mm.neighbour, mm.owner[:mm.n_internal]))
    ka, kb = key(m), key(lm)
    assert nrel(lm.Sf[:lm.n_internal][kb], m.Sf[:m.n_internal][ka]) < 1e-13
    assert nrel(lm.Sf[lm.n_internal:], m.Sf[m.n_internal:]) < 1e-13
    assert nrel(lm.V, m.V) < 1e-13 and nrel(lm.C, m.C) < 1e-13


FOAM_TEXT = {
    "points": """/*--------------------------------*- C++ -*----------------------------------*\\
  a hand-written two-hex mesh
\\*---------------------------------------------------------------------------*/
FoamFile
{
    version     2.0;
    format      ascii;
    class       vectorField;
    object      points;
}
// * * * * * * * * * * //

12
(
(0 0 0) (1 0 0) (2 0 0)
(0 1 0) (1 1 0) (2 1 0)
(0 0 1) (1 0 1) (2 0 1)
(0 1 1) (1 1 1) (2 1 1)
)
""",
    "faces": """FoamFile { version 2.0; format ascii; class faceList; object faces; }
11
(
4(1 4 10 7)
4(0 6 9 3)
4(2 5 11 8)
4(0 1 7 6)
4(1 2 8 7)
4(3 9 10 4)
4(4 10 11 5)
4(0 3 4 1)
4(1 4 5 2)
4(6 7 10 9)
4(7 8 11 10)
)
""",
    "owner": """FoamFile { version 2.0; format ascii; class labelList; object owner; }
// note: nPoints 12 nCells 2 nFaces 11 nInternalFaces 1
11 ( 0 0 1 0 1 0 1 0 1 0 1 )
""",
    "neighbour": """FoamFile { version 2.0; format ascii; class labelList; object neighbour; }
1
(
1
)
""",
    "boundary": """FoamFile { version 2.0; format ascii; class polyBoundaryMesh; object boundary; }
3
(
    inlet
    {
        type            patch;
        nFaces          1;
        startFace       1;
    }
    outlet
    {
        type            patch;
        nFaces          1;
        startFace       2;
    }
    walls
    {
        type            wall;
        inGroups        List<word> 1(wall);
        nFaces          8;
        startFace       3;
    }
)
""",
}


def test_read_openfoam_syntax(tmp_path):
    d = tmp_path / "polyMesh"
    d.mkdir()
    for name, text in FOAM_TEXT.items():
        (d / name).write_text(text)
    t = pm.read_polymesh(str(d))
    assert t["n_cells"] == 2 and t["points"].shape == (12, 3) and t["face_ptr"][-1] == 44
    assert [p[:2] for p in t["patches"]] == [("inlet", "patch"), ("outlet", "patch"), ("walls", "wall")]
    lm = pm.load_mesh(str(d), patch_types=dict(inlet=mg.INLET, outlet=mg.OUTLET))
    np.testing.assert_allclose(lm.V, [1.0, 1.0], rtol=1e-15)
    np.testing.assert_allclose(lm.C, [[0.5, 0.5, 0.5], [1.5, 0.5, 0.5]], rtol=1e-15)
    np.testing.assert_allclose(lm.Sf[0], [1, 0, 0], atol=1e-15)      # owner 0 -> neighbour 1
    assert list(lm.patch_type) == [mg.INLET, mg.OUTLET, mg.WALL]
