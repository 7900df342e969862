"""The multi-core build of the oracle (the all-cores CPU baseline) against the
single-thread oracle.

The multi-core build runs the same source with OpenMP: its LDU apply sums each
cell's faces in ascending face id (bitwise the face loop's sums) and its inner
products add fixed blocks, so a PISO step must not depend on the thread count
(bitwise) and must agree with the single-thread oracle to solver tolerance.
"""
import numpy as np

import oracle as O
from paper_2603_15920_b300 import meshgen as mg


def _cavity():
    m = mg.shuffle(mg.kuhn_cube(6, 0.2, 3), 4)
    om = O.OMesh.from_mesh(m)
    Ub = np.zeros((3, m.n_boundary))
    Ub[0, m.patch_faces("y1") - m.n_internal] = 1.0
    U, p, pb = np.zeros((3, m.n_cells)), np.zeros(m.n_cells), np.zeros(m.n_boundary)
    return m, om, U, p, O.flux_from_U(om, U, Ub), Ub, pb


def _steps(om, U, p, phi, Ub, pb, n=3):
    kw = dict(nu=0.01, dt=0.02, tolU=1e-12, tolp=1e-12, pref_cell=0, nonorth=1)
    for _ in range(n):
        U, p, phi, pb, _, _ = O.piso_step(om, U, p, phi, Ub, pb, **kw)
    return U, p, phi


def test_ldu_apply_multicore_is_bitwise_the_face_loop():
    m, om, *_ = _cavity()
    rng = np.random.default_rng(0)
    D, L, U = rng.standard_normal(m.n_cells), rng.standard_normal(m.n_internal), rng.standard_normal(m.n_internal)
    x = rng.standard_normal((2, m.n_cells))
    try:
        O.use_multicore(False)
        y1 = O.ldu_apply(om, D, L, U, x)
        O.use_multicore(True)
        O.set_threads(3)
        y2 = O.ldu_apply(om, D, L, U, x)
    finally:
        O.use_multicore(False)
    assert np.array_equal(y1, y2)


def test_piso_step_multicore_matches_single_thread():
    m, om, U, p, phi, Ub, pb = _cavity()
    try:
        O.use_multicore(False)
        assert O.threads() == 1
        ref = _steps(om, U, p, phi, Ub, pb)
        O.use_multicore(True)
        O.set_threads(1)
        a = _steps(om, U, p, phi, Ub, pb)
        O.set_threads(4)
        assert O.threads() == 4
        b = _steps(om, U, p, phi, Ub, pb)
    finally:
        O.use_multicore(False)
    for x, y, r in zip(a, b, ref):
        assert np.array_equal(x, y)                       # independent of the thread count
        assert np.abs(x - r).max() <= 1e-9 * np.abs(r).max()
