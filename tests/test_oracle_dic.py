"""Pins of the oracle's diagonal incomplete Cholesky (DIC), the CG preconditioner
the paper names (Sec. 2.6.1).

For a symmetric LDU matrix A and an elimination order, DIC builds
M = (Dd + Lo) Dd^-1 (Dd + Lo^T) with d chosen so that M equals A on the diagonal
and on A's off-diagonal pattern (the fill-in of exact Cholesky is dropped).  The
pins: that defining property on a 3-D mesh in a random order (with fill-in present,
so M != A), exactness on a chain (no fill-in: one CG iteration), and the
DIC-preconditioned CG against a dense solve.
"""
import numpy as np

import oracle as O
from paper_2603_15920_b300 import meshgen as mg


def _spd(m, seed, shift=0.01):
    om = O.OMesh.from_mesh(m)
    w, c, k = O.face_coeffs(om)
    rng = np.random.default_rng(seed)
    a = c[:m.n_internal] * rng.uniform(0.5, 2.0, m.n_internal)
    D = np.bincount(m.owner[:m.n_internal], a, m.n_cells) + np.bincount(m.neighbour, a, m.n_cells) \
        + shift * m.V
    return om, D, -a


def _dense(m, D, L):
    A = np.diag(D)
    o, n = m.owner[:m.n_internal], m.neighbour
    A[o, n] += L
    A[n, o] += L
    return A


def _M(m, d, L, rank):
    nc, ni = m.n_cells, m.n_internal
    o, n = m.owner[:ni], m.neighbour
    lo = np.where(rank[o] < rank[n], o, n)
    hi = np.where(rank[o] < rank[n], n, o)
    F = np.diag(d)
    F[hi, lo] += L                      # Dd + Lo (rows of the later cell)
    return F @ np.diag(1.0 / d) @ F.T


def test_dic_matches_matrix_on_diagonal_and_pattern():
    m = mg.shuffle(mg.kuhn_cube(3, 0.2, 5), 6)
    om, D, L = _spd(m, 1)
    rank = np.random.default_rng(2).permutation(m.n_cells).astype(np.int32)
    d = O.dic_factor(om, D, L, rank)
    A, M = _dense(m, D, L), _M(m, d, L, rank)
    pattern = A != 0
    np.testing.assert_allclose(M[pattern], A[pattern], rtol=1e-12, atol=1e-12 * np.abs(A).max())
    assert np.abs(M - A).max() > 1e-3 * np.abs(A).max()     # fill-in dropped: M is not A
    assert np.all(d > 0)


def test_dic_is_exact_without_fill_in():
    m = mg.hex_box(12, 1, 1)                                 # a chain of cells
    om, D, L = _spd(m, 3)
    rank = np.arange(m.n_cells, dtype=np.int32)
    d = O.dic_factor(om, D, L, rank)
    np.testing.assert_allclose(_M(m, d, L, rank), _dense(m, D, L), rtol=1e-13, atol=1e-14)
    b = np.random.default_rng(4).standard_normal(m.n_cells)
    x, info = O.pcg_dic(om, D, L, b, rank, tol_rel=1e-12)
    assert info["status"] == 0 and info["iters"] == 1


def test_pcg_dic_matches_dense_solve_and_beats_jacobi():
    m = mg.shuffle(mg.kuhn_cube(5, 0.2, 7), 8)
    om, D, L = _spd(m, 5, shift=1e-2)        # cond(A) ~ 3e5
    rank = np.random.default_rng(9).permutation(m.n_cells).astype(np.int32)
    b = np.random.default_rng(10).standard_normal(m.n_cells)
    x, info = O.pcg_dic(om, D, L, b, rank, tol_rel=1e-12)
    A = _dense(m, D, L)
    xd = np.linalg.solve(A, b)
    assert info["status"] == 0
    # the recursive residual stops at 1e-12; the true one within cond(A) eps of it
    assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
    np.testing.assert_allclose(x, xd, atol=1e-9 * np.abs(xd).max())
    xj, ij = O.pcg(om, D, L, None, b, tol_rel=1e-12)
    assert info["iters"] < ij["iters"]
