"""Pins of the oracle's diagonal incomplete LU (DILU), the incomplete factorisation
(Sec. 2.6.1 preconditions the solvers with ILU) in its form for the non-symmetric
momentum matrix.

For an LDU matrix A (row O of an internal face holds U_f in column N, row N holds
L_f in column O) and an elimination order, DILU builds
M = (Dd + Lo) Dd^-1 (Dd + Up), Lo / Up the strictly lower / upper parts of A in
that order, with d chosen so that M equals A on the diagonal and on A's
off-diagonal pattern.  The pins: that defining property on a 3-D mesh in a random
order (fill-in present, so M != A), the symmetric case reducing to the DIC
factor, exactness on a chain (no fill-in: M = A, one BiCGStab iteration), the
preconditioner's application against a dense solve with M, and the
DILU-preconditioned BiCGStab against a dense solve with A.
"""
import numpy as np

import oracle as O
from paper_2603_15920_b300 import meshgen as mg


def _nonsym(m, seed, shift=0.05):
    """A diagonally dominant convection-diffusion-like LDU matrix."""
    om = O.OMesh.from_mesh(m)
    w, c, k = O.face_coeffs(om)
    rng = np.random.default_rng(seed)
    ni = m.n_internal
    a = c[:ni] * rng.uniform(0.5, 2.0, ni)
    mf = rng.normal(size=ni) * a.mean()
    L = -a - np.maximum(mf, 0.0)          # row N, column O
    U = -a + np.minimum(mf, 0.0)          # row O, column N
    D = (np.bincount(m.owner[:ni], -U, m.n_cells) + np.bincount(m.neighbour, -L, m.n_cells)
         + shift * m.V * a.mean() / m.V.mean())
    return om, D, L, U


def _dense(m, D, L, U):
    A = np.diag(D)
    o, n = m.owner[:m.n_internal], m.neighbour
    A[o, n] += U
    A[n, o] += L
    return A


def _M(m, d, A, rank):
    """(Dd + Lo) Dd^-1 (Dd + Up) from A's entries and the order."""
    lower = rank[:, None] > rank[None, :]
    Lo = np.where(lower, A, 0.0)
    Up = np.where(lower.T, A, 0.0)
    np.fill_diagonal(Lo, 0.0)
    np.fill_diagonal(Up, 0.0)
    Dd = np.diag(d)
    return (Dd + Lo) @ np.diag(1.0 / d) @ (Dd + Up)


def test_dilu_matches_matrix_on_diagonal_and_pattern():
    m = mg.shuffle(mg.kuhn_cube(3, 0.2, 7), 8)
    om, D, L, U = _nonsym(m, 1)
    rank = np.random.default_rng(3).permutation(m.n_cells).astype(np.int32)
    d = O.dilu_factor(om, D, L, U, rank)
    A = _dense(m, D, L, U)
    M = _M(m, d, A, rank)
    pattern = A != 0
    np.testing.assert_allclose(M[pattern], A[pattern], rtol=1e-12, atol=1e-12 * np.abs(A).max())
    assert np.abs(M - A).max() > 1e-3 * np.abs(A).max()     # fill-in dropped: M is not A
    assert not np.allclose(A, A.T)                           # a non-symmetric case


def test_dilu_of_a_symmetric_matrix_is_dic():
    m = mg.shuffle(mg.kuhn_cube(3, 0.2, 9), 10)
    om, D, L, _ = _nonsym(m, 2)
    rank = np.random.default_rng(4).permutation(m.n_cells).astype(np.int32)
    np.testing.assert_array_equal(O.dilu_factor(om, D, L, L, rank), O.dic_factor(om, D, L, rank))


def test_dilu_is_exact_without_fill_in():
    m = mg.hex_box(12, 1, 1)                                 # a chain of cells
    om, D, L, U = _nonsym(m, 5)
    rank = np.arange(m.n_cells, dtype=np.int32)
    A = _dense(m, D, L, U)
    b = np.random.default_rng(6).normal(size=m.n_cells)
    z = O.dilu_apply(om, D, L, U, rank, b)
    np.testing.assert_allclose(z, np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)
    x, info = O.bicgstab_dilu(om, D, L, U, b, rank, tol_rel=1e-12)
    assert info["status"] == 0 and info["iters"] == 1


def test_dilu_apply_is_the_inverse_of_M():
    m = mg.shuffle(mg.kuhn_cube(3, 0.2, 11), 12)
    om, D, L, U = _nonsym(m, 7)
    rank = np.random.default_rng(8).permutation(m.n_cells).astype(np.int32)
    r = np.random.default_rng(9).normal(size=m.n_cells)
    M = _M(m, O.dilu_factor(om, D, L, U, rank), _dense(m, D, L, U), rank)
    np.testing.assert_allclose(O.dilu_apply(om, D, L, U, rank, r), np.linalg.solve(M, r), rtol=1e-10,
                               atol=1e-12)


def test_bicgstab_dilu_solves_the_system():
    m = mg.shuffle(mg.kuhn_cube(4, 0.2, 13), 14)
    om, D, L, U = _nonsym(m, 9)
    rank = np.arange(m.n_cells, dtype=np.int32)
    b = np.random.default_rng(10).normal(size=m.n_cells)
    x, info = O.bicgstab_dilu(om, D, L, U, b, rank, tol_rel=1e-13)
    ref = np.linalg.solve(_dense(m, D, L, U), b)
    assert info["status"] == 0
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
    _, ij = O.bicgstab(om, D, L, U, b, tol_rel=1e-13)
    assert info["iters"] < ij["iters"]                     # a better preconditioner than Jacobi
