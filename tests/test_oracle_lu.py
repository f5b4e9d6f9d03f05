"""Pins of the tile LU oracle (incremental pivoting, PLASMA DGETRF of Section 4.1), CPU only.

Each pin is fixed by something other than the oracle itself:
  * one tile (T = 1): GETRF is LAPACK's partial-pivoting LU, so scipy's getrf gives the
    same pivots and factors (after moving the multipliers of each block to LAPACK's row
    order); on column diagonally dominant matrices no interchange happens at any T, and the
    tile factors are LAPACK's L and U across all tiles;
  * A = L U with dyadic L (|l| < 1) and integer U: no interchange can happen and every
    intermediate is exact, so the factors come back bitwise and integer solutions exactly;
  * the recorded transformations reduce A itself to U = triu(F) (the definition of what the
    factor stores), and partial pivoting bounds every multiplier by 1;
  * the solve reaches a backward error at the level of the unit roundoff;
  * the task graph derived from access modes, checked by hand at T = 2.
A mistake in any step (a dropped interchange, a transposed L11, a wrong block offset) breaks
at least the reduction pin, the multiplier bound or the solve.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from oracle import dag
from oracle import lu


def _to_lapack(F, piv, nb, n, ib):
    """(LU, ipiv) in LAPACK's convention for a one-tile factor: the interchanges of block b
    moved onto the multipliers of the blocks before it."""
    LU = F.copy()
    ipiv = np.zeros(n, dtype=np.int64)
    for c0 in range(0, n, ib):
        c1 = min(n, c0 + ib)
        for j in range(c0, c1):
            r = c0 + int(piv[(0, 0)][j])
            ipiv[j] = r
            if r != j:
                LU[[j, r], :c0] = LU[[r, j], :c0]
    return LU, ipiv


@pytest.mark.parametrize("n,ib", [(5, 32), (64, 32), (100, 32), (100, 7), (37, 8)])
def test_one_tile_is_lapack_getrf(n, ib):
    A = synth.general_matrix(n, seed=n).numpy()
    F, piv, Lw, info = lu.lu_incpiv(A, nb=n, ib=ib)
    assert info == 0 and not Lw
    LU, ipiv = _to_lapack(F, piv, n, n, ib)
    ref, ref_piv = scipy.linalg.lu_factor(A)
    np.testing.assert_array_equal(ipiv, ref_piv)
    assert np.abs(LU - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n,nb,ib", [(64, 16, 8), (100, 32, 32), (97, 24, 8), (130, 64, 16)])
def test_dyadic_factor_and_solve_exact(n, nb, ib):
    L, U, A = synth.dyadic_lu(n, seed=n)
    F, piv, Lw, info = lu.lu_incpiv(A, nb=nb, ib=ib)
    assert info == 0
    np.testing.assert_array_equal(np.triu(F), U)
    T = lu.tiles(n, nb)
    for k in range(T):
        for i in range(k, T):
            rows = slice(i * nb, min(n, (i + 1) * nb))
            cols = slice(k * nb, min(n, (k + 1) * nb))
            Lt = F[rows, cols] if i > k else np.tril(F[rows, cols], -1)
            ref = L[rows, cols] if i > k else np.tril(L[rows, cols], -1)
            np.testing.assert_array_equal(Lt, ref)
            np.testing.assert_array_equal(piv[(i, k)], np.arange(cols.stop - cols.start) % ib)
            if i > k:
                assert not Lw[(i, k)].any()
    X = synth.integer_vector(n, 3, seed=n)
    B = A @ X
    np.testing.assert_array_equal(lu.lu_solve(F, piv, Lw, nb, B, ib), X)


@pytest.mark.parametrize("n,nb,ib", [(96, 32, 32), (150, 48, 16), (200, 64, 8), (130, 128, 32)])
def test_column_dominant_matrices_match_lapack_across_tiles(n, nb, ib):
    # strictly column diagonally dominant: the Schur complements stay so, every pivot search
    # keeps the diagonal row, and the tile factors are LAPACK's unpivoted L and U
    G = synth.general_matrix(n, seed=n).numpy()
    A = G + np.diag(np.abs(G).sum(axis=0) + 1.0)
    F, piv, Lw, info = lu.lu_incpiv(A, nb=nb, ib=ib)
    P, L, U = scipy.linalg.lu(A)
    np.testing.assert_array_equal(P, np.eye(n))
    assert info == 0
    assert np.abs(np.triu(F) - U).max() <= 1e-14 * np.abs(U).max()
    assert np.abs(np.tril(F, -1) - np.tril(L, -1)).max() <= 1e-14
    assert all((p == np.arange(len(p)) % ib).all() for p in piv.values())
    assert not any(w.any() for w in Lw.values())


@pytest.mark.parametrize("n,nb,ib", [(96, 32, 32), (100, 32, 8), (150, 48, 16), (77, 77, 32), (70, 16, 32)])
def test_transformations_reduce_A_to_U_and_multipliers_bounded(n, nb, ib):
    A = synth.general_matrix(n, seed=3 * n).numpy()
    F, piv, Lw, info = lu.lu_incpiv(A, nb=nb, ib=ib)
    assert info == 0
    U = np.triu(F)
    MA = lu.forward_transform(F, piv, Lw, nb, A, ib)
    assert np.abs(MA - U).max() <= 1e-12 * np.abs(A).max() * n
    # partial pivoting: every multiplier is at most 1 in magnitude
    T = lu.tiles(n, nb)
    for k in range(T):
        for i in range(k, T):
            rows = slice(i * nb, min(n, (i + 1) * nb))
            cols = slice(k * nb, min(n, (k + 1) * nb))
            Lt = F[rows, cols] if i > k else np.tril(F[rows, cols], -1)
            assert np.abs(Lt).max(initial=0.0) <= 1.0
            if i > k:
                assert np.abs(Lw[(i, k)]).max(initial=0.0) <= 1.0
                assert (piv[(i, k)] >= 0).all()


@pytest.mark.parametrize("n,nb,ib,nrhs", [(200, 64, 32, 3), (130, 32, 8, 1), (256, 256, 32, 2)])
def test_solve_backward_error(n, nb, ib, nrhs):
    A = synth.general_matrix(n, seed=n + 1).numpy()
    B = synth.rhs(n, nrhs, seed=n + 2).numpy()
    F, piv, Lw, info = lu.lu_incpiv(A, nb=nb, ib=ib)
    X = lu.lu_solve(F, piv, Lw, nb, B, ib)
    assert oracle.backward_error(A, X, B) <= 1e-14


def test_planted_missing_interchange_is_caught():
    # a factor whose TSTRF interchanges are dropped fails the reduction pin
    n, nb, ib = 64, 32, 16
    A = synth.general_matrix(n, seed=11).numpy()
    F, piv, Lw, _ = lu.lu_incpiv(A, nb=nb, ib=ib)
    assert any((piv[(1, 0)] != np.arange(nb) % ib))
    bad = dict(piv)
    bad[(1, 0)] = np.arange(nb) % ib
    MA = lu.forward_transform(F, bad, Lw, nb, A, ib)
    assert np.abs(MA - np.triu(F)).max() > 1e-3


def test_singular_column_reported():
    n = 40
    A = synth.general_matrix(n, seed=5).numpy()
    A[:, 17] = 0.0
    _, _, _, info = lu.lu_incpiv(A, nb=16, ib=8)
    assert info == 18


def test_lu_task_graph_by_hand_T2():
    tasks, preds, succs = dag.build(2, dag.program_lu(2))
    G, E, S, M = dag.GETRF, dag.GESSM, dag.TSTRF, dag.SSSSM
    assert tasks == [(G, 0, 0, 0), (E, 0, 1, 0), (S, 1, 0, 0), (M, 1, 1, 0), (G, 1, 1, 1)]
    assert preds[(E, 0, 1, 0)] == {(G, 0, 0, 0)}
    assert preds[(S, 1, 0, 0)] == {(G, 0, 0, 0)}  # GESSM reads the L part, TSTRF writes U
    assert preds[(M, 1, 1, 0)] == {(E, 0, 1, 0), (S, 1, 0, 0)}
    assert preds[(G, 1, 1, 1)] == {(M, 1, 1, 0)}


def test_lu_task_counts():
    # per step with m trailing tiles: 1 GETRF, m GESSM, m TSTRF, m^2 SSSSM
    for T in (1, 3, 6):
        tasks, preds, _ = dag.build(T, dag.program_lu(T))
        assert len(tasks) == sum(1 + 2 * m + m * m for m in range(T))
        for kind, i, j, k in tasks:
            # chains: TSTRF(i, k) after TSTRF(i-1, k); SSSSM(i, j, k) after SSSSM(i-1, j, k)
            if kind == dag.TSTRF and i > k + 1:
                assert (dag.TSTRF, i - 1, k, k) in preds[(kind, i, j, k)]
            if kind == dag.SSSSM and i > k + 1:
                assert (dag.SSSSM, i - 1, j, k) in preds[(kind, i, j, k)]
