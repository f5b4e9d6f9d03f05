"""Pins of the oracle against facts fixed by the mathematics, not by the oracle itself.

The oracle writes out the definition of the Cholesky factor (the unique lower-triangular L
with positive diagonal and A = L L^T); the tile algorithm of the paper (PLASMA DPOTRF,
Section 4.1) reaches that factor under every schedule. Each test below would fail for a
plausible slip in the oracle: a dropped term, a wrong sign or index, a transposed operand.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n", [1, 2, 3, 5, 12, 20])
def test_pascal_closed_form_bitwise(n):
    # Symmetric Pascal matrix P_ij = C(i+j, i) has the lower Pascal matrix L_ij = C(i, j) as
    # its Cholesky factor (Vandermonde's identity); every intermediate is an integer < 2^53.
    F, info = oracle.cholesky(synth.pascal(n))
    assert info == 0
    np.testing.assert_array_equal(np.tril(F), synth.pascal_lower(n))


@pytest.mark.parametrize("n,seed", [(1, 0), (7, 1), (64, 2), (257, 3)])
def test_integer_factor_recovered_bitwise(n, seed):
    L, A = synth.integer_factor(n, seed)
    F, info = oracle.cholesky(A)
    assert info == 0
    np.testing.assert_array_equal(np.tril(F), L)


@pytest.mark.parametrize("n,nrhs", [(5, 1), (64, 3), (200, 2)])
def test_integer_solves_exact(n, nrhs):
    # L y = b and L^T x = y with integer data: every quotient is an exact integer.
    L, A = synth.integer_factor(n, 11)
    X = synth.integer_vector(n, nrhs, 3)
    Y = L.T @ X           # exact integers
    B = L @ Y             # exact integers, B = A X
    np.testing.assert_array_equal(oracle.forward_solve(L, B), Y)
    np.testing.assert_array_equal(oracle.backward_solve(L, Y), X)
    np.testing.assert_array_equal(oracle.solve(L, B), X)


def test_forward_and_backward_are_not_interchangeable():
    # A solve with the wrong triangle (L^T instead of L) must not pass the pins above.
    L, _ = synth.integer_factor(6, 5)
    b = L @ np.arange(1.0, 7.0)
    y = oracle.forward_solve(L, b)
    np.testing.assert_array_equal(y, np.arange(1.0, 7.0))
    assert not np.array_equal(oracle.backward_solve(L, b), np.arange(1.0, 7.0))


@pytest.mark.parametrize("n", [2, 3, 4, 10, 100])
def test_matches_lapack(n):
    A = synth.gram_spd(n, seed=n).numpy()
    F, info = oracle.cholesky(A)
    assert info == 0
    ref = np.linalg.cholesky(A)
    assert oracle.rel_frobenius(np.tril(F), ref) <= 1e-14


@pytest.mark.parametrize("n", [2, 3, 4])
def test_brute_force_small_against_lapack_and_reconstruction(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(50):
        M = rng.standard_normal((n, n))
        A = M @ M.T + n * np.eye(n)
        F, info = oracle.cholesky(A)
        L = np.tril(F)
        assert info == 0
        assert np.all(np.diag(L) > 0)
        np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(L @ L.T, A, rtol=1e-14, atol=1e-13)


def test_uniqueness_of_factor():
    # A = M M^T with M lower and positive diagonal has M as its unique Cholesky factor.
    rng = np.random.default_rng(7)
    n = 120
    M = np.tril(0.1 * rng.standard_normal((n, n)), -1) + np.diag(rng.uniform(1.0, 2.0, n))
    A = M @ M.T
    L = oracle.factor(A)
    assert oracle.rel_frobenius(L, M) <= 1e-13


def test_invariants_and_upper_untouched():
    n = 256
    A = synth.gram_spd(n, seed=5).numpy().copy(order="F")
    marker = np.triu(np.full((n, n), 12345.0), 1)
    Ain = np.tril(A) + marker        # upper triangle holds a marker the factor must keep
    F, info = oracle.cholesky(Ain)
    assert info == 0
    np.testing.assert_array_equal(np.triu(F, 1), marker)
    L = np.tril(F)
    assert np.all(np.diag(L) > 0)
    assert oracle.factor_residual(A, L) <= 1e-14


@pytest.mark.parametrize("diag,expect", [((1.0, 2.0, -1.0, 4.0), 3), ((-1.0, 1.0), 1),
                                         ((1.0, 1.0, 1.0, 0.0), 4)])
def test_not_positive_definite_info(diag, expect):
    F, info = oracle.cholesky(np.diag(diag))
    assert info == expect


def test_singular_leading_minor():
    A = np.array([[1.0, 1.0, 0.0], [1.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    _, info = oracle.cholesky(A)
    assert info == 2
    A[0, 0] = np.nan
    _, info = oracle.cholesky(A)
    assert info == 1


def test_solve_backward_error_and_lapack():
    n, nrhs = 300, 4
    A = synth.gram_spd(n, seed=9).numpy()
    B = synth.rhs(n, nrhs, seed=10).numpy()
    L = oracle.factor(A)
    X = oracle.solve(L, B)
    assert oracle.backward_error(A, X, B) <= 1e-15 * 10
    np.testing.assert_allclose(X, np.linalg.solve(A, B), rtol=1e-12, atol=1e-12)


def test_empty():
    F, info = oracle.cholesky(np.zeros((0, 0)))
    assert info == 0 and F.shape == (0, 0)
