"""Pins of the reference gradients by central finite differences (CPU only)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint
import synth


def _sym_fd(f, A, h, idx):
    out = []
    for (i, j) in idx:
        E = np.zeros_like(A)
        E[i, j] = 1.0
        E[j, i] = 1.0
        g = (f(A + h * E) - f(A - h * E)) / (2 * h)
        out.append(g if i == j else 0.5 * g)
    return np.array(out)


@pytest.mark.parametrize("n", [5, 24])
def test_cholesky_backward_matches_finite_differences(n):
    rng = np.random.default_rng(n)
    A = synth.gram_spd(n, seed=n).numpy()
    Lbar = np.tril(rng.standard_normal((n, n)))
    f = lambda M: float(np.sum(Lbar * oracle.factor(M)))
    G = adjoint.cholesky_backward(oracle.factor(A), Lbar)
    idx = [(i, j) for i in range(n) for j in range(i + 1)][:: max(1, n // 4)]
    fd = _sym_fd(f, A, 1e-6, idx)
    got = np.array([G[i, j] for (i, j) in idx])
    np.testing.assert_allclose(got, fd, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(G, G.T)


@pytest.mark.parametrize("n,nrhs", [(6, 1), (20, 3)])
def test_solve_backward_matches_finite_differences(n, nrhs):
    rng = np.random.default_rng(3 * n)
    A = synth.gram_spd(n, seed=n + 1).numpy()
    B = rng.standard_normal((n, nrhs))
    W = rng.standard_normal((n, nrhs))
    L = oracle.factor(A)
    X = oracle.solve(L, B)
    Bbar, Lbar = adjoint.solve_backward(L, X, W)
    # d/dB of sum(W * solve(L, B))
    h = 1e-6
    for (i, c) in [(0, 0), (n - 1, nrhs - 1), (n // 2, 0)]:
        E = np.zeros_like(B)
        E[i, c] = 1.0
        fd = (np.sum(W * oracle.solve(L, B + h * E)) - np.sum(W * oracle.solve(L, B - h * E))) / (2 * h)
        assert abs(Bbar[i, c] - fd) <= 1e-7 * max(1.0, abs(fd))
    # d/dL (lower entries) of sum(W * solve(L, B))
    for (i, j) in [(0, 0), (n - 1, 0), (n - 1, n - 1), (n // 2, n // 3)]:
        E = np.zeros_like(L)
        E[i, j] = 1.0
        fd = (np.sum(W * oracle.solve(L + h * E, B)) - np.sum(W * oracle.solve(L - h * E, B))) / (2 * h)
        assert abs(Lbar[i, j] - fd) <= 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("n", [4, 16])
def test_composition_equals_closed_form(n):
    rng = np.random.default_rng(11 * n)
    A = synth.gram_spd(n, seed=2 * n).numpy()
    b = rng.standard_normal((n, 2))
    w = rng.standard_normal((n, 2))
    L = oracle.factor(A)
    X = oracle.solve(L, b)
    _, Lbar = adjoint.solve_backward(L, X, w)
    G = adjoint.cholesky_backward(L, Lbar)
    np.testing.assert_allclose(G, adjoint.solve_grad_A(A, b, w), rtol=1e-10, atol=1e-12)
    # and the closed form against finite differences of the loss itself
    f = lambda M: float(np.sum(w * np.linalg.solve(M, b)))
    idx = [(0, 0), (n - 1, 0), (n // 2, n // 2 - 1)]
    fd = _sym_fd(f, A, 1e-6, idx)
    np.testing.assert_allclose([G[i, j] for (i, j) in idx], fd, rtol=1e-6, atol=1e-8)
