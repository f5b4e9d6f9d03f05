"""Reference gradients for the Cholesky factor and the solve: TEST INFRASTRUCTURE ONLY.

Not in the paper (the differentiable form of its factorization). Conventions:
  * A is symmetric; a gradient with respect to A is returned symmetric, so that a finite
    difference that moves a_ij and a_ji together (i != j) sees 2 * Abar_ij, and one that
    moves a_ii sees Abar_ii.
  * L is lower triangular; its gradient Lbar is lower triangular.

cholesky_backward(L, Lbar): the gradient of <Lbar, chol(A)> with respect to A, written out
as S = L^-T Phi(L^T Lbar) L^-1, Abar = (S + S^T) / 2, Phi = lower triangle with the diagonal
halved (the reverse-mode rule for the Cholesky factor; I. Murray, "Differentiation of the
Cholesky decomposition", 2016). Pinned by central finite differences in the tests.

solve_backward(L, X, Xbar): for X = A^-1 B with A = L L^T, Bbar = A^-1 Xbar and
Lbar = -tril((Bbar X^T + X Bbar^T) L) (from dX = -A^-1 dA X and dA = dL L^T + L dL^T).

solve_grad_A(A, B, W): the closed form of d(sum W*X)/dA for X = A^-1 B: -sym(Bbar X^T)
with Bbar = A^-1 W, the plain definition the composed adjoint must reach.
"""
import numpy as np
import scipy.linalg as sla


def _phi(P):
    Q = np.tril(P).copy()
    Q[np.diag_indices_from(Q)] *= 0.5
    return Q


def cholesky_backward(L, Lbar):
    L = np.tril(np.asarray(L, dtype=np.float64))
    Lbar = np.tril(np.asarray(Lbar, dtype=np.float64))
    P = _phi(L.T @ Lbar)
    # S = L^-T P L^-1: solve L^T S = P L^-1, with P L^-1 = (L^-T P^T)^T
    M = sla.solve_triangular(L, P.T, lower=True, trans="T").T
    S = sla.solve_triangular(L, M, lower=True, trans="T")
    return 0.5 * (S + S.T)


def solve_backward(L, X, Xbar):
    L = np.tril(np.asarray(L, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64).reshape(L.shape[0], -1)
    Xbar = np.asarray(Xbar, dtype=np.float64).reshape(L.shape[0], -1)
    Y = sla.solve_triangular(L, Xbar, lower=True)
    Bbar = sla.solve_triangular(L, Y, lower=True, trans="T")
    Lbar = -np.tril((Bbar @ X.T + X @ Bbar.T) @ L)
    return Bbar, Lbar


def solve_grad_A(A, B, W):
    A = np.asarray(A, dtype=np.float64)
    X = np.linalg.solve(A, B)
    Bbar = np.linalg.solve(A, W)
    G = Bbar @ np.asarray(X).reshape(A.shape[0], -1).T if X.ndim == 2 else np.outer(Bbar, X)
    return -0.5 * (G + G.T)
