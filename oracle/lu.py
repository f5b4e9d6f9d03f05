"""Tile LU factorization with incremental pivoting, and the solve that uses it.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's second workload is the PLASMA tile algorithm for DGETRF (Section 4.1,
"Benchmarks"), run in double precision with tiles of 512 and an inner block IB of 128
(Section 4.1, "Methodology"). The paper does not write the algorithm out; PLASMA's tile LU
factors with incremental pivoting, and this module restates it from its definition, one
kernel after the other in the order the sequential tile program calls them:

  for k in 0..T-1:
    GETRF(k)       P A_kk = L U, partial pivoting inside the diagonal tile
    GESSM(k, j)    the row interchanges and L^{-1} of GETRF(k) applied to A_kj, j > k
    for i in k+1..T-1:
      TSTRF(i, k)  LU with partial pivoting of the tall matrix [U_kk; A_ik]: U_kk is
                   updated, A_ik receives the multipliers
      SSSSM(i,j,k) the transformation of TSTRF(i, k) applied to [A_kj; A_ij], j > k

Every kernel works on inner blocks of IB columns. For one block the elimination is an LU
with partial pivoting of a panel of rows; the rows of the panel are numbered by
"positions" (0 .. w-1 are the w rows the block's pivots end up in, w .. are the rows below
them), the pivot of column j is the position swapped with position j, and the block's
transformation of any set of rows [X1; X2] laid out the same way is (apply_block):

  1. the interchanges j <-> piv[j], j = 0 .. w-1, in that order,
  2. X1 <- L11^{-1} X1 with L11 the unit lower triangle of the panel's first w rows,
  3. X2 <- X2 - L21 X1 with L21 the multipliers of the panel's remaining rows.

Multipliers of earlier blocks are not swapped by later blocks (the transformation of block
b is applied after those of blocks 0 .. b-1, to the rows in their order at that time).
In TSTRF the first w positions are rows of U_kk, whose strict lower triangle holds the
factor of GETRF(k); the unit lower L11 of the block therefore goes to a separate array Lw
(one ib x nk array per tile (i, k)), as in PLASMA.

Results (all in place, float64):
  F            the factored matrix: np.triu(F) is U; the strict lower triangle of a diagonal
               tile holds the multipliers of GETRF; tile (i, k), i > k, the multipliers of
               TSTRF(i, k)
  piv[(k, k)]  GETRF(k) pivot positions, per column of tile k, relative to the block start
  piv[(i, k)]  TSTRF(i, k) pivot positions (0 .. w-1: a row of U_kk; w + r: row r of A_ik)
  Lw[(i, k)]   ib x nk, block b's L11 (strict lower part) in columns b*ib ...
  info         0, or the 1-based global column of the first zero pivot (the factor is then
               singular; the elimination goes on without scaling that column, as LAPACK)

The arithmetic is plain: a division per multiplier, an outer-product update per column,
and numpy products for the block applications; nothing is fused or reordered beyond the
kernels' own definitions.
"""
import math

import numpy as np

IB = 32


def tiles(n, nb):
    return max(1, math.ceil(n / nb)) if n > 0 else 0


def _rows(n, nb, t):
    return slice(t * nb, min(n, (t + 1) * nb))


def panel_lu(P):
    """Unblocked LU with partial pivoting of the m x w panel P in place (LAPACK's unblocked
    getrf: the first largest magnitude wins). Returns (piv, info) with info the 1-based
    column of the first zero pivot or 0."""
    m, w = P.shape
    piv = np.zeros(w, dtype=np.int64)
    info = 0
    for j in range(min(m, w)):
        p = j + int(np.argmax(np.abs(P[j:, j])))
        piv[j] = p
        if p != j:
            P[[j, p], :] = P[[p, j], :]
        d = P[j, j]
        if d != 0.0:
            P[j + 1:, j] = P[j + 1:, j] / d
        elif info == 0:
            info = j + 1
        P[j + 1:, j + 1:] -= np.outer(P[j + 1:, j], P[j, j + 1:])
    return piv, info


def unit_lower(B):
    """The unit lower triangle of the square block B (its strict lower part plus I)."""
    return np.tril(B, -1) + np.eye(B.shape[0])


def apply_block(X1, X2, piv, L11, L21):
    """One inner block's transformation applied in place to the rows [X1; X2] (see the
    module docstring): interchanges, X1 <- L11^{-1} X1, X2 <- X2 - L21 X1."""
    w = X1.shape[0]
    for j in range(w):
        q = int(piv[j])
        if q == j:
            continue
        if q < w:
            X1[[j, q], :] = X1[[q, j], :]
        else:
            t = X1[j, :].copy()
            X1[j, :] = X2[q - w, :]
            X2[q - w, :] = t
    for r in range(1, w):
        X1[r, :] -= L11[r, :r] @ X1[:r, :]
    if X2.shape[0] and w:
        X2 -= L21 @ X1


def _blocks(nk, ib):
    for c0 in range(0, nk, ib):
        yield c0, min(nk, c0 + ib)


def getrf_tile(Akk, ib=IB):
    """GETRF on the diagonal tile in place. Returns (piv, info)."""
    nk = Akk.shape[0]
    piv = np.zeros(nk, dtype=np.int64)
    info = 0
    for c0, c1 in _blocks(nk, ib):
        pb, inf = panel_lu(Akk[c0:, c0:c1])
        if inf and not info:
            info = c0 + inf
        piv[c0:c1] = pb
        apply_block(Akk[c0:c1, c1:], Akk[c1:, c1:], pb, unit_lower(Akk[c0:c1, c0:c1]), Akk[c1:, c0:c1])
    return piv, info


def gessm_tile(Akj, Akk, piv, ib=IB):
    """GESSM: GETRF(k)'s transformation applied to A_kj in place."""
    nk = Akk.shape[0]
    for c0, c1 in _blocks(nk, ib):
        apply_block(Akj[c0:c1, :], Akj[c1:, :], piv[c0:c1], unit_lower(Akk[c0:c1, c0:c1]), Akk[c1:, c0:c1])


def tstrf_tile(Ukk, Aik, ib=IB):
    """TSTRF: LU with partial pivoting of [U_kk; A_ik] in place (U_kk's strict lower triangle
    is left alone). Returns (piv, Lw, info)."""
    nk = Ukk.shape[0]
    mi = Aik.shape[0]
    piv = np.zeros(nk, dtype=np.int64)
    Lw = np.zeros((ib, nk))
    info = 0
    for c0, c1 in _blocks(nk, ib):
        w = c1 - c0
        P = np.vstack([np.triu(Ukk[c0:c1, c0:c1]), Aik[:, c0:c1]])
        pb, inf = panel_lu(P)
        if inf and not info:
            info = c0 + inf
        piv[c0:c1] = pb
        Ukk[c0:c1, c0:c1] = np.tril(Ukk[c0:c1, c0:c1], -1) + np.triu(P[:w])
        Lw[:w, c0:c1] = np.tril(P[:w], -1)
        Aik[:, c0:c1] = P[w:]
        apply_block(Ukk[c0:c1, c1:], Aik[:, c1:], pb, unit_lower(P[:w]), Aik[:, c0:c1])
    del mi
    return piv, Lw, info


def ssssm_tile(Akj, Aij, Aik, piv, Lw, ib=IB):
    """SSSSM: TSTRF(i, k)'s transformation applied to [A_kj; A_ij] in place."""
    nk = Aik.shape[1]
    for c0, c1 in _blocks(nk, ib):
        w = c1 - c0
        apply_block(Akj[c0:c1, :], Aij, piv[c0:c1], unit_lower(Lw[:w, c0:c1]), Aik[:, c0:c1])


def lu_incpiv(A, nb, ib=IB):
    """Tile LU with incremental pivoting of the n x n matrix A. Returns (F, piv, Lw, info)."""
    F = np.array(A, dtype=np.float64, copy=True)
    n = F.shape[0]
    T = tiles(n, nb)
    piv, Lw = {}, {}
    info = 0
    R = lambda t: _rows(n, nb, t)  # noqa: E731
    for k in range(T):
        Akk = F[R(k), R(k)]
        piv[(k, k)], inf = getrf_tile(Akk, ib)
        if inf and not info:
            info = k * nb + inf
        for j in range(k + 1, T):
            gessm_tile(F[R(k), R(j)], Akk, piv[(k, k)], ib)
        for i in range(k + 1, T):
            piv[(i, k)], Lw[(i, k)], inf = tstrf_tile(Akk, F[R(i), R(k)], ib)
            if inf and not info:
                info = k * nb + inf
            for j in range(k + 1, T):
                ssssm_tile(F[R(k), R(j)], F[R(i), R(j)], F[R(i), R(k)], piv[(i, k)], Lw[(i, k)], ib)
    return F, piv, Lw, info


def forward_transform(F, piv, Lw, nb, B, ib=IB):
    """Apply the factorization's transformations to B (n x nrhs) in the order the factor
    recorded them: GETRF(k) to block row k, then TSTRF(i, k) to block rows (k, i), i > k.
    Applied to A itself the result is U = np.triu(F)."""
    n = F.shape[0]
    Y = np.array(B, dtype=np.float64, copy=True).reshape(n, -1)
    T = tiles(n, nb)
    R = lambda t: _rows(n, nb, t)  # noqa: E731
    for k in range(T):
        Akk = F[R(k), R(k)]
        Yk = Y[R(k)]
        gessm_tile(Yk, Akk, piv[(k, k)], ib)
        for i in range(k + 1, T):
            ssssm_tile(Yk, Y[R(i)], F[R(i), R(k)], piv[(i, k)], Lw[(i, k)], ib)
    return Y


def back_substitute(U, Y):
    """Solve U X = Y for upper triangular U by back substitution (one division per row)."""
    X = np.array(Y, dtype=np.float64, copy=True)
    n = U.shape[0]
    for r in range(n - 1, -1, -1):
        if r + 1 < n:
            X[r] -= U[r, r + 1:] @ X[r + 1:]
        X[r] = X[r] / U[r, r]
    return X


def lu_solve(F, piv, Lw, nb, B, ib=IB):
    """x = A^{-1} b from the tile LU factors."""
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    X = back_substitute(np.triu(F), forward_transform(F, piv, Lw, nb, B, ib))
    return X.reshape(-1) if vec else X
