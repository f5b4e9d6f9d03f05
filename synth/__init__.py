"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the method's arithmetic: it only draws matrices and right-hand
sides with the shapes and value distributions of the workloads (the paper factors dense
double-precision SPD matrices of order 8192 and 16384 with 512 x 512 tiles, Section 4.1
"Methodology" and Section 4.2; it does not say how the matrices are drawn, so the recipes
below stand in for them).

Random numbers come from torch's seeded generators on the device the data is made on; a
test that feeds the same input to the oracle and to the CUDA library makes it once and
copies the bytes, so both sides always see identical values.

Recipes
  gram_spd(n)         A = sym(G G^T)/n + I, G n x n i.i.d. N(0,1) drawn in FP32, product in
                      FP32 (TF32 off), symmetrised and promoted to FP64; kappa(A) <~ 5.
  householder_spd(n)  A = Q diag(lambda) Q^T, lambda_i = 10^(6 i/(n-1)), Q = H_1 ... H_32,
                      H = I - 2 v v^T / v^T v with v ~ N(0,1); kappa(A) = 1e6 (and, with
                      inverse=True, Q diag(1/lambda) Q^T from the same reflectors).
  integer_factor(n)   integer lower L, diag in [1, 8], off-diagonal in [-8, 8]; A = L L^T is
                      then exact in FP64 (|a_ij| <= 64 n < 2^53).
  pascal(n)           P_ij = C(i + j, i) (0-based).
  general_matrix(n)   A with i.i.d. N(0,1) entries in float64 (the LU workload: a dense
                      general matrix; kappa grows like n).
  dyadic_lu(n)        unit lower L with off-diagonal entries in {0, +-1/4, +-1/2}, upper U
                      with integer entries (|u_jj| in [16, 32], off-diagonal in [-8, 8]);
                      A = L U is exact in FP64, and since every multiplier is below 1 in
                      magnitude, partial pivoting never interchanges rows.
"""
import math

import numpy as np
import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def gram_spd(n, seed=0, device="cpu"):
    """A = sym(G G^T)/n + I in float64 (column-major friendly: A is symmetric)."""
    device = torch.device(device)
    g = _gen(seed, device)
    G = torch.randn(n, n, generator=g, device=device, dtype=torch.float32)
    prev = None
    if device.type == "cuda":
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
    try:
        S = G @ G.T
    finally:
        if prev is not None:
            torch.backends.cuda.matmul.allow_tf32 = prev
    del G
    A = S.to(torch.float64)
    del S
    A = (A + A.T) * (0.5 / n)
    A.diagonal().add_(1.0)
    return A


def rhs(n, nrhs, seed=1, device="cpu"):
    """B n x nrhs i.i.d. N(0,1) in float64, column-major (Fortran) layout."""
    device = torch.device(device)
    g = _gen(seed, device)
    B = torch.randn(nrhs, n, generator=g, device=device, dtype=torch.float64)
    return B.T  # n x nrhs view whose columns are contiguous


def householder_spd(n, seed=0, device="cpu", n_reflectors=32, cond=1e6, inverse=False):
    """A = Q diag(lambda) Q^T with geometrically spaced lambda in [1, cond]. With inverse=True
    the same reflectors (same seed) are applied to diag(1/lambda): the inverse of that A up to
    rounding, for condition numbers in norms other than the 2-norm."""
    device = torch.device(device)
    g = _gen(seed, device)
    lam = torch.pow(torch.tensor(10.0, dtype=torch.float64, device=device),
                    torch.arange(n, dtype=torch.float64, device=device) * (math.log10(cond) / max(n - 1, 1)))
    if inverse:
        lam = 1.0 / lam
    A = torch.diag(lam)
    for _ in range(n_reflectors):
        v = torch.randn(n, generator=g, device=device, dtype=torch.float64)
        beta = 2.0 / torch.dot(v, v)
        # H A H with H = I - beta v v^T, applied as two rank-one updates
        w = A @ v
        A -= beta * torch.outer(v, w)
        w = A @ v
        A -= beta * torch.outer(w, v)
    A = 0.5 * (A + A.T)
    return A


def integer_factor(n, seed=0):
    """(L, A) with L integer lower triangular and A = L L^T exact, both float64 numpy."""
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-8, 9, size=(n, n)), -1).astype(np.float64)
    L[np.arange(n), np.arange(n)] = rng.integers(1, 9, size=n)
    A = L @ L.T  # every partial sum is an integer below 2^53: exact in any order
    return L, A


def integer_vector(n, nrhs, seed=0):
    rng = np.random.default_rng(seed + 7919)
    return rng.integers(-4, 5, size=(n, nrhs)).astype(np.float64)


def general_matrix(n, seed=0, device="cpu"):
    """A with i.i.d. N(0,1) entries, float64, column-major (Fortran) layout."""
    device = torch.device(device)
    g = _gen(seed, device)
    return torch.randn(n, n, generator=g, device=device, dtype=torch.float64).T


def dyadic_lu(n, seed=0):
    """(L, U, A) float64 numpy with A = L U exact (see the module docstring)."""
    rng = np.random.default_rng(seed + 104729)
    L = np.tril(rng.integers(-2, 3, size=(n, n)) * 0.25, -1)
    L[np.arange(n), np.arange(n)] = 1.0
    U = np.triu(rng.integers(-8, 9, size=(n, n)).astype(np.float64), 1)
    U[np.arange(n), np.arange(n)] = rng.integers(16, 33, size=n) * rng.choice([-1.0, 1.0], size=n)
    A = L @ U  # two fractional bits, magnitudes far below 2^53: exact in any order
    return L, U, A


def pascal(n):
    P = np.empty((n, n), dtype=np.float64)
    for i in range(n):
        for j in range(n):
            P[i, j] = math.comb(i + j, i)
    return P


def pascal_lower(n):
    Lp = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for j in range(i + 1):
            Lp[i, j] = math.comb(i, j)
    return Lp


def batch_orders(count, lo=16, hi=512, seed=0):
    """Orders of a batch of matrices, uniform on [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count).astype(np.int32)


def gram_spd_batch(orders, seed=0, device="cpu", dtype=torch.float64):
    """A batch of Gram matrices A_m = sym(G G^T)/n_m + I (recipe of gram_spd) packed
    column-major one after the other in one flat tensor. Matrices of equal order are drawn
    and multiplied together. Returns (flat, offsets) with offsets[m] the element offset of
    matrix m."""
    device = torch.device(device)
    orders = [int(n) for n in orders]
    offsets, off = [], 0
    for n in orders:
        offsets.append(off)
        off += n * n
    flat = torch.empty(max(off, 1), dtype=dtype, device=device)
    g = _gen(seed, device)
    by_n = {}
    for m, n in enumerate(orders):
        by_n.setdefault(n, []).append(m)
    for n in sorted(by_n):
        idx = by_n[n]
        if n == 0:
            continue
        G = torch.randn(len(idx), n, n, generator=g, device=device, dtype=torch.float32)
        S = torch.bmm(G, G.transpose(1, 2)).to(torch.float64)
        A = (S + S.transpose(1, 2)) * (0.5 / n)
        A.diagonal(dim1=1, dim2=2).add_(1.0)
        A = A.to(dtype)
        for q, m in enumerate(idx):
            # symmetric, so the row-major copy of A is also its column-major storage
            flat[offsets[m]:offsets[m] + n * n].copy_(A[q].reshape(-1))
    return flat, offsets
