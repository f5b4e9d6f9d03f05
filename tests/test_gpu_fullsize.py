"""Parity at the benchmark's full sizes, with the inputs and launch configurations bench.py
times, on outputs the oracle can compute piece by piece and on properties that hold at any
size.

FP64 factor + solve, n = 32768, 64 right-hand sides, tile 256 (HEFT) and 512 (DADA):
  - the leading k x k block of L is the Cholesky factor of the leading k x k block of A, so
    the oracle factors A[:k, :k] (k = 1024) and the GPU's block must agree within relative
    Frobenius 1e-12;
  - any row i of L restricted to those columns solves L[:k, :k] y = A[i, :k]^T, so sampled
    rows come from the oracle's forward substitution against its own leading factor
    (relative 1e-12);
  - info = 0 and a positive diagonal over the whole factor;
  - the normwise (Rigal-Gaches, infinity norm) backward error of sampled right-hand sides,
    computed on the host in FP64 from A, x and b, is <= 1e-14;
  - the factor residual in four seeded random directions v, ||(A - L L^T) v||_inf /
    (||A||_inf ||v||_inf), computed on the host in FP64 by row blocks, is <= n u (the bound
    of a backward-stable Cholesky; an O(n^2) check of the whole factor).
FP64 factor, n = 8192 (bench.py's policy-comparison size), tiles 256 and 128 under HEFT,
DADA(0.5)+CP and work stealing: the whole L against the oracle's factor of the same A,
relative Frobenius 1e-12 (kappa(A) <= 5).
Mixed precision, n = 16384, kappa = 1e6, 16 right-hand sides: each form that reaches the
target (FP32, three-term BF16) must report and have backward error <= 1e-14, and its X must
agree with the oracle's FP64 solution of the same A and B within the forward-error bound
that both backward errors imply, sum of 2 kappa_inf eta / (1 - kappa_inf eta) (Higham,
Accuracy and Stability, Thm 7.2), with kappa_inf = ||A||_inf ||A^-1||_inf computed from
A^-1 = Q diag(1/lambda) Q^T built from the same reflectors.
Batched, 10,000 matrices of orders uniform in [16, 512] (FP64 and FP32): sampled members
against the oracle's factor and their backward errors.
Adjoint, 64 matrices of order 1024: sampled gradients against the oracle's gradient.
LU with incremental pivoting, n = 8192, automatic tile (128), HEFT (the LU leg of bench.py):
  - the multipliers, pivots and L11 blocks of every task in the leading T' x T' tiles
    (T' = 8) depend only on A's leading T' x T' tiles, so they must agree with the oracle's
    factorization of A[:1024, :1024] (pivots identical, values within relative Frobenius
    max(1e-12, kappa_2(A[:1024, :1024]) k u), k = 1024, u = 2^-53: rounding differences
    amplified by the conditioning, the bound of test_gpu_lu.py);
  - every multiplier is at most 1 in magnitude (partial pivoting inside each panel);
  - the backward error of the solve is at most n u rho with rho = max|U| / max|A| the growth
    factor of the computed U (the classical bound of Gaussian elimination; incremental
    pivoting lets rho rise with n).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import adjoint as oadj
from oracle import lu as olu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chol():
    import paper_1402_6601_gb300 as c
    return c


def _berr_cols(A_dev, X, B, cols, chunk=2048):
    """Rigal-Gaches backward error of the columns `cols`, on the host in FP64, reading A from
    the device in row blocks (no full-size temporaries)."""
    n = A_dev.shape[0]
    Xc = X[:, cols].cpu().numpy().astype(np.float64)
    Bc = B[:, cols].cpu().numpy().astype(np.float64)
    R = Bc.copy()
    normA = 0.0
    for r0 in range(0, n, chunk):
        blk = A_dev[r0:r0 + chunk, :].cpu().numpy()  # rows r0.. of the symmetric A
        R[r0:r0 + chunk] -= blk @ Xc
        normA = max(normA, float(np.abs(blk).sum(axis=1).max()))
    num = np.abs(R).max(axis=0)
    den = normA * np.abs(Xc).max(axis=0) + np.abs(Bc).max(axis=0)
    return float((num / den).max())


@pytest.mark.parametrize("nb,policy,alpha", [(256, "heft", 0.5), (512, "dada", 0.5)])
def test_factor_solve_n32768(chol, nb, policy, alpha):
    n, nrhs, k, seed = 32768, 64, 1024, 1  # bench.py's main leg: A seed 1, B seed 1001
    A = chol.colmajor(synth.gram_spd(n, seed=seed, device="cuda"))
    B = chol.colmajor(synth.rhs(n, nrhs, seed=seed + 1000, device="cuda"))
    F = A.clone()
    info, _ = chol.factor(F, chol.opts(nb=nb, policy=policy, alpha=alpha))
    X = B.clone()
    chol.solve(F, X)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert bool((torch.diagonal(F) > 0).all().item())
    # leading block
    L_lead = oracle.factor(A[:k, :k].cpu().numpy())
    assert oracle.rel_frobenius(np.tril(F[:k, :k].cpu().numpy()), L_lead) <= 1e-12
    # sampled rows below it
    rows = np.sort(np.random.default_rng(7).choice(np.arange(k, n), size=16, replace=False))
    idx = torch.as_tensor(rows, device="cuda")
    a_rows = A[idx, :k].cpu().numpy()                        # 16 x k
    ref = oracle.forward_solve(L_lead, np.asfortranarray(a_rows.T)).T   # L_lead y = a^T
    got = F[idx, :k].cpu().numpy()
    assert oracle.rel_frobenius(got, ref) <= 1e-12
    # backward error of sampled right-hand sides
    assert _berr_cols(A, X, B, [0, 17, 40, 63]) <= 1e-14
    # factor residual in random directions
    assert _factor_residual_dirs(A, F, nv=4, seed=11) <= n * 2.0 ** -53


def _factor_residual_dirs(A_dev, F_dev, nv, seed, chunk=2048):
    """max over nv random directions v of ||(A - L L^T) v||_inf / (||A||_inf ||v||_inf), on
    the host in FP64: w = L^T v by column blocks of L, then A v - L w by row blocks."""
    n = A_dev.shape[0]
    V = np.random.default_rng(seed).standard_normal((n, nv))
    W = np.zeros((n, nv))
    for c0 in range(0, n, chunk):           # W[c0:c1] = L[:, c0:c1]^T V
        c1 = min(n, c0 + chunk)
        Lc = np.tril(F_dev[c0:, c0:c1].cpu().numpy())   # rows c0.. of columns c0..c1-1
        W[c0:c1] = Lc.T @ V[c0:]
    R = np.zeros((n, nv))
    normA = 0.0
    for r0 in range(0, n, chunk):           # R[r0:r1] = A[r0:r1] V - L[r0:r1, :r1] W[:r1]
        r1 = min(n, r0 + chunk)
        Ab = A_dev[r0:r1, :].cpu().numpy()
        normA = max(normA, float(np.abs(Ab).sum(axis=1).max()))
        Lb = F_dev[r0:r1, :r1].cpu().numpy()
        Lb[:, r0:r1] = np.tril(Lb[:, r0:r1])
        R[r0:r1] = Ab @ V - Lb @ W[:r1]
    return float((np.abs(R).max(axis=0) / (normA * np.abs(V).max(axis=0))).max())


@pytest.fixture(scope="module")
def factor8192():
    n, seed = 8192, 1
    A = synth.gram_spd(n, seed=seed, device="cuda")
    return A, oracle.factor(A.cpu().numpy())


@pytest.mark.parametrize("nb", [256, 128, 512])
@pytest.mark.parametrize("policy,alpha,cp", [("heft", 0.5, False), ("dada", 0.5, True), ("steal", 0.5, False)])
def test_factor_n8192_whole_L(chol, factor8192, nb, policy, alpha, cp):
    A, Lo = factor8192
    F = chol.colmajor(A)
    info, _ = chol.factor(F, chol.opts(nb=nb, policy=policy, alpha=alpha, use_cp=cp))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert oracle.rel_frobenius(np.tril(F.cpu().numpy()), Lo) <= 1e-12


@pytest.fixture(scope="module")
def mixed16384():
    """bench.py's mixed-precision input, the oracle's FP64 solution and kappa_inf(A)."""
    n, nrhs, seed = 16384, 16, 1
    A = synth.householder_spd(n, seed=seed, cond=1e6, device="cuda")
    B = synth.rhs(n, nrhs, seed=seed + 7, device="cuda")
    Ai = synth.householder_spd(n, seed=seed, cond=1e6, device="cuda", inverse=True)
    kinf = float(A.abs().sum(1).max() * Ai.abs().sum(1).max())
    del Ai
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    Xo = oracle.solve(oracle.factor(Ah), Bh)
    eta_o = [oracle.backward_error(Ah, Xo[:, c], Bh[:, c]) for c in range(nrhs)]
    return A, B, Xo, eta_o, kinf


@pytest.mark.parametrize("precision", ["f32", "bf16x3"])
def test_mixed_precision_n16384(chol, mixed16384, precision):
    n, nrhs = 16384, 16  # bench.py's mixed leg
    A0, B0, Xo, eta_o, kinf = mixed16384
    A = chol.colmajor(A0)
    B = chol.colmajor(B0)
    X, info, iters, berr = chol.solve_refine(A, B, tol=1e-14, max_iter=30, o=chol.opts(nb=256),
                                             precision=precision)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert float(berr.item()) <= 1e-14
    # four refinement steps for both forms (the three-term form runs its SYRK updates in
    # FFMA; with them on the tensor cores it needed five)
    assert 2 <= int(iters.item()) <= 4
    assert _berr_cols(A, X, B, list(range(nrhs))) <= 1e-14
    # X against the oracle's FP64 solution, column by column, within the forward-error bound
    # that the two backward errors imply
    Xh, Ah, Bh = X.cpu().numpy(), A.cpu().numpy(), B.cpu().numpy()
    for c in range(nrhs):
        eta_g = oracle.backward_error(Ah, Xh[:, c], Bh[:, c])
        bound = sum(2 * kinf * e / (1 - kinf * e) for e in (eta_g, eta_o[c]))
        err = np.abs(Xh[:, c] - Xo[:, c]).max() / np.abs(Xo[:, c]).max()
        assert err <= bound, (c, err, bound, kinf)


@pytest.mark.parametrize("dtype,tol_l,tol_b", [(torch.float64, 1e-12, 1e-14), (torch.float32, 2e-5, 1e-6)])
def test_batched_10000(chol, dtype, tol_l, tol_b):
    seed = 1  # bench.py's batched leg
    orders = [int(n) for n in synth.batch_orders(10000, 16, 512, seed=seed)]
    roffs, off = [], 0
    for n in orders:
        roffs.append(off)
        off += n
    flat, offs = synth.gram_spd_batch(orders, seed=seed + 3, device="cuda", dtype=dtype)
    g = torch.Generator(device="cuda").manual_seed(seed + 4)
    rhs = torch.randn(off, generator=g, device="cuda", dtype=torch.float64).to(dtype)
    bt = chol.Batch(flat.clone(), offs, orders, rhs.clone(), roffs)
    src = chol.Batch(flat, offs, orders, rhs, roffs)
    chol.posv_batched(bt)
    torch.cuda.synchronize()
    assert int(bt.info.abs().max().item()) == 0
    rng = np.random.default_rng(3)
    sample = list(rng.choice(len(orders), size=24, replace=False)) + [int(np.argmax(orders))]
    for m in sample:
        A0 = src.matrix(m).cpu().numpy().astype(np.float64)
        L = np.tril(bt.matrix(m).cpu().numpy().astype(np.float64))
        assert oracle.rel_frobenius(L, oracle.factor(A0)) <= tol_l, m
        x = bt.rhs(m).cpu().numpy().astype(np.float64)
        b = src.rhs(m).cpu().numpy().astype(np.float64)
        assert oracle.backward_error(A0, x, b) <= tol_b, m


def test_adjoint_64_matrices_n1024(chol):
    n, m, seed = 1024, 64, 1  # bench.py's adjoint leg
    bw = synth.rhs(n, 2 * m, seed=seed + 11, device="cuda")
    o = chol.opts(nb=128, num_workers=32)
    for i in (0, 31, m - 1):
        A = chol.colmajor(synth.gram_spd(n, seed=seed + 100 + i, device="cuda"))
        b = chol.colmajor(bw[:, i:i + 1])
        w = chol.colmajor(bw[:, m + i:m + i + 1])
        F = A.clone()
        chol.factor(F, o, check=True)
        X = b.clone()
        chol.solve(F, X)
        _, Lbar = chol.solve_backward(F, X, w)
        Abar = chol.cholesky_backward(F, Lbar)
        torch.cuda.synchronize()
        # oracle: the same chain of adjoints on the oracle's factor
        An = A.cpu().numpy()
        Lo = oracle.factor(An)
        xo = oracle.solve(Lo, b.cpu().numpy())
        _, Lbar_o = oadj.solve_backward(Lo, xo, w.cpu().numpy())
        Abar_o = oadj.cholesky_backward(Lo, Lbar_o)
        assert oracle.rel_frobenius(Abar.cpu().numpy(), Abar_o) <= 1e-10, i


def test_lu_n8192(chol):
    n, k = 8192, 1024
    o = chol.opts(nb=0)
    nb = 128
    A0 = chol.colmajor(synth.general_matrix(n, seed=1 + 11, device="cuda"))  # bench.py's LU input (seed 1)
    A = A0.clone()
    f = chol.lu_factor(A, o)
    torch.cuda.synchronize()
    assert int(f.info.item()) == 0
    T, Tk = n // nb, k // nb
    Ak = A0[:k, :k].cpu().numpy()
    Fr, pr, Lr, info = olu.lu_incpiv(Ak, nb)
    assert info == 0
    F = A[:k, :k].cpu().numpy()
    P = f.piv.cpu().numpy()
    W = f.lw.cpu().numpy()
    tol = max(1e-12, np.linalg.cond(Ak) * k * 2.0 ** -53)
    got, ref = [], []
    for kk in range(Tk):
        cols = slice(kk * nb, (kk + 1) * nb)
        for i in range(kk, Tk):
            rows = slice(i * nb, (i + 1) * nb)
            off = (kk * T + i) * nb
            np.testing.assert_array_equal(P[off:off + nb], pr[(i, kk)])
            if i == kk:
                got.append(np.tril(F[rows, cols], -1).ravel())
                ref.append(np.tril(Fr[rows, cols], -1).ravel())
            else:
                got.append(F[rows, cols].ravel())
                ref.append(Fr[rows, cols].ravel())
                woff = (kk * T + i) * olu.IB * nb
                got.append(W[woff:woff + olu.IB * nb].reshape(nb, olu.IB).T.ravel())
                ref.append(Lr[(i, kk)].ravel())
    got, ref = np.concatenate(got), np.concatenate(ref)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    # multipliers bounded by 1 everywhere (strict lower part of the tiled factor and Lw)
    low = torch.tril(A, -1)
    assert float(low.abs().max()) <= 1.0
    assert float(f.lw.abs().max()) <= 1.0
    # backward error of a solve against the classical bound n u rho
    rho = float(torch.triu(A).abs().max() / A0.abs().max())
    b = chol.colmajor(synth.rhs(n, 2, seed=5, device="cuda"))
    x = b.clone()
    chol.lu_solve(f, x)
    torch.cuda.synchronize()
    R = b - A0 @ x
    berr = float((R.abs().amax(0) / (A0.abs().sum(1).amax() * x.abs().amax(0) + b.abs().amax(0))).amax())
    assert berr <= n * 1.11e-16 * rho
