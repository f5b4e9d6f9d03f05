"""GPU checks of the FP32 tile factor and of the mixed-precision solver with FP64 refinement.

FP32 factor: integer data stays exact in FP32 while every intermediate is an integer below
2^24 (here |a_ij| <= 64 n), so L must come back bitwise; on Gram matrices (kappa <= 5) the
FP32 factor must match the FP64 oracle within relative Frobenius 2e-5 (~ n u_32 growth).
Refinement: the backward error must reach 1e-14 (the accuracy target of the FP64 path) on
matrices with kappa = 1e6, and X must match the oracle's FP64 solution within the forward
error bound 2 kappa_inf eta / (1 - kappa_inf eta) that the backward errors of both imply.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chol():
    import paper_1402_6601_gb300 as c
    return c


def _f32(chol, A_np):
    return chol.colmajor(torch.from_numpy(np.ascontiguousarray(A_np)).to("cuda", torch.float32))


def _assert_forward_error(A, X, B, Xref):
    """Column-wise forward error against the perturbation bound of a normwise (Rigal-Gaches)
    backward error eta: ||x - x*||_inf / ||x*||_inf <= 2 kappa_inf eta / (1 - kappa_inf eta)
    (Higham, Accuracy and Stability, Thm 7.2), kappa_inf = ||A||_inf ||A^-1||_inf computed
    here; Xref (the oracle's FP64 solution) carries its own error, bounded the same way."""
    kinf = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
    for c in range(B.shape[1]):
        eta = oracle.backward_error(A, X[:, c:c + 1], B[:, c:c + 1])
        eta_ref = oracle.backward_error(A, Xref[:, c:c + 1], B[:, c:c + 1])
        bound = sum(2 * kinf * e / (1 - kinf * e) for e in (eta, eta_ref))
        err = np.abs(X[:, c] - Xref[:, c]).max() / np.abs(Xref[:, c]).max()
        assert err <= bound, (c, err, bound)


@pytest.mark.parametrize("n,nb,policy", [(600, 64, "heft"), (700, 128, "dada"), (1030, 256, "steal"),
                                         (1024, 256, "dada")])
def test_f32_integer_factor_bitwise(chol, n, nb, policy):
    L, A = synth.integer_factor(n, seed=n)
    Ad = _f32(chol, A)
    info, _ = chol.factor_f32(Ad, chol.opts(nb=nb, policy=policy))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    np.testing.assert_array_equal(np.tril(Ad.cpu().numpy().astype(np.float64)), L)


@pytest.mark.parametrize("n,nb", [(1024, 128), (1000, 256), (333, 64)])
def test_f32_factor_parity(chol, n, nb):
    A = synth.gram_spd(n, seed=n).numpy()
    Ad = _f32(chol, A)
    info, _ = chol.factor_f32(Ad, chol.opts(nb=nb))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    rel = oracle.rel_frobenius(np.tril(Ad.cpu().numpy().astype(np.float64)), oracle.factor(A))
    assert rel <= 2e-5


@pytest.mark.parametrize("n,nrhs,nb", [(1024, 4, 128), (777, 16, 256), (520, 1, 64)])
def test_refine_reaches_fp64_backward_error(chol, n, nrhs, nb):
    A = synth.householder_spd(n, seed=3, cond=1e6).numpy()
    B = synth.rhs(n, nrhs, seed=4).numpy()
    Ad = chol.colmajor(torch.from_numpy(A).to("cuda"))
    Bd = chol.colmajor(torch.from_numpy(B).to("cuda"))
    X, info, iters, berr = chol.solve_refine(Ad, Bd, tol=1e-14, max_iter=40, o=chol.opts(nb=nb))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    Xh = X.cpu().numpy()
    eta = oracle.backward_error(A, Xh, B)
    assert eta <= 1e-14, (eta, int(iters.item()))
    assert float(berr.item()) <= 1e-14
    assert 1 <= int(iters.item()) <= 40
    # refinement stops at backward error eta <= 1e-14: the forward error is bounded through
    # the condition number
    _assert_forward_error(A, Xh, B, oracle.solve(oracle.factor(A), B))
    # inputs untouched
    np.testing.assert_array_equal(Bd.cpu().numpy(), B)
    np.testing.assert_array_equal(Ad.cpu().numpy(), A)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (63, 2), (64, 16), (65, 5), (127, 1), (128, 3), (777, 16), (1100, 33),
                                    (1024, 64), (4097, 16), (3000, 1)])
def test_f32_solve_matches_oracle_substitution(chol, n, nrhs):
    """The first refinement step from x0 = 0 returns the FP32 forward and back substitution of
    b (rounded to FP32) with the FP32 factor (no diagonal scaling in this form). The oracle
    substitutes in FP64 with the same factor and right-hand sides; the difference is the FP32
    substitution's rounding error (kappa(A) <= 5 here), far below the O(1) error of a wrong
    block, chunk or transposed inverse. Sizes: one item, ragged last items (64-row items),
    one to two 32-column groups."""
    A = synth.gram_spd(n, seed=5).numpy()
    B = synth.rhs(n, nrhs, seed=6).numpy()
    Ad = chol.colmajor(torch.from_numpy(A).to("cuda"))
    Bd = chol.colmajor(torch.from_numpy(B).to("cuda"))
    o = chol.opts(nb=128)
    X, info, iters, _ = chol.solve_refine(Ad, Bd, tol=0.0, max_iter=1, o=o, precision="f32")
    L32 = chol.colmajor(torch.from_numpy(A).to("cuda").float())
    chol.factor_f32(L32, o, check=True)
    torch.cuda.synchronize()
    assert int(info.item()) == 0 and int(iters.item()) == 1
    L = np.tril(L32.cpu().numpy().astype(np.float64))
    ref = oracle.solve(L, B.astype(np.float32).astype(np.float64))
    got = X.cpu().numpy()
    err = np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)
    assert err.max() <= 1e-4, err.max()


def test_refine_reports_indefinite(chol):
    n = 300
    A = synth.gram_spd(n, seed=1).numpy()
    A[150, 150] = -5.0
    B = synth.rhs(n, 2, seed=2).numpy()
    Ad = chol.colmajor(torch.from_numpy(A).to("cuda"))
    Bd = chol.colmajor(torch.from_numpy(B).to("cuda"))
    X, info, iters, berr = chol.solve_refine(Ad, Bd, o=chol.opts(nb=64))
    torch.cuda.synchronize()
    assert int(info.item()) == 151
    assert np.isinf(float(berr.item()))
    assert int(iters.item()) == 0


# ---- tensor-core forms of the low-precision factor (tcgen05, BF16 operands, FP32 accumulation)

@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("n,nb,policy", [(600, 64, "heft"), (1030, 256, "dada"), (1024, 256, "heft")])
def test_tc_integer_factor_bitwise(chol, precision, n, nb, policy):
    # the update operands are entries of L (integers in [-8, 8]: exact in one BF16 term) and
    # every partial sum is an integer below 2^24, so both forms must return L bitwise
    L, A = synth.integer_factor(n, seed=n + 1)
    Ad = _f32(chol, A)
    info, _ = chol.factor_f32(Ad, chol.opts(nb=nb, policy=policy), precision=precision)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    np.testing.assert_array_equal(np.tril(Ad.cpu().numpy().astype(np.float64)), L)


@pytest.mark.parametrize("n,nb", [(1024, 128), (1000, 256), (333, 64)])
def test_bf16x3_factor_parity(chol, n, nb):
    # three BF16 terms carry all 24 bits of an FP32 operand: FP32-level agreement
    A = synth.gram_spd(n, seed=n).numpy()
    Ad = _f32(chol, A)
    info, _ = chol.factor_f32(Ad, chol.opts(nb=nb), precision="bf16x3")
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    rel = oracle.rel_frobenius(np.tril(Ad.cpu().numpy().astype(np.float64)), oracle.factor(A))
    assert rel <= 2e-5


@pytest.mark.parametrize("n,nb", [(1024, 128), (1000, 256)])
def test_bf16_factor_parity(chol, n, nb):
    # one BF16 term: each update operand carries a relative error <= u = 2^-9, so the Schur
    # complements, and with kappa(A) <= 5 the factor, are off by a few u times sqrt(growth)
    A = synth.gram_spd(n, seed=n).numpy()
    Ad = _f32(chol, A)
    info, _ = chol.factor_f32(Ad, chol.opts(nb=nb), precision="bf16")
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    rel = oracle.rel_frobenius(np.tril(Ad.cpu().numpy().astype(np.float64)), oracle.factor(A))
    assert 1e-6 < rel <= 16 * 2.0 ** -9, rel


@pytest.mark.parametrize("n,nrhs,nb", [(1024, 4, 128), (777, 16, 256)])
def test_refine_bf16x3_reaches_fp64_backward_error(chol, n, nrhs, nb):
    A = synth.householder_spd(n, seed=3, cond=1e6).numpy()
    B = synth.rhs(n, nrhs, seed=4).numpy()
    Ad = chol.colmajor(torch.from_numpy(A).to("cuda"))
    Bd = chol.colmajor(torch.from_numpy(B).to("cuda"))
    X, info, iters, berr = chol.solve_refine(Ad, Bd, tol=1e-14, max_iter=40, o=chol.opts(nb=nb),
                                             precision="bf16x3")
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    Xh = X.cpu().numpy()
    assert oracle.backward_error(A, Xh, B) <= 1e-14
    assert float(berr.item()) <= 1e-14
    _assert_forward_error(A, Xh, B, oracle.solve(oracle.factor(A), B))


def test_refine_bf16_well_conditioned(chol):
    # plain BF16 operands: refinement contracts when kappa(A) u_bf16 < 1 (Gram, kappa <= 5)
    n, nrhs = 1024, 4
    A = synth.gram_spd(n, seed=5).numpy()
    B = synth.rhs(n, nrhs, seed=6).numpy()
    Ad = chol.colmajor(torch.from_numpy(A).to("cuda"))
    Bd = chol.colmajor(torch.from_numpy(B).to("cuda"))
    X, info, iters, berr = chol.solve_refine(Ad, Bd, tol=1e-14, max_iter=40, o=chol.opts(nb=128),
                                             precision="bf16")
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert oracle.backward_error(A, X.cpu().numpy(), B) <= 1e-14
    assert int(iters.item()) >= 2  # a BF16 factor alone cannot reach it


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
def test_refine_scaled_forms_wide_diagonal_and_zero_blocks(chol, precision):
    # A = D M D with D = diag(2^u), u in [-40, 40], and M two independent Gram blocks (the
    # off-diagonal blocks exactly zero): entries span 2^-80 .. 2^81, far outside what one
    # FP32 exponent range keeps accurate together; the power-of-two diagonal scaling maps A
    # back to a matrix within a factor two of M's scaling exactly (the zeros take the FP64
    # product path of the conversion). Refinement must reach the FP64 target as on M.
    n, nrhs = 512, 3
    rng = np.random.default_rng(11)
    M = np.zeros((n, n))
    M[:256, :256] = synth.gram_spd(256, seed=12).numpy()
    M[256:, 256:] = synth.gram_spd(256, seed=13).numpy()
    d = np.ldexp(1.0, rng.integers(-40, 41, n))
    A = d[:, None] * M * d[None, :]  # exact: powers of two
    B = synth.rhs(n, nrhs, seed=14).numpy()
    Ad = chol.colmajor(torch.from_numpy(A).to("cuda"))
    Bd = chol.colmajor(torch.from_numpy(B).to("cuda"))
    X, info, iters, berr = chol.solve_refine(Ad, Bd, tol=1e-14, max_iter=40, o=chol.opts(nb=128),
                                             precision=precision)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert oracle.backward_error(A, X.cpu().numpy(), B) <= 1e-14
    assert float(berr.item()) <= 1e-14


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("n,nb", [(700, 80), (1100, 512)])
def test_tc_register_staged_path(chol, precision, n, nb):
    # tiles that are not a multiple of 32, or larger than 256, have no pre-split side buffer:
    # the tensor-core update splits its FP32 operands itself (integer data stays exact)
    L, A = synth.integer_factor(n, seed=n + 3)
    Ad = _f32(chol, A)
    info, _ = chol.factor_f32(Ad, chol.opts(nb=nb), precision=precision)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    np.testing.assert_array_equal(np.tril(Ad.cpu().numpy().astype(np.float64)), L)
    if precision == "bf16x3":
        G = synth.gram_spd(n, seed=n).numpy()
        Gd = _f32(chol, G)
        info, _ = chol.factor_f32(Gd, chol.opts(nb=nb), precision=precision)
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        assert oracle.rel_frobenius(np.tril(Gd.cpu().numpy().astype(np.float64)), oracle.factor(G)) <= 2e-5


def test_refine_overflowing_fp32_norm_reports_nan(chol):
    # A = 2e37 (G G^T / n + I): every entry is finite in FP32 and so is the factor (L scales by
    # ~4.5e18), but the FP32 row sums of |a_ij| (up to ~4.8e38 > FLT_MAX) overflow. The solver
    # must not read the resulting eta = 0 as convergence: no step is taken, X stays zero and
    # the backward error is NaN.
    n = 512
    A = 2e37 * synth.gram_spd(n, seed=9).numpy()
    B = 2e37 * synth.rhs(n, 2, seed=10).numpy()
    Ad = chol.colmajor(torch.from_numpy(A).to("cuda"))
    Bd = chol.colmajor(torch.from_numpy(B).to("cuda"))
    X, info, iters, berr = chol.solve_refine(Ad, Bd, tol=1e-14, max_iter=5, o=chol.opts(nb=128))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert np.isnan(float(berr.item()))
    assert int(iters.item()) == 0
    assert not X.abs().max().item()


@pytest.mark.parametrize("precision", ["f32", "bf16x3", "bf16"])
def test_lowp_factor_split_and_kept_bitwise(chol, precision):
    # split TRSM bands (with their BF16 terms written band by band), split FFMA SYRK / GEMM
    # blocks and kept successors change who computes what, not how
    n = 1100  # ragged last tile
    A = synth.gram_spd(n, seed=31).numpy()
    ref = None
    for split in (0, 1, 2):
        for keep in (0, 1):
            for nw in (0, 3):
                Ad = _f32(chol, A)
                info, _ = chol.factor_f32(Ad, chol.opts(nb=256, split=split, keep_next=keep, num_workers=nw),
                                          precision=precision)
                torch.cuda.synchronize()
                assert int(info.item()) == 0
                L = np.tril(Ad.cpu().numpy())
                if ref is None:
                    ref = L
                    tol = 16 * 2.0 ** -9 if precision == "bf16" else 2e-5  # as in the parity tests above
                    assert oracle.rel_frobenius(L.astype(np.float64), oracle.factor(A)) <= tol
                else:
                    np.testing.assert_array_equal(L, ref, err_msg=str((split, keep, nw)))


@pytest.mark.parametrize("precision,nb", [("f32", 77), ("bf16x3", 80)])
def test_lowp_factor_odd_tile_and_leading_dimension(chol, precision, nb):
    # lda 503 (and tile 77): the band TRSM's 16-byte asynchronous copies of L cannot start on
    # 16-byte boundaries everywhere and fall back to plain loads piece by piece
    n, lda = 500, 503
    L, A = synth.integer_factor(n, seed=12)
    buf = torch.zeros(n, lda, dtype=torch.float32, device="cuda")   # column j at buf[j, :]
    buf[:, :n] = torch.from_numpy(A.T.astype(np.float32)).to("cuda")
    Ad = buf.t()[:n, :]                                              # n x n view, stride (1, lda)
    assert Ad.stride() == (1, lda)
    info, _ = chol.factor_f32(Ad, chol.opts(nb=nb), precision=precision)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    np.testing.assert_array_equal(np.tril(Ad.cpu().numpy().astype(np.float64)), L)
