"""GPU checks of the FP32 tile factor and of the mixed-precision solver with FP64 refinement.

FP32 factor: integer data stays exact in FP32 while every intermediate is an integer below
2^24 (here |a_ij| <= 64 n), so L must come back bitwise; on Gram matrices (kappa <= 5) the
FP32 factor must match the FP64 oracle within relative Frobenius 2e-5 (~ n u_32 growth).
Refinement: the backward error must reach 1e-14 (the accuracy target of the FP64 path) on
matrices with kappa = 1e6, and X must match the oracle's FP64 solution within kappa * 1e-14
(forward error <= kappa * backward error).
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
    # refinement stops at backward error eta <= 1e-14, so the forward error is only bounded by
    # kappa(A) * eta (the standard perturbation bound for A x = b): 1e6 * 1e-14
    Xref = oracle.solve(oracle.factor(A), B)
    assert oracle.rel_frobenius(Xh, Xref) <= 1e6 * 1e-14
    # inputs untouched
    np.testing.assert_array_equal(Bd.cpu().numpy(), B)
    np.testing.assert_array_equal(Ad.cpu().numpy(), A)


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
