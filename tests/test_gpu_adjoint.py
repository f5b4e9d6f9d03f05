"""GPU checks of the Cholesky and solve adjoints against the reference gradients and against
central finite differences (FP64). Tolerances: relative Frobenius 1e-10 against the oracle's
gradients on well-conditioned Gram matrices; 1e-6 against finite differences (h = 1e-6)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adjoint
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chol():
    import paper_1402_6601_gb300 as c
    return c


def _cm(chol, a):
    return chol.colmajor(torch.from_numpy(np.ascontiguousarray(a)).to("cuda"))


@pytest.mark.parametrize("n", [64, 200, 1000])
def test_cholesky_backward_matches_reference(chol, n):
    rng = np.random.default_rng(n)
    A = synth.gram_spd(n, seed=n).numpy()
    L = oracle.factor(A)
    Lbar = np.tril(rng.standard_normal((n, n)))
    got = chol.cholesky_backward(_cm(chol, L), _cm(chol, Lbar + np.triu(np.full((n, n), 9.0), 1)))
    torch.cuda.synchronize()
    ref = adjoint.cholesky_backward(L, Lbar)
    assert oracle.rel_frobenius(got.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("n,nrhs", [(64, 1), (333, 3), (1024, 64)])
def test_solve_backward_matches_reference(chol, n, nrhs):
    rng = np.random.default_rng(7 + n)
    A = synth.gram_spd(n, seed=n + 3).numpy()
    L = oracle.factor(A)
    B = rng.standard_normal((n, nrhs))
    X = oracle.solve(L, B)
    W = rng.standard_normal((n, nrhs))
    Bbar, Lbar = chol.solve_backward(_cm(chol, L), _cm(chol, X), _cm(chol, W))
    torch.cuda.synchronize()
    rB, rL = adjoint.solve_backward(L, X, W)
    assert oracle.rel_frobenius(Bbar.cpu().numpy(), rB) <= 1e-10
    assert oracle.rel_frobenius(Lbar.cpu().numpy(), rL) <= 1e-10
    assert np.all(np.triu(Lbar.cpu().numpy(), 1) == 0)


@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_solve_matches_closed_form(chol, recompute):
    n, nrhs = 300, 2
    rng = np.random.default_rng(5)
    A = synth.gram_spd(n, seed=17).numpy()
    B = rng.standard_normal((n, nrhs))
    W = rng.standard_normal((n, nrhs))
    At = _cm(chol, A).requires_grad_(True)
    Bt = _cm(chol, B).requires_grad_(True)
    X = chol.solve_spd(At, Bt, nb=64, recompute=recompute)
    loss = (X * torch.from_numpy(W).to("cuda")).sum()
    loss.backward()
    torch.cuda.synchronize()
    np.testing.assert_allclose(X.detach().cpu().numpy(), np.linalg.solve(A, B), rtol=1e-11, atol=1e-12)
    assert oracle.rel_frobenius(At.grad.cpu().numpy(), adjoint.solve_grad_A(A, B, W)) <= 1e-10
    assert oracle.rel_frobenius(Bt.grad.cpu().numpy(), np.linalg.solve(A, W)) <= 1e-10


def test_recompute_gives_identical_gradient(chol):
    n = 256
    A = synth.gram_spd(n, seed=4).numpy()
    b = np.random.default_rng(1).standard_normal(n)
    grads = []
    for rc in (False, True):
        At = _cm(chol, A).requires_grad_(True)
        x = chol.solve_spd(At, torch.from_numpy(b).to("cuda"), nb=64, recompute=rc)
        x.sum().backward()
        grads.append(At.grad.cpu().numpy())
    np.testing.assert_array_equal(grads[0], grads[1])


def test_adjoint_against_central_finite_differences(chol):
    # the loss of the differentiation workload: sum(w * x), x = A^-1 b, n = 64
    n = 64
    rng = np.random.default_rng(64)
    A = synth.gram_spd(n, seed=64).numpy()
    b = rng.standard_normal(n)
    w = rng.standard_normal(n)
    At = _cm(chol, A).requires_grad_(True)
    x = chol.solve_spd(At, torch.from_numpy(b).to("cuda"), nb=16)
    (x * torch.from_numpy(w).to("cuda")).sum().backward()
    G = At.grad.cpu().numpy()
    f = lambda M: float(w @ oracle.solve(oracle.factor(M), b))
    h = 1e-6
    for (i, j) in [(0, 0), (63, 0), (40, 17), (63, 63), (5, 4)]:
        E = np.zeros((n, n))
        E[i, j] = E[j, i] = 1.0
        fd = (f(A + h * E) - f(A - h * E)) / (2 * h)
        fd = fd if i == j else 0.5 * fd
        assert abs(G[i, j] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, j, G[i, j], fd)


def test_autograd_cholesky_factor(chol):
    n = 200
    rng = np.random.default_rng(9)
    A = synth.gram_spd(n, seed=9).numpy()
    Lbar = np.tril(rng.standard_normal((n, n)))
    At = _cm(chol, A).requires_grad_(True)
    L = chol.cholesky(At, nb=64)
    (L * torch.from_numpy(Lbar).to("cuda")).sum().backward()
    torch.cuda.synchronize()
    np.testing.assert_allclose(L.detach().cpu().numpy(), oracle.factor(A), rtol=1e-12, atol=1e-13)
    ref = adjoint.cholesky_backward(oracle.factor(A), Lbar)
    assert oracle.rel_frobenius(At.grad.cpu().numpy(), ref) <= 1e-10


def test_inputs_are_not_modified(chol):
    n = 128
    A = synth.gram_spd(n, seed=2).numpy()
    At = _cm(chol, A).requires_grad_(True)
    b = torch.ones(n, dtype=torch.float64, device="cuda", requires_grad=True)
    chol.solve_spd(At, b, nb=32).sum().backward()
    chol.cholesky(At, nb=32).sum().backward()
    np.testing.assert_array_equal(At.detach().cpu().numpy(), A)
    assert torch.all(b.detach() == 1.0)
