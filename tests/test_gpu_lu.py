"""GPU parity of the tile LU with incremental pivoting (the paper's DGETRF workload, Section
4.1) against the oracle on the same input bytes.

Tolerances (derived from the arithmetic): both sides run the same pivoted elimination in
binary64, the GPU with fused multiply-adds and the oracle with separately rounded products,
so the two factorizations differ by rounding only: each is the exact factorization of a
matrix within gamma_n ~ n u of A entrywise, and the factors move by at most the condition
number times that, so F and the L11 blocks must agree within relative Frobenius error
max(1e-12, kappa_2(A) n u) (u = 2^-53; the L11 blocks come from cancelling updates inside a
panel and are the most sensitive part); the pivots identical (the argmax decisions are taken in
binary64 on both sides); the solution within kappa_2(A) 1e-14 of the oracle's; the solve's
normwise backward error <= 1e-14 at these orders (incremental pivoting lets the growth factor
rise with n, so at the full order the bound is n u rho, rho the growth factor, in
test_gpu_fullsize.py). Dyadic inputs whose every intermediate is exact must match bitwise,
and so must factors made under different scheduling policies (every tile's update sequence
is fixed by the graph).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import lu as olu

pytestmark = pytest.mark.gpu

REL_F = 1e-12
BERR = 1e-14


@pytest.fixture(scope="module")
def chol():
    import paper_1402_6601_gb300 as c
    return c


def _run(chol, A, o):
    Ad = chol.colmajor(torch.from_numpy(np.ascontiguousarray(A)).to("cuda"))
    f = chol.lu_factor(Ad, o)
    torch.cuda.synchronize()
    return f


def _unpack(f, n, nb):
    """(F, piv dict, Lw dict) from the library's outputs, in the oracle's layout."""
    T = olu.tiles(n, nb)
    F = f.F.cpu().numpy()
    P = f.piv.cpu().numpy()
    W = f.lw.cpu().numpy()
    piv, Lw = {}, {}
    for k in range(T):
        nk = min(nb, n - k * nb)
        for i in range(k, T):
            off = (k * T + i) * nb
            piv[(i, k)] = P[off:off + nk].astype(np.int64)
            if i > k:
                woff = (k * T + i) * olu.IB * nb
                Lw[(i, k)] = W[woff:woff + olu.IB * nk].reshape(nk, olu.IB).T
    return F, piv, Lw


U_ROUND = 2.0 ** -53


def _tol(A):
    return max(REL_F, np.linalg.cond(A) * A.shape[0] * U_ROUND)


def _compare(F, piv, Lw, ref, tol):
    Fr, pr, Lr, _ = ref
    for key in pr:
        np.testing.assert_array_equal(piv[key], pr[key], err_msg="pivots of %s" % (key,))
    assert oracle.rel_frobenius(F, Fr) <= tol
    if Lr:
        got = np.concatenate([Lw[key].ravel() for key in sorted(Lr)])
        ref_lw = np.concatenate([Lr[key].ravel() for key in sorted(Lr)])
        assert np.linalg.norm(got - ref_lw) <= tol * max(np.linalg.norm(ref_lw), 1.0)


@pytest.mark.parametrize("n,nb", [(300, 64), (520, 128), (129, 32), (1000, 128), (256, 256), (77, 16), (1, 16)])
def test_lu_parity_general(chol, n, nb):
    A = synth.general_matrix(n, seed=n + nb).numpy()
    f = _run(chol, A, chol.opts(nb=nb))
    assert int(f.info.item()) == 0
    F, piv, Lw = _unpack(f, n, nb)
    _compare(F, piv, Lw, olu.lu_incpiv(A, nb), _tol(A))


@pytest.mark.parametrize("n,nb", [(260, 64), (200, 128), (97, 32)])
def test_lu_dyadic_bitwise(chol, n, nb):
    L, U, A = synth.dyadic_lu(n, seed=n)
    f = _run(chol, A, chol.opts(nb=nb))
    assert int(f.info.item()) == 0
    F, piv, Lw = _unpack(f, n, nb)
    Fr, pr, Lr, _ = olu.lu_incpiv(A, nb)
    np.testing.assert_array_equal(F, Fr)
    np.testing.assert_array_equal(np.triu(F), U)
    for key in pr:
        np.testing.assert_array_equal(piv[key], pr[key])
    for key in Lr:
        assert not Lw[key].any()
    X = synth.integer_vector(n, 5, seed=n)
    Bd = chol.colmajor(torch.from_numpy(A @ X).to("cuda"))
    chol.lu_solve(f, Bd)
    np.testing.assert_array_equal(Bd.cpu().numpy(), X)


@pytest.mark.parametrize("policy,alpha,cp", [("dada", 0.0, False), ("dada", 0.5, False), ("dada", 1.0, True),
                                             ("steal", 0.5, False), ("static", 0.5, False), ("heft", 0.5, True)])
def test_lu_schedule_invariance_bitwise(chol, policy, alpha, cp):
    n, nb = 700, 64
    A = synth.general_matrix(n, seed=9).numpy()
    ref = _run(chol, A, chol.opts(nb=nb))
    got = _run(chol, A, chol.opts(nb=nb, policy=policy, alpha=alpha, use_cp=cp))
    assert int(got.info.item()) == 0
    assert torch.equal(got.F, ref.F) and torch.equal(got.piv, ref.piv) and torch.equal(got.lw, ref.lw)


@pytest.mark.parametrize("n,nb,nrhs", [(1000, 128, 70), (300, 64, 1), (33, 16, 3), (512, 256, 64), (400, 64, 13),
                                       (250, 128, 6)])
def test_lu_solve_backward_error_and_parity(chol, n, nb, nrhs):
    A = synth.general_matrix(n, seed=2 * n).numpy()
    B = synth.rhs(n, nrhs, seed=2 * n + 1).numpy()
    f = _run(chol, A, chol.opts(nb=nb))
    Bd = chol.colmajor(torch.from_numpy(B).to("cuda"))
    chol.lu_solve(f, Bd)
    X = Bd.cpu().numpy()
    assert oracle.backward_error(A, X, B) <= BERR
    Fr, pr, Lr, _ = olu.lu_incpiv(A, nb)
    Xr = olu.lu_solve(Fr, pr, Lr, nb, B)
    assert oracle.rel_frobenius(X, Xr) <= np.linalg.cond(A) * 1e-14


def test_lu_singular_column_reported(chol):
    n, nb = 300, 64
    A = synth.general_matrix(n, seed=5).numpy()
    A[:, 150] = 0.0
    f = _run(chol, A, chol.opts(nb=nb))
    _, _, _, info = olu.lu_incpiv(A, nb)
    assert int(f.info.item()) == info == 151


def test_lu_timeout_is_reported_not_hung(chol):
    # task 7 gets an extra dependency nobody satisfies: every worker's bounded wait expires
    n, nb = 512, 64
    A = synth.general_matrix(n, seed=4).numpy()
    f = _run(chol, A, chol.opts(nb=nb, timeout_ns=200_000_000, hold_task=7))
    assert int(f.info.item()) == chol.INFO_TIMEOUT
    g = _run(chol, A, chol.opts(nb=nb))
    assert int(g.info.item()) == 0


def test_lu_argument_checks(chol):
    import ctypes
    o = chol.opts(nb=512)  # above the LU tile limit
    assert chol.lib.chol_lu_workspace_size(1000, ctypes.byref(o)) == 0
    o = chol.opts(nb=128)
    assert chol.lib.chol_lu_factor(100, None, 100, None, None, ctypes.byref(o), None, 0, None, None) == -1
