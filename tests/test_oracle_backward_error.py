"""Pins of ``oracle.backward_error``, the normwise backward error every accuracy target of
the suite is stated in (the paper states no norm; the reading is Rigal and Gaches' normwise
backward error in the infinity norm, maximised over the right-hand sides).

Three independent checks, each chosen so that a plausible slip in the function fails one:
* values worked by hand (``tests/golden/backward_error_worked_example.txt``) on matrices
  whose row-sum and column-sum norms differ, with the slips' values written beside them;
* the Rigal-Gaches construction: for a random x the perturbation
  dA = (||A|| / d) r z^T, db = -(||b|| / d) r (d = ||A|| ||x|| + ||b||, z^T x = ||x||,
  ||z||_1 = 1) makes x an exact solution of (A + dA) x = b + db with relative sizes exactly
  eta, so eta is attained;
* minimality: every split of r between dA and db (dA = t r z^T / ||x||, db = -(1 - t) r)
  needs a relative size max(t ||r|| / (||A|| ||x||), (1 - t) ||r|| / ||b||) >= eta, with
  equality at one t -- so the function is the smallest such size, not merely an upper bound.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    cases = []
    cur = None
    for line in open(os.path.join(HERE, "golden", "backward_error_worked_example.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tag, *rest = line.split()
        if tag == "case":
            cur = {"name": rest[0], "n": int(rest[1]), "nrhs": int(rest[2]), "A": [], "X": [], "B": []}
            cases.append(cur)
        elif tag in ("A", "X", "B"):
            cur[tag].append([float(v) for v in rest])
        elif tag == "eta":
            cur["eta"] = Fraction(rest[0])
    for c in cases:
        c["A"] = np.array(c["A"])
        c["X"] = np.array(c["X"]).T   # stored column by column
        c["B"] = np.array(c["B"]).T
        assert c["A"].shape == (c["n"], c["n"]) and c["X"].shape == (c["n"], c["nrhs"])
    return cases


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_worked_values(case):
    eta = oracle.backward_error(case["A"], case["X"], case["B"])
    assert eta == pytest.approx(float(case["eta"]), rel=1e-15)


def _slips(A, X, B):
    """The values that the plausible slips would give on these inputs."""
    R = B - A @ X
    num = np.abs(R).max(axis=0)
    xn = np.abs(X).max(axis=0)
    bn = np.abs(B).max(axis=0)
    row = np.abs(A).sum(axis=1).max()
    col = np.abs(A).sum(axis=0).max()
    amax = np.abs(A).max()
    return {
        "column-sum norm": (num / (col * xn + bn)).max(),
        "entry-max norm": (num / (amax * xn + bn)).max(),
        "||b|| dropped": (num / (row * xn)).max(),
        "first column only": (num / (row * xn + bn))[0],
        "sum over columns": (num / (row * xn + bn)).sum(),
    }


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_slips_give_other_values(case):
    # the hand-worked inputs separate the definition from each slip: if the function made one
    # of these mistakes, test_hand_worked_values would fail
    eta = float(case["eta"])
    for name, v in _slips(case["A"], case["X"], case["B"]).items():
        if case["nrhs"] == 1 and name in ("first column only", "sum over columns"):
            continue
        assert abs(v - eta) > 1e-3 * eta, name


def _random_problem(seed, n, nrhs):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) * rng.uniform(0.1, 10.0, size=(n, 1))  # rows of uneven size
    X = rng.standard_normal((n, nrhs))
    B = A @ X + 1e-3 * rng.standard_normal((n, nrhs))
    return A, X, B


@pytest.mark.parametrize("seed,n,nrhs", [(0, 7, 1), (1, 33, 3), (2, 100, 5)])
def test_rigal_gaches_perturbation_attains_eta(seed, n, nrhs):
    A, X, B = _random_problem(seed, n, nrhs)
    eta = oracle.backward_error(A, X, B)
    normA = np.abs(A).sum(axis=1).max()
    etas = []
    for c in range(nrhs):
        x, b = X[:, c], B[:, c]
        r = b - A @ x
        d = normA * np.abs(x).max() + np.abs(b).max()
        p = int(np.argmax(np.abs(x)))
        z = np.zeros(n)
        z[p] = np.sign(x[p])                 # z^T x = ||x||_inf, ||z||_1 = 1
        dA = (normA / d) * np.outer(r, z)
        db = -(np.abs(b).max() / d) * r
        # x solves the perturbed system exactly (to rounding)
        lhs = (A + dA) @ x
        np.testing.assert_allclose(lhs, b + db, rtol=0, atol=1e-13 * (normA * np.abs(x).max() + np.abs(b).max()))
        ea = np.abs(dA).sum(axis=1).max() / normA
        eb = np.abs(db).max() / np.abs(b).max()
        assert ea == pytest.approx(eb, rel=1e-12)
        etas.append(ea)
    assert eta == pytest.approx(max(etas), rel=1e-12)


@pytest.mark.parametrize("seed,n", [(3, 9), (4, 50)])
def test_eta_is_the_smallest_perturbation(seed, n):
    A, X, B = _random_problem(seed, n, 1)
    x, b = X[:, 0], B[:, 0]
    eta = oracle.backward_error(A, x, b)
    r = b - A @ x
    nr = np.abs(r).max()
    normA = np.abs(A).sum(axis=1).max()
    nx, nb = np.abs(x).max(), np.abs(b).max()
    t = np.linspace(0.0, 1.0, 20001)
    size = np.maximum(t * nr / (normA * nx), (1.0 - t) * nr / nb)
    assert size.min() >= eta * (1 - 1e-12)
    assert size.min() == pytest.approx(eta, rel=1e-3)   # grid spacing
    # the balanced split t* = ||A|| ||x|| / d gives exactly eta
    ts = normA * nx / (normA * nx + nb)
    assert max(ts * nr / (normA * nx), (1 - ts) * nr / nb) == pytest.approx(eta, rel=1e-13)


def test_exact_solution_and_zero_rhs():
    A = np.array([[2.0, 1.0], [1.0, 3.0]])
    x = np.array([1.0, -1.0])
    assert oracle.backward_error(A, x, A @ x) == 0.0
    # x = 0 with b != 0: r = b, eta = ||b|| / ||b|| = 1 (the largest possible value)
    assert oracle.backward_error(A, np.zeros(2), np.array([1.0, 2.0])) == 1.0
