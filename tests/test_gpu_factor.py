"""GPU parity of the tiled Cholesky factor and solves against the oracle (same input bytes).

Tolerances: the FP64 factor must match the oracle's L within relative Frobenius error
1e-12 (kappa(A) <= 5 for the Gram workloads), the solve's normwise backward error must be
<= 1e-14, and integer inputs (exact in binary64 at every step) must match bitwise.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

REL_L = 1e-12
BERR = 1e-14


@pytest.fixture(scope="module")
def chol():
    import paper_1402_6601_gb300 as c
    return c


def _gpu(a):
    t = torch.from_numpy(np.asfortranarray(a)).to("cuda")
    return t.t().contiguous().t() if t.dim() == 2 else t


def _factor(chol, A_np, o, upper_marker=None):
    A = chol.colmajor(torch.from_numpy(np.ascontiguousarray(A_np)).to("cuda"))
    info, work = chol.factor(A, o)
    torch.cuda.synchronize()
    return A.cpu().numpy(), int(info.item()), work


@pytest.mark.parametrize("n,nb", [(1024, 128), (1000, 128), (300, 64), (77, 32), (16, 16), (1, 16),
                                  (520, 256), (1100, 512)])
def test_factor_parity_gram(chol, n, nb):
    A = synth.gram_spd(n, seed=n + nb).numpy()
    F, info, _ = _factor(chol, A, chol.opts(nb=nb))
    assert info == 0
    Lref = oracle.factor(A)
    assert oracle.rel_frobenius(np.tril(F), Lref) <= REL_L
    assert np.all(np.diag(F) > 0)


def test_upper_triangle_untouched(chol):
    n = 700
    A = synth.gram_spd(n, seed=3).numpy()
    Ain = np.tril(A) + np.triu(np.full((n, n), -7.25), 1)
    F, info, _ = _factor(chol, Ain, chol.opts(nb=128))
    assert info == 0
    np.testing.assert_array_equal(np.triu(F, 1), np.triu(Ain, 1))


@pytest.mark.parametrize("n,nb", [(20, 16), (20, 32), (14, 16)])
def test_pascal_bitwise(chol, n, nb):
    F, info, _ = _factor(chol, synth.pascal(n), chol.opts(nb=nb))
    assert info == 0
    np.testing.assert_array_equal(np.tril(F), synth.pascal_lower(n))


@pytest.mark.parametrize("policy,alpha", [("heft", 0.5), ("dada", 0.0), ("dada", 0.5), ("dada", 1.0),
                                          ("steal", 0.5), ("static", 0.5)])
def test_integer_factor_bitwise_every_policy(chol, policy, alpha):
    L, A = synth.integer_factor(600, seed=5)
    F, info, _ = _factor(chol, A, chol.opts(nb=64, policy=policy, alpha=alpha))
    assert info == 0
    np.testing.assert_array_equal(np.tril(F), L)


def test_schedule_invariance_bitwise(chol):
    # every tile's updates are applied in a fixed k order, so L must not depend on the schedule
    n = 900
    A = synth.gram_spd(n, seed=21).numpy()
    ref = None
    configs = [chol.opts(nb=64, policy="heft"), chol.opts(nb=64, policy="dada", alpha=0.0),
               chol.opts(nb=64, policy="dada", alpha=1.0), chol.opts(nb=64, policy="steal"),
               chol.opts(nb=64, policy="static"), chol.opts(nb=64, policy="heft", workers_per_sm=1),
               chol.opts(nb=64, policy="heft", num_workers=3), chol.opts(nb=64, policy="dada", num_workers=1),
               chol.opts(nb=64, policy="dada", alpha=0.5, use_cp=True), chol.opts(nb=64, policy="heft", use_cp=True)]
    for o in configs:
        F, info, _ = _factor(chol, A, o)
        assert info == 0
        if ref is None:
            ref = np.tril(F)
        else:
            np.testing.assert_array_equal(np.tril(F), ref)


@pytest.mark.parametrize("nb", [256, 512])
def test_split_units_and_kept_successors_bitwise(chol, nb):
    # TRSM/SYRK tasks cut into 64-row / 64 x 64 units that other workers help with, and the
    # finishing worker keeping the most urgent successor, change who computes what, not how:
    # every element is computed by the same operations in the same order
    n = 1100
    A = synth.gram_spd(n, seed=23).numpy()
    ref = None
    for split in (0, 1, 2):
        for keep in (0, 1):
            for nw in (0, 1, 3):
                o = chol.opts(nb=nb, split=split, keep_next=keep, num_workers=nw)
                F, info, _ = _factor(chol, A, o)
                assert info == 0
                if ref is None:
                    ref = np.tril(F)
                    assert oracle.rel_frobenius(ref, oracle.factor(A)) <= REL_L
                else:
                    np.testing.assert_array_equal(np.tril(F), ref, err_msg=str((split, keep, nw)))


@pytest.mark.parametrize("policy", ["heft", "dada", "steal"])
def test_integer_factor_bitwise_split_every_task(chol, policy):
    L, A = synth.integer_factor(700, seed=6)
    F, info, _ = _factor(chol, A, chol.opts(nb=256, policy=policy, split=2))
    assert info == 0
    np.testing.assert_array_equal(np.tril(F), L)


@pytest.mark.parametrize("bad", [1, 200, 511, 512, 700])
def test_not_spd_info(chol, bad):
    n = 768
    A = synth.gram_spd(n, seed=8).numpy()
    # make the leading minor of order `bad` indefinite: a_jj far below what the rest needs
    A[bad - 1, bad - 1] = -1.0
    _, info_ref = oracle.cholesky(A)
    assert info_ref == bad
    _, info, _ = _factor(chol, A, chol.opts(nb=128))
    assert info == bad


def test_trace_topological_and_complete(chol):
    import oracle.dag as odag
    n, nb = 640, 64
    T = n // nb
    o = chol.opts(nb=nb, policy="dada", alpha=0.5, trace=True)
    A = chol.colmajor(synth.gram_spd(n, seed=2).to("cuda"))
    info, work = chol.factor(A, o)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    tr = chol.trace(work, n, o).cpu().numpy()
    kind, ti, tj, tk, indeg, ptr, succ = chol.dag_describe(T)
    nw = chol.num_workers(o)
    assert np.all(tr[:, 0] >= 0) and np.all(tr[:, 0] < nw)       # every task ran once
    assert np.all(tr[:, 3] >= tr[:, 2])
    for t in range(len(kind)):
        for s in succ[ptr[t]:ptr[t + 1]]:
            assert tr[s, 2] >= tr[t, 3], (t, s)                    # start after predecessor ends
    assert len(kind) == len(odag.build(T)[0])


def test_timeout_is_reported_not_hung(chol):
    # task 5 gets an extra dependency nobody satisfies: every worker's bounded wait expires
    n, nb = 512, 64
    o = chol.opts(nb=nb, timeout_ns=200_000_000, hold_task=5)
    A = chol.colmajor(synth.gram_spd(n, seed=2).to("cuda"))
    info, _ = chol.factor(A, o)
    torch.cuda.synchronize()
    assert int(info.item()) == chol.INFO_TIMEOUT
    # the context is still usable
    A2 = chol.colmajor(synth.gram_spd(n, seed=2).to("cuda"))
    info2, _ = chol.factor(A2, chol.opts(nb=nb))
    torch.cuda.synchronize()
    assert int(info2.item()) == 0


# right-hand-side counts reach every form of the sweep: one warp per column (<= 4 columns),
# solved blocks split over warps with the eight-warp diagonal solve (5-8), columns split over
# warps (9-16 and 17-32 per group), and ragged last groups
@pytest.mark.parametrize("n,nrhs", [(1024, 1), (1000, 70), (33, 3), (64, 64), (5, 1), (500, 6), (700, 13),
                                    (257, 16), (300, 40)])
def test_solve_parity(chol, n, nrhs):
    A = synth.gram_spd(n, seed=n).numpy()
    B = synth.rhs(n, nrhs, seed=n + 1).numpy()
    Ad = chol.colmajor(torch.from_numpy(A).to("cuda"))
    chol.factor(Ad, chol.opts(nb=128), check=True)
    Bd = _gpu(B)
    chol.solve(Ad, Bd)
    torch.cuda.synchronize()
    X = Bd.cpu().numpy()
    assert oracle.backward_error(A, X, B) <= BERR
    Xref = oracle.solve(oracle.factor(A), B)
    assert oracle.rel_frobenius(X, Xref) <= 1e-12


@pytest.mark.parametrize("n,nrhs", [(200, 1), (333, 65), (300, 6), (260, 16), (100, 40)])
def test_sweeps_exact_on_integers(chol, n, nrhs):
    L, A = synth.integer_factor(n, seed=9)
    X = synth.integer_vector(n, nrhs, 4)
    Y = L.T @ X
    B = L @ Y
    Ld = _gpu(L)
    Bd = _gpu(B)
    chol.trsm_sweep(Ld, Bd, transpose=False)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Bd.cpu().numpy(), Y)
    chol.trsm_sweep(Ld, Bd, transpose=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Bd.cpu().numpy(), X)


@pytest.mark.parametrize("lu", [False, True])
@pytest.mark.parametrize("T", [1, 2, 3, 6, 9])
def test_device_bottom_levels_match_oracle(chol, lu, T):
    # the bottom levels the device computes before each factor launch (Section 3.1's upward
    # rank), against the oracle's longest-path recursion over the access-mode graph
    import oracle.dag as odag
    cost = [11, 30, 29, 60] if lu else [7, 30, 31, 60]
    bl = chol.dag_bottom_levels_device(T, cost, lu=lu).cpu().numpy()
    kind, ti, tj, tk, *_ = chol.lu_dag_describe(T) if lu else chol.dag_describe(T)
    prog = odag.program_lu(T) if lu else None
    ref = odag.bottom_levels(T, dict(enumerate(cost)), prog) if lu else odag.bottom_levels(T, dict(enumerate(cost)))
    assert len(bl) == len(ref)
    for i in range(len(bl)):
        assert bl[i] == ref[(int(kind[i]), int(ti[i]), int(tj[i]), int(tk[i]))]


@pytest.mark.parametrize("lu", [False, True])
@pytest.mark.parametrize("T,cost", [(32, [7, 30, 31, 60]), (64, [3_500, 9_000, 12_000, 20_000]),
                                    (130, [1, 1, 1, 1]), (64, [5, 0, 2, 0]), (17, [4, -3, 0, 2])])
def test_device_bottom_levels_match_host(chol, lu, T, cost):
    # larger graphs against the library's host recursion, which the oracle pins above; zero
    # and negative costs check that every maximum starts from 0 as the host's does
    dev = chol.dag_bottom_levels_device(T, cost, lu=lu).cpu().numpy()
    host = chol.lu_dag_bottom_levels(T, cost) if lu else chol.dag_bottom_levels(T, cost)
    assert np.array_equal(dev, host)


def test_device_bottom_levels_large_T(chol):
    # T = 400 (10.7 million Cholesky tasks: n = 51200 at tile 128), every step with more
    # tasks than the block has threads
    cost = [2_000, 5_000, 6_000, 11_000]
    dev = chol.dag_bottom_levels_device(400, cost).cpu().numpy()
    assert np.array_equal(dev, chol.dag_bottom_levels(400, cost))


def test_sched_device_matches_host(chol):
    import random
    rng = random.Random(3)
    for policy in ("heft", "dada"):
        for alpha in (0.0, 0.5, 1.0):
            for _ in range(5):
                W = rng.randint(1, 300)
                LR = [dict(tid=i * 7 + 1, p=rng.choice([200, 600, 600, 1200]), prio=rng.randint(0, 9000),
                           aff=rng.choice([-1, rng.randint(0, W - 1)]), score=rng.choice([0, 524288]))
                      for i in range(rng.randint(1, 127))]
                load = [rng.choice([0, rng.randint(0, 5000)]) for _ in range(W)]
                host = chol.sched_activate(policy, LR, load, alpha=alpha)
                dev = chol.sched_activate_device(policy, LR, load, alpha=alpha)
                assert host == dev
                for t in LR:
                    t["own"] = [rng.choice([-1, rng.randint(0, W - 1)]) for _ in range(3)]
                    t["nin"] = 3
                    t["comm"] = rng.choice([5, 50, 500])
                host = chol.sched_activate(policy, LR, load, alpha=alpha, use_cp=True)
                dev = chol.sched_activate_device(policy, LR, load, alpha=alpha, use_cp=True)
                assert host == dev


def test_posv_host(chol):
    n, nrhs = 600, 3
    A = np.asfortranarray(synth.gram_spd(n, seed=13).numpy())
    B = np.asfortranarray(synth.rhs(n, nrhs, seed=14).numpy())
    A0, B0 = A.copy(), B.copy()
    info = chol.posv_host(A, B, chol.opts(nb=128))
    assert info == 0
    assert oracle.backward_error(A0, B, B0) <= BERR
    assert oracle.rel_frobenius(np.tril(A), oracle.factor(A0)) <= REL_L
    np.testing.assert_array_equal(np.triu(A, 1), np.triu(A0, 1))


def test_zero_size_and_bad_args(chol):
    A = torch.zeros(0, 0, dtype=torch.float64, device="cuda")
    info, _ = chol.factor(A)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    B = torch.zeros(8, 8, dtype=torch.float64, device="cuda")  # row-major: rejected
    with pytest.raises(ValueError):
        chol.factor(B)
    with pytest.raises(chol.CholeskyError):
        chol.factor(chol.colmajor(torch.eye(64, dtype=torch.float64, device="cuda")), chol.opts(nb=8))
