"""Pins of the DAG and scheduling oracles (CPU only)."""
import pytest

from oracle import dag, sched


def test_task_counts():
    # POTRF: T, TRSM and SYRK: T(T-1)/2 each, GEMM: T(T-1)(T-2)/6
    for T, expect in [(1, 1), (2, 4), (3, 10), (8, 120)]:
        tasks, _, _ = dag.build(T)
        assert len(tasks) == expect
        assert len(set(tasks)) == expect


def test_dependencies_by_hand_T3():
    _, preds, _ = dag.build(3)
    P, Tr, S, G = dag.POTRF, dag.TRSM, dag.SYRK, dag.GEMM
    assert preds[(P, 0, 0, 0)] == set()
    assert preds[(Tr, 2, 0, 0)] == {(P, 0, 0, 0)}
    assert preds[(S, 1, 1, 0)] == {(Tr, 1, 0, 0)}
    assert preds[(G, 2, 1, 0)] == {(Tr, 2, 0, 0), (Tr, 1, 0, 0)}
    assert preds[(P, 1, 1, 1)] == {(S, 1, 1, 0)}
    assert preds[(Tr, 2, 1, 1)] == {(P, 1, 1, 1), (G, 2, 1, 0)}
    assert preds[(S, 2, 2, 1)] == {(Tr, 2, 1, 1), (S, 2, 2, 0)}
    assert preds[(P, 2, 2, 2)] == {(S, 2, 2, 1)}


def test_bottom_levels_by_hand_T3():
    # costs POTRF 1, TRSM 3, SYRK 3, GEMM 6; longest paths worked out on paper
    bl = dag.bottom_levels(3, {0: 1, 1: 3, 2: 3, 3: 6})
    assert bl[(0, 2, 2, 2)] == 1
    assert bl[(2, 2, 2, 1)] == 4
    assert bl[(1, 2, 1, 1)] == 7
    assert bl[(0, 1, 1, 1)] == 8
    assert bl[(3, 2, 1, 0)] == 13
    assert bl[(2, 1, 1, 0)] == 11
    assert bl[(2, 2, 2, 0)] == 7
    assert bl[(1, 2, 0, 0)] == 16
    assert bl[(1, 1, 0, 0)] == 16
    assert bl[(0, 0, 0, 0)] == 17


def _task(tid, p, prio=0, aff=-1, score=0):
    return dict(tid=tid, p=p, prio=prio, aff=aff, score=score)


def test_heft_picks_earliest_finish_worker():
    load = [50, 10, 30]
    out = sched.heft([_task(0, 20, prio=5), _task(1, 20, prio=9)], load)
    # higher priority first: task 1 -> worker 1 (10+20); then task 0: loads [50, 30, 30] -> worker 1
    assert out == [(1, 1), (0, 1)]


def test_heft_tie_goes_to_lowest_worker():
    assert sched.heft([_task(3, 5)], [0, 0, 0]) == [(3, 0)]


def test_dada_alpha_zero_ignores_affinity():
    load = [0, 0, 0, 0]
    LR = [_task(i, 10, prio=10 - i, aff=3, score=100) for i in range(4)]
    out0, _ = sched.dada(LR, load, alpha=0.0)
    # with alpha = 0 the affinity phase places nothing; LPT/EFT spreads the four tasks
    assert sorted(w for _, w in out0) == [0, 1, 2, 3]
    out1, _ = sched.dada(LR, load, alpha=1.0)
    assert any(w == 3 for _, w in out1)


def test_dada_schedule_fits_bound():
    import random
    rng = random.Random(4)
    for _ in range(200):
        W = rng.randint(1, 8)
        load = [rng.randint(0, 100) for _ in range(W)]
        LR = [_task(i, rng.randint(1, 60), prio=rng.randint(0, 50), aff=rng.randint(-1, W - 1),
                    score=rng.choice([0, 64, 128])) for i in range(rng.randint(1, 12))]
        for alpha in (0.0, 0.5, 1.0):
            out, it = sched.dada(LR, load, alpha)
            assert len(out) == len(LR) and it <= 16
            fin = list(load)
            for tid, w in out:
                fin[w] += LR[tid]["p"]
            # the kept schedule fits (2 + alpha) * upper at worst
            upper = sum(t["p"] for t in LR) + max(load)
            assert max(fin) <= (2 + alpha) * upper
