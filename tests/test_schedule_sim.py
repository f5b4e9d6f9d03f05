"""Whole schedules on the CPU: the data-flow loop simulated on W identical workers
(oracle/simulate.py) with the oracle's Algorithms 1 and 2, and with the library's host
placement code, on the Cholesky and the tile LU graphs.

Pins (each fixed by something other than the placement code):
  * every task runs exactly once and never before all its predecessors have finished (the
    data-flow rule of Section 2);
  * one worker: the makespan is the total work;
  * with stealing the schedule is a greedy list schedule, so Graham's bounds hold:
    max(critical path, total / W) <= makespan <= total / W + critical path;
  * the library's placement gives the same schedule as the oracle's.
"""
import pytest

from oracle import dag as odag
from oracle import sched as osched
from oracle import simulate as osim

COSTS = {"chol": {0: 7, 1: 20, 2: 19, 3: 40}, "lu": {0: 15, 1: 20, 2: 22, 3: 40}}


def _graph(kind, T):
    prog = odag.program(T) if kind == "chol" else odag.program_lu(T)
    tasks, preds, succs = odag.build(T, prog)
    idx = {t: i for i, t in enumerate(tasks)}
    P = [[idx[p] for p in preds[t]] for t in tasks]
    S = [[idx[s] for s in sorted(succs[t])] for t in tasks]
    cost = [COSTS[kind][t[0]] for t in tasks]
    bl = odag.bottom_levels(T, COSTS[kind], prog)
    prio = [bl[t] for t in tasks]
    rw = [(t[1], t[2]) for t in tasks]  # the tile each task writes, in both graphs
    return tasks, P, S, cost, prio, rw, bl[tasks[0]]


def _oracle_place(policy, alpha):
    if policy == "heft":
        return lambda LR, load: osched.heft(LR, load)
    return lambda LR, load: osched.dada(LR, load, alpha)[0]


def _run(kind, T, W, place, steal=True):
    tasks, P, S, cost, prio, rw, cp = _graph(kind, T)
    span, start, end, worker = osim.simulate(len(tasks), P, S, cost, prio, rw, W, place, steal=steal)
    return tasks, P, cost, cp, span, start, end, worker


POLICIES = [("heft", 0.5), ("dada", 0.0), ("dada", 0.5), ("dada", 1.0)]
GRAPHS = [("chol", 6), ("lu", 5)]


@pytest.mark.parametrize("kind,T", GRAPHS)
@pytest.mark.parametrize("policy,alpha", POLICIES)
@pytest.mark.parametrize("W", [1, 3, 8])
def test_every_task_once_after_its_predecessors(kind, T, policy, alpha, W):
    tasks, P, cost, cp, span, start, end, worker = _run(kind, T, W, _oracle_place(policy, alpha))
    assert all(s is not None for s in start)
    for t in range(len(tasks)):
        assert end[t] == start[t] + cost[t]
        assert all(start[t] >= end[p] for p in P[t]), tasks[t]
    # no worker runs two tasks at once
    for w in range(W):
        runs = sorted((start[t], end[t]) for t in range(len(tasks)) if worker[t] == w)
        assert all(a[1] <= b[0] for a, b in zip(runs, runs[1:]))


@pytest.mark.parametrize("kind,T", GRAPHS)
@pytest.mark.parametrize("policy,alpha", POLICIES)
def test_one_worker_makespan_is_total_work(kind, T, policy, alpha):
    _, _, cost, _, span, _, _, _ = _run(kind, T, 1, _oracle_place(policy, alpha))
    assert span == sum(cost)


@pytest.mark.parametrize("kind,T", GRAPHS + [("chol", 8), ("lu", 7)])
@pytest.mark.parametrize("policy,alpha", POLICIES)
@pytest.mark.parametrize("W", [2, 4, 16])
def test_makespan_within_list_scheduling_bounds(kind, T, policy, alpha, W):
    _, _, cost, cp, span, _, _, _ = _run(kind, T, W, _oracle_place(policy, alpha))
    total = sum(cost)
    assert span >= max(cp, total / W)
    assert span <= total / W + cp


@pytest.mark.parametrize("kind,T", GRAPHS)
@pytest.mark.parametrize("policy,alpha", POLICIES)
def test_library_placement_gives_the_oracle_schedule(kind, T, policy, alpha):
    import paper_1402_6601_gb300 as chol
    W = 4
    lib_place = lambda LR, load: chol.sched_activate(policy, LR, load, alpha=alpha)[0]  # noqa: E731
    ref = _run(kind, T, W, _oracle_place(policy, alpha))
    got = _run(kind, T, W, lib_place)
    assert got[4:] == ref[4:]


@pytest.mark.parametrize("kind,T", GRAPHS)
def test_owner_computes_without_stealing_completes(kind, T):
    # the static map (a task goes to the worker its tile maps to) never deadlocks either
    tasks, P, S, cost, prio, rw, cp = _graph(kind, T)
    W = 3
    place = lambda LR, load: [(t["tid"], (rw[t["tid"]][0] + rw[t["tid"]][1] * T) % W) for t in LR]  # noqa: E731
    span, start, end, worker = osim.simulate(len(tasks), P, S, cost, prio, rw, W, place, steal=False)
    assert all(worker[t] == (rw[t][0] + rw[t][1] * T) % W for t in range(len(tasks)))
    assert all(start[t] >= max([end[p] for p in P[t]], default=0) for t in range(len(tasks)))
