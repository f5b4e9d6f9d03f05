"""Discrete-event simulation of the data-flow execution on W identical workers.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2 describes the execution: a worker takes a task from its own ready queue (or, idle,
steals one from another worker's queue), runs it, and on completion activates its successors;
those whose predecessors have all completed are placed on workers' queues by the policy's
activate (Section 2.2; Algorithms 1 and 2 decide the placement). The predicted completion
time-stamp of a worker (Section 2.3) is the remaining time of its running task plus the
processing times queued on it; the activate receives it as the worker's load.

This module runs that loop in simulated time with a fixed processing time per task, so that
whole schedules can be checked on the CPU: every task runs exactly once, never before its
predecessors have finished, and the makespan obeys the bounds of list scheduling. The
placement is a callable, so the same loop can drive the oracle's Algorithms 1 and 2 or the
library's host placement code.

A queue is served highest priority first (ties: lower task id); an idle worker with an empty
queue steals from the first non-empty queue in worker order (a deterministic stand-in for a
random victim) when stealing is on.
"""
import heapq


def simulate(ntasks, preds, succs, cost, prio, rw_tile, W, place, steal=True):
    """Run the data-flow loop.

    ntasks       tasks are 0 .. ntasks-1
    preds/succs  lists of predecessor / successor ids per task
    cost         processing time per task (int)
    prio         priority per task (bottom level)
    rw_tile      the tile each task writes (its affinity key)
    place        place(LR, load) -> [(tid, worker)], LR a list of dicts with tid, p, prio,
                 aff, score; load[w] the predicted remaining work of worker w
    Returns (makespan, start, end, worker) with per-task lists; raises on a deadlock.
    """
    remaining = [len(p) for p in preds]
    queues = [[] for _ in range(W)]  # heaps of (-prio, tid)
    qcost = [0] * W
    running = [None] * W  # (tid, end)
    owner = {}
    start = [None] * ntasks
    end = [None] * ntasks
    worker = [None] * ntasks
    events = []  # (end time, worker)
    now = 0

    def activate(ready):
        if not ready:
            return
        LR = []
        for t in ready:
            a = owner.get(rw_tile[t], -1)
            LR.append(dict(tid=t, p=cost[t], prio=prio[t], aff=a, score=1 if a >= 0 else 0))
        load = [max(0, running[w][1] - now) + qcost[w] if running[w] else qcost[w] for w in range(W)]
        for t, w in place(LR, load):
            heapq.heappush(queues[w], (-prio[t], t))
            qcost[w] += cost[t]

    def take(w):
        q = queues[w]
        if not q and steal:
            q = next((queues[v] for v in range(W) if queues[v]), None)
            if q is None:
                return None
        if not q:
            return None
        _, t = heapq.heappop(q)
        for v in range(W):
            if queues[v] is q:
                qcost[v] -= cost[t]
        return t

    activate([t for t in range(ntasks) if remaining[t] == 0])
    done = 0
    while done < ntasks:
        for w in range(W):
            if running[w] is None:
                t = take(w)
                if t is None:
                    continue
                if start[t] is not None:
                    raise AssertionError("task %d started twice" % t)
                start[t], worker[t] = now, w
                running[w] = (t, now + cost[t])
                heapq.heappush(events, (now + cost[t], w))
        if not events:
            raise AssertionError("deadlock: %d of %d tasks done, nothing running" % (done, ntasks))
        now, w = heapq.heappop(events)
        t = running[w][0]
        running[w] = None
        end[t] = now
        done += 1
        owner[rw_tile[t]] = w
        ready = []
        for s in succs[t]:
            remaining[s] -= 1
            if remaining[s] == 0:
                ready.append(s)
        activate(ready)
    return now, start, end, worker
