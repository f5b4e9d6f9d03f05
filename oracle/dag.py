"""Tile task graph of the right-looking lower Cholesky, derived from data access modes.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper runs the PLASMA tile algorithm for DPOTRF (Section 4.1, "Benchmarks") on a
data-flow runtime in which the dependencies between tasks follow from the data they read
and write (Section 2: synchronisations are detected implicitly; a completed task activates
its successors once they are ready). This module writes that rule out: it walks the
sequential tile program in its natural order and makes every task depend on the last
writer of each tile it touches (read-after-write, write-after-write) and, for a writer, on
the readers since that write (write-after-read).

Task kinds and tuples (kind, i, j, k):
  0 POTRF(k)      (0, k, k, k)  RW A_kk
  1 TRSM(i, k)    (1, i, k, k)  R A_kk,           RW A_ik
  2 SYRK(i, k)    (2, i, i, k)  R A_ik,           RW A_ii
  3 GEMM(i, j, k) (3, i, j, k)  R A_ik, R A_jk,   RW A_ij     (k < j < i)

The tile LU with incremental pivoting (DGETRF, the paper's second workload) has its own
program (program_lu). A diagonal tile is two regions there: its unit lower part L, written
by GETRF and read by GESSM, and its upper part U, which the TSTRF chain of the step updates;
a task that writes the whole tile writes both. The kernels' pivots and the L11 blocks of
TSTRF travel with the tile whose multipliers they describe.
  0 GETRF(k)        (0, k, k, k)  RW A_kk (L and U)
  1 GESSM(k, j)     (1, k, j, k)  R A_kk.L,             RW A_kj          (j > k)
  2 TSTRF(i, k)     (2, i, k, k)  RW A_kk.U, RW A_ik                     (i > k)
  3 SSSSM(i, j, k)  (3, i, j, k)  R A_ik,  RW A_kj, RW A_ij              (i, j > k)
"""
from functools import lru_cache

POTRF, TRSM, SYRK, GEMM = 0, 1, 2, 3


def program(T):
    """Tasks in sequential program order with (reads, writes) tile sets."""
    out = []
    for k in range(T):
        out.append(((POTRF, k, k, k), [], [(k, k)]))
        for i in range(k + 1, T):
            out.append(((TRSM, i, k, k), [(k, k)], [(i, k)]))
        for i in range(k + 1, T):
            out.append(((SYRK, i, i, k), [(i, k)], [(i, i)]))
            for j in range(k + 1, i):
                out.append(((GEMM, i, j, k), [(i, k), (j, k)], [(i, j)]))
    return out


GETRF, GESSM, TSTRF, SSSSM = 0, 1, 2, 3


def _whole(i, j):
    """The regions of tile (i, j): a diagonal tile has an L and a U part."""
    return [(i, j, "L"), (i, j, "U")] if i == j else [(i, j)]


def program_lu(T):
    """Tile LU with incremental pivoting in sequential program order, (reads, writes)."""
    out = []
    for k in range(T):
        out.append(((GETRF, k, k, k), [], _whole(k, k)))
        for j in range(k + 1, T):
            out.append(((GESSM, k, j, k), [(k, k, "L")], _whole(k, j)))
        for i in range(k + 1, T):
            out.append(((TSTRF, i, k, k), [], [(k, k, "U")] + _whole(i, k)))
            for j in range(k + 1, T):
                out.append(((SSSSM, i, j, k), _whole(i, k), _whole(k, j) + _whole(i, j)))
    return out


def build(T, prog=None):
    """Return (tasks, preds, succs): tasks in program order, dict task -> set of tasks.
    prog: a program as returned by program / program_lu (default: the Cholesky one)."""
    prog = program(T) if prog is None else prog
    last_writer = {}
    readers = {}
    preds = {}
    for task, reads, writes in prog:
        p = set()
        for tile in reads:
            if tile in last_writer:
                p.add(last_writer[tile])
        for tile in writes:
            if tile in last_writer:
                p.add(last_writer[tile])
            p.update(readers.get(tile, ()))
        p.discard(task)
        preds[task] = p
        for tile in reads:
            readers.setdefault(tile, set()).add(task)
        for tile in writes:
            last_writer[tile] = task
            readers[tile] = set()
    succs = {t: set() for t, _, _ in prog}
    for t, p in preds.items():
        for q in p:
            succs[q].add(t)
    return [t for t, _, _ in prog], preds, succs


def bottom_levels(T, cost, prog=None):
    """Longest cost-weighted path from each task to the exit, the task itself included.

    cost maps a task kind to its (integer) cost. bl(t) = cost(t) + max over successors.
    """
    tasks, _, succs = build(T, prog)

    @lru_cache(maxsize=None)
    def bl(t):
        c = cost[t[0]]
        best = 0
        for s in succs[t]:
            best = max(best, bl(s))
        return c + best

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 100000))
    try:
        # evaluate from the end of the program backwards so the recursion stays shallow
        for t in reversed(tasks):
            bl(t)
        return {t: bl(t) for t in tasks}
    finally:
        sys.setrecursionlimit(old)
