"""CPU checks of the C ABI library: it loads, exports every declared symbol, and its
host-side graph and placement code (the code the persistent kernel runs) matches the
oracles derived from the paper's data-flow rule (Section 2) and Algorithms 1 and 2."""
import ctypes
import os
import random
import re

import numpy as np
import pytest

import oracle.dag as odag
import oracle.sched as osched

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "chol.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(chol_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    import paper_1402_6601_gb300 as chol
    names = _declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(chol.build.LIB)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_opts_struct_layout_matches_header():
    import paper_1402_6601_gb300 as chol
    o = chol.ChOpts()
    chol.lib.chol_opts_default(ctypes.byref(o))
    assert o.nb == 0 and o.policy == 0 and o.alpha == 0.5 and o.steal == 1
    assert o.dada_max_iter == 16 and abs(o.dada_eps - 0.01) < 1e-15
    assert o.timeout_ns == 10_000_000_000 and o.trace == 0
    assert ctypes.sizeof(chol.ChOpts) == chol.lib.chol_opts_size() == 128
    assert o.hold_task == -1 and o.use_cp == 0 and o.cp_gbs == 40.0 and o.split == 1 and o.keep_next == 1


@pytest.mark.parametrize("T", [1, 2, 3, 5, 8, 11])
def test_dag_matches_dataflow_oracle(T):
    import paper_1402_6601_gb300 as chol
    kind, ti, tj, tk, indeg, ptr, succ = chol.dag_describe(T)
    tasks, preds, succs = odag.build(T)
    assert len(kind) == len(tasks)
    lib_tasks = [(int(kind[i]), int(ti[i]), int(tj[i]), int(tk[i])) for i in range(len(kind))]
    assert sorted(lib_tasks) == sorted(tasks)
    index = {t: i for i, t in enumerate(lib_tasks)}
    for i, t in enumerate(lib_tasks):
        assert indeg[i] == len(preds[t]), t
        got = {lib_tasks[int(s)] for s in succ[ptr[i]:ptr[i + 1]]}
        assert got == succs[t], t
    assert int(chol.lib.chol_dag_edge_count(T)) == sum(len(s) for s in succs.values())
    assert index[(0, 0, 0, 0)] == 0


@pytest.mark.parametrize("T,count", [(8, 120), (64, 45760), (128, 357760)])
def test_task_counts(T, count):
    import paper_1402_6601_gb300 as chol
    assert chol.lib.chol_dag_task_count(T) == count


@pytest.mark.parametrize("T", [1, 3, 6, 9])
def test_bottom_levels_match_oracle(T):
    import paper_1402_6601_gb300 as chol
    cost = [7, 30, 31, 60]
    bl = chol.dag_bottom_levels(T, cost)
    kind, ti, tj, tk, *_ = chol.dag_describe(T)
    ref = odag.bottom_levels(T, dict(enumerate(cost)))
    for i in range(len(bl)):
        assert bl[i] == ref[(int(kind[i]), int(ti[i]), int(tj[i]), int(tk[i]))]


@pytest.mark.parametrize("T", [1, 2, 3, 4, 7, 10])
def test_lu_dag_matches_dataflow_oracle(T):
    # the tile LU graph (GETRF/GESSM/TSTRF/SSSSM) the persistent kernel runs, against the
    # graph derived from the kernels' access modes
    import paper_1402_6601_gb300 as chol
    kind, ti, tj, tk, indeg, ptr, succ = chol.lu_dag_describe(T)
    tasks, preds, succs = odag.build(T, odag.program_lu(T))
    lib_tasks = [(int(kind[i]), int(ti[i]), int(tj[i]), int(tk[i])) for i in range(len(kind))]
    assert sorted(lib_tasks) == sorted(tasks) and len(set(lib_tasks)) == len(tasks)
    for i, t in enumerate(lib_tasks):
        assert indeg[i] == len(preds[t]), t
        got = {lib_tasks[int(s)] for s in succ[ptr[i]:ptr[i + 1]]}
        assert got == succs[t], t
        assert all(int(s) > i for s in succ[ptr[i]:ptr[i + 1]])  # ids are a topological order


def test_device_bottom_levels_reject_invalid_args():
    # argument checks come before any CUDA call, so they run without a GPU
    import paper_1402_6601_gb300 as chol
    cost = np.array([1, 2, 3, 4], np.int64)
    fake = ctypes.c_void_p(256)  # never dereferenced: every call below fails its checks first
    for lu in (0, 1):
        assert chol.lib.chol_dag_bottom_levels_device(lu, 0, cost.ctypes.data, fake, None) == -1
        assert chol.lib.chol_dag_bottom_levels_device(lu, 1025, cost.ctypes.data, fake, None) == -1
        assert chol.lib.chol_dag_bottom_levels_device(lu, 4, None, fake, None) == -1
        assert chol.lib.chol_dag_bottom_levels_device(lu, 4, cost.ctypes.data, None, None) == -1


@pytest.mark.parametrize("T", [1, 3, 6])
def test_lu_bottom_levels_match_oracle(T):
    import paper_1402_6601_gb300 as chol
    cost = [11, 30, 29, 60]
    bl = chol.lu_dag_bottom_levels(T, cost)
    kind, ti, tj, tk, *_ = chol.lu_dag_describe(T)
    ref = odag.bottom_levels(T, dict(enumerate(cost)), odag.program_lu(T))
    for i in range(len(bl)):
        assert bl[i] == ref[(int(kind[i]), int(ti[i]), int(tj[i]), int(tk[i]))]


def _random_ready(rng, m, W):
    return [dict(tid=rng.randint(0, 10**6) * 64 + i, p=rng.choice([100, 300, 300, 600, rng.randint(1, 900)]),
                 prio=rng.randint(0, 5000), aff=rng.choice([-1] + list(range(W))),
                 score=rng.choice([0, 131072, 524288])) for i in range(m)]


@pytest.mark.parametrize("seed", range(6))
def test_heft_host_matches_algorithm_1(seed):
    import paper_1402_6601_gb300 as chol
    rng = random.Random(seed)
    for _ in range(40):
        W = rng.randint(1, 40)
        LR = _random_ready(rng, rng.randint(1, 30), W)
        load = [rng.randint(0, 3000) for _ in range(W)]
        got, it = chol.sched_activate("heft", LR, load)
        assert got == osched.heft(LR, load) and it == 0


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0])
def test_dada_host_matches_algorithm_2(seed, alpha):
    import paper_1402_6601_gb300 as chol
    rng = random.Random(100 + seed)
    for _ in range(40):
        W = rng.randint(1, 40)
        LR = _random_ready(rng, rng.randint(1, 30), W)
        load = [rng.choice([0, rng.randint(0, 3000)]) for _ in range(W)]
        got, it = chol.sched_activate("dada", LR, load, alpha=alpha)
        ref, rit = osched.dada(LR, load, alpha)
        assert got == ref and it == rit


def test_sched_rejects_bad_arguments():
    import paper_1402_6601_gb300 as chol
    with pytest.raises(chol.CholeskyError):
        chol.sched_activate("dada", [dict(tid=0, p=1, prio=0, aff=-1, score=0)], [0], alpha=1.5)
    with pytest.raises(chol.CholeskyError):
        chol.sched_activate("steal", [dict(tid=0, p=1, prio=0, aff=-1, score=0)], [0])


def test_workspace_sizes_are_positive_and_monotone():
    import paper_1402_6601_gb300 as chol
    o = chol.opts(nb=128)
    a = chol.workspace_size(1024, o)
    b = chol.workspace_size(4096, o)
    assert 0 < a < b
    assert chol.workspace_size(1024, chol.opts(nb=8)) == 0  # nb below 16 is rejected
    assert chol.solve_workspace_size(1024, 1) > 0


def _random_ready_cp(rng, m, W):
    out = []
    for t in _random_ready(rng, m, W):
        nin = rng.randint(1, 3)
        t["own"] = [rng.choice([-1] + list(range(W))) for _ in range(nin)] + [-1] * (3 - nin)
        t["nin"] = nin
        t["comm"] = rng.choice([0, 10, 40, 400])
        out.append(t)
    return out


@pytest.mark.parametrize("seed", range(4))
def test_heft_cp_host_matches_oracle(seed):
    import paper_1402_6601_gb300 as chol
    rng = random.Random(500 + seed)
    for _ in range(40):
        W = rng.randint(1, 24)
        LR = _random_ready_cp(rng, rng.randint(1, 20), W)
        load = [rng.randint(0, 3000) for _ in range(W)]
        got, _ = chol.sched_activate("heft", LR, load, use_cp=True)
        assert got == osched.heft_cp(LR, load)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0])
def test_dada_cp_host_matches_oracle(seed, alpha):
    import paper_1402_6601_gb300 as chol
    rng = random.Random(900 + seed)
    for _ in range(40):
        W = rng.randint(1, 24)
        LR = _random_ready_cp(rng, rng.randint(1, 20), W)
        load = [rng.choice([0, rng.randint(0, 3000)]) for _ in range(W)]
        got, it = chol.sched_activate("dada", LR, load, alpha=alpha, use_cp=True)
        ref, rit = osched.dada_cp(LR, load, alpha)
        assert got == ref and it == rit


def test_cp_with_zero_comm_equals_plain():
    import paper_1402_6601_gb300 as chol
    rng = random.Random(77)
    for _ in range(30):
        W = rng.randint(1, 16)
        LR = _random_ready_cp(rng, rng.randint(1, 12), W)
        for t in LR:
            t["comm"] = 0
        load = [rng.randint(0, 999) for _ in range(W)]
        assert chol.sched_activate("heft", LR, load, use_cp=True) == chol.sched_activate("heft", LR, load)
        assert chol.sched_activate("dada", LR, load, use_cp=True) == chol.sched_activate("dada", LR, load)


def test_automatic_tile_size():
    import paper_1402_6601_gb300 as chol
    # nb = 0 picks 128 up to n = 32768 and 256 above (the workspace size depends on the tile count)
    for n, nb in ((8192, 128), (32768, 128), (32769, 256), (40000, 256)):
        auto = chol.workspace_size(n, chol.opts(nb=0))
        assert auto == chol.workspace_size(n, chol.opts(nb=nb)), (n, nb)
        assert auto != chol.workspace_size(n, chol.opts(nb=64 if nb == 128 else 128)), n


@pytest.mark.parametrize("n,nb", [(8192, 128), (1000, 128), (300, 64), (1, 16), (0, 128)])
def test_lu_aux_sizes(n, nb):
    # pivots: T^2 nb ints; L11 blocks: T^2 x 32 x nb doubles (T = ceil(n / nb))
    import paper_1402_6601_gb300 as chol
    o = chol.opts(nb=nb)
    npiv, nlw = ctypes.c_longlong(-1), ctypes.c_longlong(-1)
    assert chol.lib.chol_lu_aux_size(n, ctypes.byref(o), ctypes.byref(npiv), ctypes.byref(nlw)) == 0
    T = -(-n // nb)
    assert npiv.value == T * T * nb and nlw.value == T * T * 32 * nb


def test_lu_options_checked_on_the_host():
    import paper_1402_6601_gb300 as chol
    n = ctypes.c_longlong(0)
    # the LU tile kernels take tiles up to 256
    assert chol.lib.chol_lu_aux_size(1000, ctypes.byref(chol.opts(nb=512)), ctypes.byref(n), None) == -1
    assert chol.lib.chol_lu_workspace_size(1000, ctypes.byref(chol.opts(nb=512))) == 0
    assert chol.lib.chol_lu_workspace_size(1000, ctypes.byref(chol.opts(nb=256))) > 0
    assert chol.lib.chol_lu_aux_size(-1, ctypes.byref(chol.opts(nb=64)), None, None) == -1


@pytest.mark.parametrize("T", [1, 2, 8, 64, 128])
def test_lu_task_counts_closed_form(T):
    import paper_1402_6601_gb300 as chol
    assert chol.lib.chol_lu_dag_task_count(T) == sum(1 + 2 * m + m * m for m in range(T))


@pytest.mark.parametrize("graph", ["chol", "lu"])
def test_chrome_trace_export(graph, tmp_path):
    # synthetic per-task records (worker, queue, start ns, end ns) in the trace's layout
    import json
    import paper_1402_6601_gb300 as chol
    T = 3
    kind, ti, tj, tk, *_ = chol.lu_dag_describe(T) if graph == "lu" else chol.dag_describe(T)
    nt = len(kind)
    rec = np.zeros((nt, 4), np.int64)
    for t in range(nt):
        rec[t] = (t % 2, (t + 1) % 2, 5000 + 2000 * t, 5000 + 2000 * t + 1500)
    rec[nt - 1] = (-1, -1, -1, -1)  # a task without a record is left out
    path = tmp_path / "trace.json"
    out = chol.chrome_trace(rec, T, graph=graph, path=str(path))
    assert json.loads(path.read_text()) == out
    ev = out["traceEvents"]
    assert len(ev) == nt - 1
    first = "GETRF(0,0,0)" if graph == "lu" else "POTRF(0,0,0)"
    assert ev[0]["name"] == first and ev[0]["ts"] == 0.0 and ev[0]["dur"] == 1.5 and ev[0]["tid"] == 0
    assert ev[1]["ts"] == 2.0 and ev[1]["tid"] == 1 and ev[1]["args"] == {"task": 1, "queue": 0}
    names = {e["name"].split("(")[0] for e in ev}
    assert names <= set(chol._KIND_NAMES[graph])


def test_lu_argument_errors_before_any_launch():
    # argument checks return before the library touches a device (they hold on a CPU-only host)
    import paper_1402_6601_gb300 as chol
    o = ctypes.byref(chol.opts(nb=128))
    big = ctypes.byref(chol.opts(nb=512))
    f, s = chol.lib.chol_lu_factor, chol.lib.chol_lu_solve
    assert f(-1, None, 1, None, None, o, None, 0, None, None) == -1            # negative order
    assert f(100, None, 100, None, None, o, None, 0, None, None) == -1         # no dInfo
    fake = ctypes.c_void_p(256)  # never dereferenced: rejected before any launch
    assert f(100, fake, 99, fake, fake, o, fake, 1 << 20, fake, None) == -1    # lda < n
    assert f(100, fake, 100, None, fake, o, fake, 1 << 20, fake, None) == -1   # no pivot array
    assert f(100, fake, 100, fake, fake, big, fake, 1 << 20, fake, None) == -1  # tile above 256
    assert s(-1, 1, None, 1, None, None, o, None, 1, None, 0, None, None) == -1
    assert s(100, 1, fake, 100, fake, fake, o, fake, 99, fake, 1 << 20, None, None) == -1   # ldb < n
    assert s(100, 1, fake, 100, fake, fake, big, fake, 100, fake, 1 << 20, None, None) == -1
    assert s(100, 0, None, 100, None, None, o, None, 100, None, 0, None, None) == 0        # nothing to solve
    assert s(100, 1, fake, 100, fake, fake, o, fake, 100, None, 0, None, None) == -3      # no workspace
    need = chol.lib.chol_lu_solve_workspace_size(100, 1, o)
    assert need > 0 and chol.lib.chol_lu_solve_workspace_size(100, 1, big) == 0
    assert s(100, 1, fake, 100, fake, fake, o, fake, 100, fake, need - 1, None, None) == -3  # too small


def test_batch_descriptor_host_logic():
    # the pointer / order / leading-dimension arrays a batched call passes, built on the host
    import torch
    import paper_1402_6601_gb300 as chol
    orders = [3, 0, 2]
    flat = torch.arange(13, dtype=torch.float64)
    offs = [0, 9, 9]
    rhs = torch.arange(5, dtype=torch.float64)
    b = chol.Batch(flat, offs, orders, rhs, [0, 3, 3])
    assert b.batch == 3 and b.N.tolist() == orders and b.lda.tolist() == [3, 1, 2]
    assert b.A.tolist() == [flat.data_ptr() + 8 * o for o in offs]
    assert b.B.tolist() == [rhs.data_ptr() + 8 * o for o in (0, 3, 3)]
    # member m is the column-major n x n block at its offset
    assert b.matrix(0)[1, 0].item() == 1.0 and b.matrix(0)[0, 1].item() == 3.0
    assert b.matrix(2).tolist() == [[9.0, 11.0], [10.0, 12.0]]
    assert b.rhs(2).tolist() == [3.0, 4.0] and b.info.tolist() == [0, 0, 0]
    assert b.work.numel() >= int(chol.lib.chol_batched_workspace_size(3))
