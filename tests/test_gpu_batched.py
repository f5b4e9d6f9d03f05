"""GPU checks of the batched factor + solve (FP64 and FP32) against the oracle, including a
CUDA-graph replay and the autotuner."""
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


def _make(chol, orders, dtype=torch.float64, seed=0):
    flat, offs = synth.gram_spd_batch(orders, seed=seed, device="cuda", dtype=dtype)
    roffs, off = [], 0
    for n in orders:
        roffs.append(off)
        off += n
    g = torch.Generator(device="cuda").manual_seed(seed + 1)
    rhs = torch.randn(max(off, 1), generator=g, device="cuda", dtype=torch.float64).to(dtype)
    return chol.Batch(flat, offs, orders, rhs, roffs)


def test_batched_fp64_parity(chol):
    rng = np.random.default_rng(0)
    orders = [int(x) for x in rng.integers(1, 200, size=300)] + [0, 1, 33, 64, 65, 257]
    bt = _make(chol, orders)
    A0 = [bt.matrix(m).cpu().numpy().copy() for m in range(bt.batch)]
    b0 = [bt.rhs(m).cpu().numpy().copy() for m in range(bt.batch)]
    chol.posv_batched(bt)
    torch.cuda.synchronize()
    assert int(bt.info.abs().max().item()) == 0
    for m in range(bt.batch):
        n = orders[m]
        if n == 0:
            continue
        L = np.tril(bt.matrix(m).cpu().numpy())
        assert oracle.rel_frobenius(L, oracle.factor(A0[m])) <= 1e-12, m
        x = bt.rhs(m).cpu().numpy()
        assert oracle.backward_error(A0[m], x, b0[m]) <= 1e-14, m


def test_batched_fp32_parity_and_integer_exact(chol):
    rng = np.random.default_rng(1)
    orders = [int(x) for x in rng.integers(2, 300, size=120)]
    bt = _make(chol, orders, dtype=torch.float32, seed=5)
    A0 = [bt.matrix(m).cpu().numpy().astype(np.float64) for m in range(bt.batch)]
    chol.posv_batched(bt)
    torch.cuda.synchronize()
    assert int(bt.info.abs().max().item()) == 0
    for m in range(bt.batch):
        L = np.tril(bt.matrix(m).cpu().numpy().astype(np.float64))
        assert oracle.rel_frobenius(L, oracle.factor(A0[m])) <= 2e-5, m
    # integer factors stay exact in FP32 (all intermediates are integers below 2^24)
    ints = [synth.integer_factor(n, seed=n) for n in (5, 40, 96, 130)]
    flat = torch.cat([torch.from_numpy(np.ascontiguousarray(A.T)).reshape(-1) for _, A in ints]).to("cuda", torch.float32)
    offs = np.cumsum([0] + [A.shape[0] ** 2 for _, A in ints])[:-1].tolist()
    bi = chol.Batch(flat, offs, [A.shape[0] for _, A in ints])
    chol.posv_batched(bi, factor_only=True)
    torch.cuda.synchronize()
    for m, (L, _) in enumerate(ints):
        np.testing.assert_array_equal(np.tril(bi.matrix(m).cpu().numpy().astype(np.float64)), L)


def test_batched_info_per_matrix(chol):
    orders = [50, 60, 70]
    bt = _make(chol, orders, seed=3)
    M = bt.matrix(1)
    M[20, 20] = -3.0  # matrix 1 is indefinite at order 21
    chol.posv_batched(bt)
    torch.cuda.synchronize()
    assert bt.info.tolist() == [0, 21, 0]


def test_batched_rejects_oversized_member(chol):
    orders = [10, 10]
    bt = _make(chol, orders, seed=4)
    bt.N[1] = 5000  # larger than the batched limit: reported, never touched
    bt.lda[1] = 5000
    chol.posv_batched(bt)
    torch.cuda.synchronize()
    assert bt.info.tolist() == [0, -3]


def test_batched_graph_replay_and_autotune(chol):
    rng = np.random.default_rng(2)
    orders = [int(x) for x in rng.integers(16, 257, size=200)]
    src = _make(chol, orders, seed=9)
    scratch = _make(chol, orders, seed=9)
    best, ms = chol.batched_autotune(src, scratch)
    assert best.workers_per_sm in (1, 2) and best.lpt_order in (0, 1) and ms > 0
    assert best.wide_panel_min_n in (0, 128, 256, 384, 4097)
    work = _make(chol, orders, seed=9)
    flat0, rhs0 = work.flat.clone(), work.rhs_flat.clone()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        chol.posv_batched(work, best, stream=stream)  # warm-up outside the capture
    torch.cuda.synchronize()
    ref_flat, ref_rhs = work.flat.clone(), work.rhs_flat.clone()
    g = torch.cuda.CUDAGraph()
    work.flat.copy_(flat0)
    work.rhs_flat.copy_(rhs0)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=stream):
        chol.posv_batched(work, best, stream=stream)
    for _ in range(2):
        work.flat.copy_(flat0)
        work.rhs_flat.copy_(rhs0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(work.flat, ref_flat) and torch.equal(work.rhs_flat, ref_rhs)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_factor_then_solve_batched_equals_posv(chol, dtype):
    # chol_factor_batched followed by chol_solve_batched runs the same bodies in the same
    # order as chol_posv_batched: bitwise the same factors and solutions
    rng = np.random.default_rng(7)
    orders = [int(x) for x in rng.integers(1, 260, size=90)] + [0, 32, 33]
    one = _make(chol, orders, dtype=dtype, seed=9)
    two = _make(chol, orders, dtype=dtype, seed=9)
    A0 = [one.matrix(m).cpu().numpy().astype(np.float64) for m in range(one.batch)]
    b0 = [one.rhs(m).cpu().numpy().astype(np.float64) for m in range(one.batch)]
    chol.posv_batched(one)
    chol.factor_batched(two)
    torch.cuda.synchronize()
    assert int(two.info.abs().max().item()) == 0
    chol.solve_batched(two)
    torch.cuda.synchronize()
    assert int(two.info.abs().max().item()) == 0
    assert torch.equal(one.flat, two.flat)
    assert torch.equal(one.rhs_flat, two.rhs_flat)
    tol = 1e-14 if dtype == torch.float64 else 1e-6
    for m in range(0, one.batch, 7):
        if orders[m] == 0:
            continue
        assert oracle.backward_error(A0[m], two.rhs(m).cpu().numpy().astype(np.float64), b0[m]) <= tol, m


@pytest.mark.parametrize("wide", [0, 100, 4097])
def test_batched_fp64_wide_panels(chol, wide):
    # members of order >= wide update their trailing matrix once per 64-column panel: parity
    # with the oracle, and integer factors stay exact (every partial sum is an integer)
    rng = np.random.default_rng(3)
    orders = [int(x) for x in rng.integers(1, 300, size=80)] + [64, 65, 127, 128, 129]
    bt = _make(chol, orders, seed=13)
    A0 = [bt.matrix(m).cpu().numpy().copy() for m in range(bt.batch)]
    b0 = [bt.rhs(m).cpu().numpy().copy() for m in range(bt.batch)]
    o = chol.BatchOpts()
    chol.lib.chol_batch_opts_default(chol.ctypes.byref(o))
    o.wide_panel_min_n = wide
    chol.posv_batched(bt, o)
    torch.cuda.synchronize()
    assert int(bt.info.abs().max().item()) == 0
    for m in range(bt.batch):
        L = np.tril(bt.matrix(m).cpu().numpy())
        assert oracle.rel_frobenius(L, oracle.factor(A0[m])) <= 1e-12, m
        assert oracle.backward_error(A0[m], bt.rhs(m).cpu().numpy(), b0[m]) <= 1e-14, m
    ints = [synth.integer_factor(n, seed=n) for n in (5, 64, 96, 130, 200)]
    flat = torch.cat([torch.from_numpy(np.ascontiguousarray(A.T)).reshape(-1) for _, A in ints]).to("cuda")
    offs = np.cumsum([0] + [A.shape[0] ** 2 for _, A in ints])[:-1].tolist()
    bi = chol.Batch(flat, offs, [A.shape[0] for _, A in ints])
    chol.posv_batched(bi, o, factor_only=True)
    torch.cuda.synchronize()
    for m, (L, _) in enumerate(ints):
        np.testing.assert_array_equal(np.tril(bi.matrix(m).cpu().numpy()), L)
