"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas). Each rank runs its own
factorization on its own GPU in the benchmark; the host logic that turns the ranks' timings
into the job's number -- the slowest rank's time and all ranks' work divided by it -- is
checked here with world_size 2 and no GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [1000.0, 1500.0][rank]  # rank 1 is the slow one
    ms, gflops = bench.job_throughput(ms_local, flops_per_rank=3.0e12)
    dist.barrier()
    out[rank] = (ms, gflops)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_job_throughput_uses_slowest_rank_and_all_work():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    assert out[0] == out[1]
    ms, gflops = out[0]
    assert ms == 1500.0
    assert abs(gflops - 2 * 3.0e12 / 1.5 / 1e9) < 1e-6


def test_single_process_is_its_own_job():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms, gflops = bench.job_throughput(250.0, flops_per_rank=1.0e12)
    assert ms == 250.0 and abs(gflops - 4000.0) < 1e-9
