"""Benchmark: FP64 tiled Cholesky factor + forward/backward solve on GB300.

One step = one pass of the whole hot path over one synthetic input: restore A from its
pristine copy (the factor works in place), chol_factor (init + persistent data-flow kernel),
chol_solve (forward and back substitution sweeps). Default workload: n = 32768, tile 256,
64 right-hand sides, HEFT ready-queue policy; A = sym(G G^T)/n + I with G ~ N(0, 1).

Metric: GFLOP/s with n^3/3 flops for the factor plus 2 n^2 nrhs for the two sweeps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--nb 256] [--policy heft] ...
  python bench.py --impl reference     # the oracle on the host cores (bounded sample)

Under torchrun (N > 1) every rank factors its own matrix on its own GPU (replicas: the
method has no exchange step on one GPU); the timed region is bracketed by barriers and the
maximum time over ranks is used; rank 0 prints the JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SMS = 152
FP64_FMA_PER_CLK_PER_SM = 2       # DFMA retires 2 FMA/clk/SM on sm_103 (shared-memory-fed probe: 1256.8 GFLOP/s)
SM_MAX_MHZ = 2070.0
FP64_PEAK_GFLOPS = SMS * FP64_FMA_PER_CLK_PER_SM * 2 * SM_MAX_MHZ / 1000.0  # 1258.6

# DRAM bytes (read + write) of one FP64 factor launch (tile 256, HEFT) from one-metric ncu
# captures of the current kernel at small sizes (profiles/factor_kernel_f64_dram_traffic_
# n8192_n12288_n16384.txt). They do not grow in proportion to the work (the L2 hit rate falls
# as the trailing matrix outgrows L2), so no full-size figure is scaled from them and the
# roofline's "traffic" stays None at the benchmark size.
FACTOR_TRAFFIC_SMALL_CASES = [
    {"n": 8192, "nb": 256, "bytes": 5.18e9, "l2_hit_pct": 88.3},
    {"n": 12288, "nb": 256, "bytes": 22.52e9, "l2_hit_pct": 84.1},
    {"n": 16384, "nb": 256, "bytes": 113.33e9, "l2_hit_pct": 58.4},
]

# two-sided 95 % quantiles of Student's t for 1..30 degrees of freedom
_T975 = [12.706, 4.303, 3.182, 2.776, 2.571, 2.447, 2.365, 2.306, 2.262, 2.228, 2.201, 2.179, 2.160, 2.145,
         2.131, 2.120, 2.110, 2.101, 2.093, 2.086, 2.080, 2.074, 2.069, 2.064, 2.060, 2.056, 2.052, 2.048,
         2.045, 2.042]


def mean_ci95(xs):
    """(mean, half width of the 95 % confidence interval of the mean, count), Student's t; the
    paper reports every point as a mean with its 95 % confidence interval (Section 4.1,
    "Methodology"). The half width is None for a single sample."""
    xs = [float(x) for x in xs]
    m = sum(xs) / len(xs)
    if len(xs) < 2:
        return m, None, len(xs)
    sd = statistics.stdev(xs)
    df = len(xs) - 1
    t = _T975[df - 1] if df <= len(_T975) else 1.96
    return m, t * sd / len(xs) ** 0.5, len(xs)


def stat(xs, digits=3):
    m, h, k = mean_ci95(xs)
    return {"mean": round(m, digits), "ci95": None if h is None else round(h, digits), "n": k}


PROBE_KINDS = (("dfma", 0), ("dfma_free_operands", 5), ("dfma_smem_tile", 6), ("mma_m8n8k4", 1),
               ("mma_m16n8k4", 2), ("mma_m16n8k8", 3), ("mma_m16n8k16", 4))


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=32768)
    p.add_argument("--nb", type=int, default=256)
    p.add_argument("--nrhs", type=int, default=64)
    p.add_argument("--policy", default="heft")
    p.add_argument("--alpha", type=float, default=0.5)
    p.add_argument("--workers-per-sm", type=int, default=2)
    p.add_argument("--cp", action="store_true", help="communication prediction in the placement")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-n", type=int, default=10240)
    p.add_argument("--cpu-one-thread-n", type=int, default=4096)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--no-mixed", action="store_true")
    p.add_argument("--mixed-n", type=int, default=16384)
    p.add_argument("--mixed-nrhs", type=int, default=16)
    p.add_argument("--mixed-steps", type=int, default=30)
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batch", type=int, default=10000)
    p.add_argument("--batched-steps", type=int, default=30)
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--adj-n", type=int, default=1024)
    p.add_argument("--adj-batch", type=int, default=64)
    p.add_argument("--adj-steps", type=int, default=10)
    p.add_argument("--adj-streams", type=int, default=16)
    p.add_argument("--adj-nb", type=int, default=64, help="tile size of the adjoint leg's factors")
    p.add_argument("--adj-workers", type=int, default=16, help="factor workers per matrix in the adjoint leg")
    p.add_argument("--no-probe", action="store_true", help="skip the FP64 throughput probe")
    p.add_argument("--fp64-probe-only", action="store_true",
                   help="run only the FP64 throughput probes (DFMA and the mma.sync .f64 shapes) and print them")
    p.add_argument("--mixed-fp64-steps", type=int, default=3)
    p.add_argument("--no-mixed-oracle", action="store_true",
                   help="skip the oracle's FP64 solution of the mixed-precision configuration (about a minute "
                        "on 16 host cores)")
    p.add_argument("--legs", default="main,mixed,batched,adjoint,lu",
                   help="comma-separated legs to run (main = the FP64 factor + solve line); without main "
                        "the other legs' results are printed alone, e.g. to profile one leg")
    p.add_argument("--bf16-pcg", action="store_true",
                   help="also measure plain BF16 as a preconditioner: conjugate gradients in FP64 preconditioned "
                        "by the shifted BF16 tensor-core factor, on the mixed-precision configuration")
    p.add_argument("--bf16-pcg-only", action="store_true", help="run only that measurement")
    p.add_argument("--pcg-maxit", type=int, default=3000)
    p.add_argument("--no-lu", action="store_true")
    p.add_argument("--lu-n", type=int, default=8192)
    p.add_argument("--lu-nb", type=int, default=0)
    p.add_argument("--lu-steps", type=int, default=10)
    p.add_argument("--lu-policy", default="heft")
    p.add_argument("--lu-sweep", action="store_true",
                   help="also time the LU leg under every ready-queue policy (HEFT, DADA(0/0.5/1), "
                        "DADA(0.5)+CP, stealing, static)")
    return p.parse_args()


def step_flops(n, nrhs):
    return n ** 3 / 3.0 + 2.0 * n * n * nrhs


def job_throughput(ms_local, flops_per_rank, device=None):
    """(ms, GFLOP/s) of the whole job: the slowest rank's time (max over ranks when a process
    group is up) and the work of all ranks divided by it (replicas: every rank runs the
    same workload)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    ms = float(ms_local)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, flops_per_rank * world / (ms / 1000.0) / 1e9


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows),
                   power_w_max=max([num(r[3]) for r in rows if num(r[3]) is not None] or [0.0]))
        return out


# ----------------------------------------------------------------------------- FP64 peak
def run_fp64_probe(chol, dev, target_ms=150.0, reps=5):
    """Throughput of the FP64 units on this GPU: DFMA chains (the instruction of the factor's
    tile bodies) and the FP64 warp MMA shapes, each launch sized to about target_ms, timed
    with CUDA events on the launching stream (best and mean of `reps` launches after a
    warm-up), with the SM clock sampled during the probe; `at_max_clock` scales the best rate
    by sm_max_mhz / median sm_mhz (time x clock is constant for a pipe-bound kernel)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    res = {}
    clocks.start()

    def once(kind, blocks, iters):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f = chol.probe_fp64(kind, blocks, 256, iters, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return f, e0.elapsed_time(e1)

    for name, kind in PROBE_KINDS:
        # 256-thread blocks, 1, 2 or 4 per SM (a whole number per SM; the MMA kernel's registers
        # allow two): the best of the grids is the unit's rate
        best = None
        for per_sm in ((1, 2, 4) if kind in (0, 5, 6) else (1, 2)):
            blocks = sms * per_sm
            iters = 2000
            _, t = once(kind, blocks, iters)
            iters = max(1, int(iters * target_ms / max(t, 1e-3)))
            once(kind, blocks, iters)
            runs = [once(kind, blocks, iters) for _ in range(reps)]
            f = runs[0][0]
            ms = [t for _, t in runs]
            v = {"gflops_best": round(f / min(ms) / 1e6, 1), "gflops": stat([f / t / 1e6 for t in ms], 1),
                 "ms": round(sum(ms) / len(ms), 2), "blocks": blocks, "threads": 256, "iters": iters,
                 "flops_per_launch": f}
            v["by_blocks_per_sm"] = dict(best["by_blocks_per_sm"]) if best else {}
            v["by_blocks_per_sm"][str(per_sm)] = v["gflops_best"]
            if best is None or v["gflops_best"] > best["gflops_best"]:
                best = v
            else:
                best["by_blocks_per_sm"] = v["by_blocks_per_sm"]
        res[name] = best
    clk = clocks.stop()
    med, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz") or SM_MAX_MHZ
    for v in res.values():
        v["at_max_clock"] = round(v["gflops_best"] * mx / med, 1) if med else None
    return {"kinds": res, "clocks": {"sm_mhz": med, "sm_max_mhz": mx, "reasons": clk.get("reasons"),
                                      "samples": clk.get("samples")},
            "derived_peak": round(FP64_PEAK_GFLOPS, 1),
            "method": "DFMA: every thread updates a 4 x 4 register tile (16 independent chains, the pattern "
                      "of the factor's tile bodies); mma.sync .f64: every warp keeps 8 independent "
                      "accumulator fragments; one launch of ~%d ms per repetition" % int(target_ms)}


# ----------------------------------------------------------------------------- oracle arm
def oracle_step(n, nrhs, seed):
    """One factor + solve by the oracle on host cores; returns (seconds, flops)."""
    import oracle
    import synth
    A = synth.gram_spd(n, seed=seed).numpy()
    B = synth.rhs(n, nrhs, seed=seed + 1).numpy()
    t0 = time.perf_counter()
    L = oracle.factor(A)
    oracle.solve(L, B)
    return time.perf_counter() - t0, step_flops(n, nrhs)


def oracle_one_thread(n, nrhs, seed, timeout_s=300):
    """The oracle's factor + solve with one OpenMP thread, in a child process (the thread
    count of the loaded oracle cannot change); None if it cannot be run."""
    code = ("import sys; sys.path.insert(0, %r); import bench; t, f = bench.oracle_step(%d, %d, %d); "
            "print('ONE_THREAD', t, f)" % (ROOT, n, nrhs, seed))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, OMP_NUM_THREADS="1"),
                           capture_output=True, text=True, timeout=timeout_s)
        line = [x for x in r.stdout.splitlines() if x.startswith("ONE_THREAD")][-1]
        _, t, f = line.split()
        return float(t), float(f)
    except Exception:
        return None


def cpu_baseline(args):
    import oracle
    t, f = oracle_step(args.cpu_sample_n, args.nrhs, args.seed)
    out = {"value": round(f / t / 1e9, 3), "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
           "seconds": round(t, 2),
           "sample": "oracle (plain C, FP64, unblocked) factor + solve of one n=%d Gram matrix with %d RHS, "
                     "same generator as the GPU workload" % (args.cpu_sample_n, args.nrhs)}
    one = oracle_one_thread(args.cpu_one_thread_n, args.nrhs, args.seed)
    if one is not None:
        out["one_thread"] = {"value": round(one[1] / one[0] / 1e9, 3), "unit": "GFLOP/s", "cores": 1,
                             "seconds": round(one[0], 2),
                             "sample": "the same with OMP_NUM_THREADS=1 on one n=%d matrix" % args.cpu_one_thread_n}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    for _ in range(args.warmup):
        oracle_step(args.cpu_sample_n, args.nrhs, args.seed)
    tt, ff = 0.0, 0.0
    for _ in range(args.steps):
        t, f = oracle_step(args.cpu_sample_n, args.nrhs, args.seed)
        tt += t
        ff += f
    v = ff / tt / 1e9
    line = {
        "metric": "Cholesky GFLOP/s (FP64 factor + solve)", "value": round(v, 3), "unit": "GFLOP/s",
        "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tt / args.steps * 1000, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": round(v, 3), "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "each step: oracle factor + solve of one n=%d Gram matrix with %d RHS (a bounded "
                                   "sample of the n=%d workload)" % (args.cpu_sample_n, args.nrhs, args.n)},
        "e2e": {"value": round(v, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": "FP64 tiled Cholesky factor + solve, n=%d, tile %d, %d RHS, %s ready queues%s; "
                        "A = sym(G G^T)/n + I, G ~ N(0,1)" % (
                            args.n, args.nb, args.nrhs, args.policy.upper(),
                            (" alpha=%g" % args.alpha if args.policy == "dada" else "") + (" +CP" if args.cp else "")),
            "n": args.n, "nb": args.nb, "nrhs": args.nrhs, "policy": args.policy, "alpha": args.alpha,
            "workers_per_sm": args.workers_per_sm, "communication_prediction": bool(args.cp),
            "l2": "inputs larger than L2 (A is %.1f GB)" % (args.n * args.n * 8 / 1e9),
            "parallelism": "replicas x%d" % args.gpus}


# ----------------------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    import synth
    import paper_1402_6601_gb300 as chol

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    if args.bf16_pcg_only:
        if rank == 0:
            print(json.dumps({"bf16_pcg": run_bf16_pcg(args, chol, dev)}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    if args.fp64_probe_only:
        if rank == 0:
            print(json.dumps({"fp64_probe": run_fp64_probe(chol, dev)}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    legs = set(x.strip() for x in args.legs.split(",") if x.strip())
    if "main" not in legs:
        if rank == 0:
            out = {}
            if "mixed" in legs:
                out["mixed_precision"] = run_mixed(args, chol, dev)
            if "batched" in legs:
                out["batched"] = run_batched(args, chol, dev)
            if "adjoint" in legs:
                out["adjoint"] = run_adjoint(args, chol, dev)
            if "lu" in legs:
                out["lu"] = run_lu(args, chol, dev)
            print(json.dumps({"legs": out}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    n, nb, nrhs = args.n, args.nb, args.nrhs
    o = chol.opts(nb=nb, policy=args.policy, alpha=args.alpha, workers_per_sm=args.workers_per_sm,
                  use_cp=args.cp)
    A0 = chol.colmajor(synth.gram_spd(n, seed=args.seed + rank, device=dev))
    B0 = chol.colmajor(synth.rhs(n, nrhs, seed=args.seed + 1000 + rank, device=dev))
    A = torch.empty_like(A0)
    B = torch.empty_like(B0)
    work = torch.empty(chol.workspace_size(n, o), dtype=torch.uint8, device=dev)
    swork = torch.empty(chol.solve_workspace_size(n, nrhs), dtype=torch.uint8, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    launches_per_step = 7  # init, bottom levels, persistent factor, info copy; 2 sweeps, info copy

    def step(ev=None, start=None):
        if start is not None:
            start.record(stream)
        A.copy_(A0)
        B.copy_(B0)
        if ev is not None:
            ev[0].record(stream)
        chol.factor(A, o, work=work, info=info, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        chol.solve(A, B, work=swork, info=info, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if int(info.item()) != 0:
        raise RuntimeError("factor info %d" % int(info.item()))

    clocks = ClockSampler(local)
    fac_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
    step_events = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e_start, e_end = step_events[0], step_events[-1]
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        step(fac_events[k], start=step_events[k])
    e_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e_start.elapsed_time(e_end)
    fac_ms = [a.elapsed_time(b) for a, b in fac_events]
    step_ms = [step_events[k].elapsed_time(step_events[k + 1]) for k in range(args.steps)]
    ms, value = job_throughput(ms, step_flops(n, nrhs) * args.steps, device=dev)

    # correctness of the timed result (cheap O(n^2 nrhs) check on the device)
    R = B0 - torch.mm(A0, B)
    berr = float((R.abs().amax(0) / (A0.abs().sum(1).amax() * B.abs().amax(0) + B0.abs().amax(0))).amax())

    fac_avg = sum(fac_ms) / len(fac_ms)
    achieved = n ** 3 / 3.0 / (fac_avg / 1000.0) / 1e9
    fac_stat = stat(fac_ms, 2)
    roofline = {"bound": "alu", "achieved": round(achieved, 1), "peak": round(FP64_PEAK_GFLOPS, 1),
                "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4),
                "traffic": None,
                "traffic_small_cases": FACTOR_TRAFFIC_SMALL_CASES,
                "kernel": "factor_kernel (persistent data-flow, DFMA tile bodies)",
                "launch_ms": fac_stat,
                "achieved_ci95": None if fac_stat["ci95"] is None else round(
                    achieved * fac_stat["ci95"] / fac_stat["mean"], 1),
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz (DFMA; FP64 mma.sync is "
                               "slower on sm_103, see fp64_probe)"}
    if not args.no_probe and rank == 0:
        roofline["fp64_probe"] = run_fp64_probe(chol, dev)

    e2e = None
    if not args.no_e2e and rank == 0:
        e2e = run_e2e(args, chol, A0, B0, o, dev)
    barrier()

    del A, B, work, R
    mixed = None
    if not args.no_mixed and "mixed" in legs and rank == 0:
        mixed = run_mixed(args, chol, dev)
    batched = None
    if not args.no_batched and "batched" in legs and rank == 0:
        batched = run_batched(args, chol, dev)
    adjoint = None
    if not args.no_adjoint and "adjoint" in legs and rank == 0:
        adjoint = run_adjoint(args, chol, dev)
    pcg = None
    if args.bf16_pcg and rank == 0:
        pcg = run_bf16_pcg(args, chol, dev)
    lu = None
    if not args.no_lu and "lu" in legs and rank == 0:
        lu = run_lu(args, chol, dev)
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        cpu = cpu_baseline(args)

    if rank == 0:
        line = {
            "metric": "Cholesky GFLOP/s (FP64 factor + solve)", "value": round(value, 2), "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "factor_ms": round(fac_avg, 2), "factor_ms_ci95": fac_stat["ci95"],
            "step_ms": stat(step_ms, 2), "solve_backward_error": berr,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "mixed_precision": mixed, "batched": batched,
            "adjoint": adjoint, "lu": lu, "bf16_pcg": pcg,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons"), "samples": clk.get("samples"),
                       "power_w_max": clk.get("power_w_max")},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _backward_error(A, X, B):
    R = B - A @ X
    return float((R.abs().amax(0) / (A.abs().sum(1).amax() * X.abs().amax(0) + B.abs().amax(0))).amax())


def run_mixed(args, chol, dev):
    """The mixed-precision configuration: A = Q diag(lambda) Q^T with kappa = 1e6 (32
    Householder reflectors), 16 RHS. FP64 factor + solve against a low-precision factor + FP64
    iterative refinement to the same backward error (1e-14), for each low-precision form
    (FP32 FFMA, three-term BF16 on tensor cores, plain BF16 on tensor cores); all timed with
    CUDA events over --mixed-steps steps after one warm-up step each. The FP64 baseline uses
    the library's automatic tile (its fastest at this order); the low-precision factors use
    256. The headline numbers are those of the fastest form that reaches the target."""
    import torch
    import synth
    n, nrhs = args.mixed_n, args.mixed_nrhs
    A = chol.colmajor(synth.householder_spd(n, seed=args.seed, cond=1e6, device=dev))
    B = chol.colmajor(synth.rhs(n, nrhs, seed=args.seed + 7, device=dev))
    o = chol.opts(nb=256)   # low-precision factors (the tensor-core update takes tiles of 256)
    o64 = chol.opts(nb=0)   # FP64 baseline: the library's automatic tile, its fastest at this n
    W = torch.empty_like(A)
    Bw = torch.empty_like(B)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    work = torch.empty(chol.workspace_size(n, o64), dtype=torch.uint8, device=dev)
    sw = torch.empty(chol.solve_workspace_size(n, nrhs), dtype=torch.uint8, device=dev)
    rwork = torch.empty(chol.refine_workspace_size(n, nrhs, o), dtype=torch.uint8, device=dev)
    X = chol.colmajor(torch.empty(n, nrhs, dtype=torch.float64, device=dev))
    stream = torch.cuda.current_stream(dev)

    def fp64_step():
        W.copy_(A)
        Bw.copy_(B)
        chol.factor(W, o64, work=work, info=info, stream=stream)
        chol.solve(W, Bw, work=sw, info=info, stream=stream)

    def mixed_step(prec, A_, B_):
        return chol.solve_refine(A_, B_, X=X, tol=1e-14, max_iter=30, o=o, work=rwork, stream=stream,
                                 precision=prec)

    def timed(fn, steps):
        fn()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        out = None
        for k in range(steps):
            ev[k].record(stream)
            out = fn()
        ev[steps].record(stream)
        torch.cuda.synchronize()
        ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
        return sum(ms) / len(ms), out, stat(ms, 3)

    t64, _, t64_stat = timed(fp64_step, args.mixed_fp64_steps)
    e64 = _backward_error(A, Bw, B)
    sols = {"fp64": Bw.clone()}
    low = {"f32": "FP32 (FFMA) tile bodies",
           "bf16x3": "FP32 storage, GEMM updates on tcgen05 with three BF16 operand terms (FP32-accurate), "
                     "SYRK updates in FFMA, diagonal scaling",
           "bf16": "FP32 storage, SYRK/GEMM on tcgen05 with one BF16 operand term, diagonal scaling"}
    variants = {}
    for prec in ("f32", "bf16x3", "bf16"):
        tmx, out, tstat = timed(lambda: mixed_step(prec, A, B), args.mixed_steps)
        _, minfo, iters, berr = out
        finfo = int(minfo.item())
        emx = _backward_error(A, X, B) if finfo == 0 else float("inf")
        reached = bool(finfo == 0 and emx <= 1e-14)
        if finfo == 0:
            sols[prec] = X.clone()
        v = {"low_precision": low[prec], "ms": round(tmx, 2), "ms_stat": tstat,
             "speedup": round(t64 / tmx, 2) if reached else None,  # only at the same backward error
             "iterations": int(iters.item()), "info": finfo,
             "backward_error": emx, "reported_backward_error": float(berr.item()),
             "reached_target": reached}
        if finfo == 0:
            v["x_rel_diff_vs_fp64"] = float(torch.linalg.norm(X - Bw) / torch.linalg.norm(Bw))
        else:
            v["note"] = ("the factor breaks down (info = %d: a pivot is not positive in this precision); "
                         "kappa(A) u_bf16 >> 1" % finfo)
        variants[prec] = v
    # plain BF16 on a well-conditioned matrix of the same order (A = sym(G G^T)/n + I), for context
    Ag = chol.colmajor(synth.gram_spd(n, seed=args.seed + 3, device=dev))
    tg, out, _ = timed(lambda: mixed_step("bf16", Ag, B), 3)
    _, ginfo, giters, gberr = out
    variants["bf16_well_conditioned"] = {
        "workload": "n=%d, %d RHS, A = sym(G G^T)/n + I (kappa <= 5)" % (n, nrhs), "ms": round(tg, 2),
        "iterations": int(giters.item()), "info": int(ginfo.item()),
        "backward_error": _backward_error(Ag, X, B) if int(ginfo.item()) == 0 else float("inf")}
    # error against the oracle's FP64 solution (plain C Cholesky + substitutions on the host
    # cores, same bytes of A and B), for every result: max over columns of
    # ||x - x_oracle||_inf / ||x_oracle||_inf
    oracle_err = None
    if not args.no_mixed_oracle:
        import numpy as np
        import oracle
        Ah = A.cpu().numpy()
        Bh = B.cpu().numpy()
        t0 = time.perf_counter()
        Xo = oracle.solve(oracle.factor(Ah), Bh)
        t_or = time.perf_counter() - t0

        def rel(Xd):
            Xh = Xd.cpu().numpy()
            return float((np.abs(Xh - Xo).max(axis=0) / np.abs(Xo).max(axis=0)).max())

        oracle_err = {"oracle_seconds": round(t_or, 1), "oracle_cores": oracle.num_threads(),
                      "oracle_backward_error": oracle.backward_error(Ah, Xo, Bh),
                      "kappa_2": 1e6,
                      "x_rel_err_vs_oracle": {k: rel(v) for k, v in sols.items()}}
        for k, v in sols.items():
            if k in variants:
                variants[k]["x_rel_err_vs_oracle"] = oracle_err["x_rel_err_vs_oracle"][k]
    ok = [p for p in ("f32", "bf16x3") if variants[p]["reached_target"]]
    best = min(ok, key=lambda p: variants[p]["ms"]) if ok else "f32"
    b = variants[best]
    return {"workload": "n=%d, %d RHS, A = Q diag(lambda) Q^T, lambda geometric 1..1e6 (32 Householder "
                        "reflectors), tile 256, HEFT" % (n, nrhs),
            "fp64_ms": round(t64, 2), "fp64_ms_stat": t64_stat, "fp64_tile": 128 if n <= 32768 else 256,
            "oracle": oracle_err,
            "mixed_ms": b["ms"], "speedup": b["speedup"], "best": best,
            "low_precision": b["low_precision"] + "; FP64 residual and update",
            "target_backward_error": 1e-14, "fp64_backward_error": e64, "mixed_backward_error": b["backward_error"],
            "mixed_reported_backward_error": b["reported_backward_error"], "iterations": b["iterations"],
            "info": b["info"], "x_rel_diff_vs_fp64": b.get("x_rel_diff_vs_fp64"), "variants": variants}


def run_bf16_pcg(args, chol, dev):
    """Plain BF16 at kappa = 1e6 as a preconditioner instead of a factor for classical
    refinement (where it breaks down): the scaled matrix D^-1/2 A D^-1/2 + sigma I, sigma the
    smallest of 2^-12, 2^-11, ... for which the BF16 tensor-core factor exists, preconditions
    conjugate gradients run in FP64 on A (one block of --mixed-nrhs independent solves; the
    preconditioner applies the library's FP32 substitution to the scaled residual). Stops when
    every column's backward error (recomputed from the true residual every 10 iterations) is
    <= 1e-14, or after --pcg-maxit iterations. The FP64 products A p are torch matrix products
    here (this leg measures an alternative algorithm, not the library's path); the library's
    own symmetric FP64 product of the same shape is the refinement's residual kernel, so the
    cost of one iteration on the library's kernels is about one refinement step."""
    import torch
    import synth
    n, nrhs = args.mixed_n, args.mixed_nrhs
    A = chol.colmajor(synth.householder_spd(n, seed=args.seed, cond=1e6, device=dev))
    B = chol.colmajor(synth.rhs(n, nrhs, seed=args.seed + 7, device=dev))
    d = torch.diagonal(A).rsqrt()                          # D^-1/2
    S = (A * d[:, None] * d[None, :])
    o = chol.opts(nb=256)
    work = torch.empty(chol.lowp_workspace_size(n, o, precision="bf16"), dtype=torch.uint8, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    sigma, L = None, None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for e in range(12, 0, -1):
        s = 2.0 ** -e
        L = chol.colmajor(S.to(torch.float32))
        L.diagonal().add_(s)  # the shift (diag(S) = 1, exact in FP32)
        e0.record()
        chol.factor_f32(L, o, work=work, info=info, precision="bf16")
        e1.record()
        torch.cuda.synchronize()
        if int(info.item()) == 0:
            sigma = s
            break
    factor_ms = e0.elapsed_time(e1)
    del S
    swork = torch.empty(chol.solve_workspace_size(n, nrhs), dtype=torch.uint8, device=dev)

    def precond(R):
        Z = chol.colmajor((R * d[:, None]).to(torch.float32))
        chol.solve_f32(L, Z, work=swork)
        return Z.to(torch.float64) * d[:, None]

    normA = float(A.abs().sum(1).max())

    def eta(X):
        R = B - A @ X
        return float((R.abs().amax(0) / (normA * X.abs().amax(0) + B.abs().amax(0))).amax())

    X = torch.zeros_like(B)
    R = B.clone()
    Z = precond(R)
    P = Z.clone()
    rz = (R * Z).sum(0)
    it, e_last = 0, 1.0
    t_mv = t_pc = 0.0
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    while it < args.pcg_maxit:
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        a2 = torch.cuda.Event(enable_timing=True)
        a0.record()
        Q = A @ P
        a1.record()
        alpha = rz / (P * Q).sum(0)
        X += alpha * P
        R -= alpha * Q
        Z = precond(R)
        a2.record()
        rz_new = (R * Z).sum(0)
        P = Z + (rz_new / rz) * P
        rz = rz_new
        it += 1
        torch.cuda.synchronize()
        t_mv += a0.elapsed_time(a1)
        t_pc += a1.elapsed_time(a2)
        if it % 10 == 0:
            e_last = eta(X)
            if e_last <= 1e-14:
                break
    total_s = time.perf_counter() - t_start
    return {"workload": "n=%d, %d RHS, kappa = 1e6 (the mixed-precision configuration)" % (n, nrhs),
            "preconditioner": "BF16 tensor-core factor (one term, FP32 accumulation) of D^-1/2 A D^-1/2 + sigma I",
            "sigma": sigma, "factor_ms": round(factor_ms, 2), "iterations": it, "backward_error": e_last,
            "reached_target": e_last <= 1e-14, "seconds": round(total_s, 3),
            "ms_per_iteration_product": round(t_mv / max(it, 1), 3),
            "ms_per_iteration_preconditioner": round(t_pc / max(it, 1), 3)}


def run_lu(args, chol, dev):
    """The LU configuration (the paper's DGETRF workload, Section 4.1): a general n x n matrix
    with i.i.d. N(0,1) entries, tile LU with incremental pivoting on the persistent kernel
    (inner blocks of 32), --lu-steps factorizations timed with CUDA events after one warm-up,
    each on a fresh copy of A; GFLOP/s with 2n^3/3 flops. One solve with one right-hand side
    checks the timed factors (backward error on the device)."""
    import torch
    import synth
    n = args.lu_n
    o = chol.opts(nb=args.lu_nb, policy=args.lu_policy, alpha=args.alpha, use_cp=args.cp)
    A0 = chol.colmajor(synth.general_matrix(n, seed=args.seed + 11, device=dev))
    A = torch.empty_like(A0)
    work = torch.empty(chol.lu_workspace_size(n, o), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed_factors(o):
        A.copy_(A0)
        f = chol.lu_factor(A, o, work=work, stream=stream)
        torch.cuda.synchronize()
        if int(f.info.item()) != 0:
            raise RuntimeError("LU info %d" % int(f.info.item()))
        ms = []
        for _ in range(args.lu_steps):
            A.copy_(A0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f = chol.lu_factor(A, o, work=work, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return f, ms

    sweep = None
    if args.lu_sweep:
        sweep = []
        for pol, alpha, cp in (("heft", 0.5, False), ("heft", 0.5, True), ("dada", 0.0, False), ("dada", 0.5, False),
                               ("dada", 1.0, False), ("dada", 0.5, True), ("steal", 0.5, False),
                               ("static", 0.5, False)):
            _, pm = timed_factors(chol.opts(nb=args.lu_nb, policy=pol, alpha=alpha, use_cp=cp))
            pt = sum(pm) / len(pm)
            sweep.append({"policy": pol + ("(%g)" % alpha if pol == "dada" else "") + ("+CP" if cp else ""),
                          "factor_ms": round(pt, 2), "gflops": round(2.0 * n ** 3 / 3.0 / (pt / 1000.0) / 1e9, 1)})
    f, ms = timed_factors(o)
    b = chol.colmajor(synth.rhs(n, 1, seed=args.seed + 12, device=dev))
    x = b.clone()
    swork = torch.empty(chol.lu_solve_workspace_size(n, 1, o), dtype=torch.uint8, device=dev)
    sinfo = torch.zeros(1, dtype=torch.int32, device=dev)
    chol.lu_solve(f, x, work=swork, info=sinfo, stream=stream)   # warm-up
    solve_ms_all = []
    for _ in range(30):
        x.copy_(b)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        chol.lu_solve(f, x, work=swork, info=sinfo, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        solve_ms_all.append(e0.elapsed_time(e1))
    if int(sinfo.item()) != 0:
        raise RuntimeError("LU solve info %d" % int(sinfo.item()))
    solve_ms = sum(solve_ms_all) / len(solve_ms_all)
    berr = _backward_error(A0, x, b)
    t = sum(ms) / len(ms)
    gf = 2.0 * n ** 3 / 3.0 / (t / 1000.0) / 1e9
    T = -(-n // (o.nb if o.nb else (128 if n <= 32768 else 256)))
    return {"workload": "tile LU with incremental pivoting (GETRF/GESSM/TSTRF/SSSSM), n=%d, tile %s, inner "
                        "block 32, %s%s ready queues; A with i.i.d. N(0,1) entries" % (
                            n, o.nb or "auto", args.lu_policy.upper(),
                            ("(%g)" % args.alpha if args.lu_policy == "dada" else "") + ("+CP" if args.cp else "")),
            "factor_ms": round(t, 2), "factor_ms_stat": stat(ms, 3), "gflops": round(gf, 1), "flops": "2n^3/3",
            "frac_of_fp64_peak": round(gf / FP64_PEAK_GFLOPS, 4), "tiles": T,
            "tasks": int(chol.lib.chol_lu_dag_task_count(T)),
            "solve_ms_1rhs": round(solve_ms, 3), "solve_ms_1rhs_stat": stat(solve_ms_all, 3),
            "solve_backward_error": berr, "info": int(f.info.item()),
            "policies": sweep}


def run_batched(args, chol, dev):
    """The batched configuration: --batch SPD matrices with orders uniform in [16, 512]
    (A_m = sym(G G^T)/n + I), one right-hand side each, factored and solved by one persistent
    launch, FP64 and FP32. The launch shape comes from the library's autotuner; each step
    (restore the inputs, order + factor + solve) is one CUDA graph replay."""
    import torch
    import synth
    orders = [int(n) for n in synth.batch_orders(args.batch, 16, 512, seed=args.seed)]
    flops = sum(n ** 3 / 3.0 + 2.0 * n * n for n in orders)
    out = {"workload": "%d SPD matrices, n uniform in [16, 512], 1 RHS each, one persistent launch per "
                       "step under a CUDA graph" % len(orders), "flops_per_step": flops}
    roffs, off = [], 0
    for n in orders:
        roffs.append(off)
        off += n
    for name, dtype in (("f64", torch.float64), ("f32", torch.float32)):
        flat, offs = synth.gram_spd_batch(orders, seed=args.seed + 3, device=dev, dtype=dtype)
        g = torch.Generator(device=dev).manual_seed(args.seed + 4)
        rhs = torch.randn(off, generator=g, device=dev, dtype=torch.float64).to(dtype)
        src = chol.Batch(flat, offs, orders, rhs, roffs)
        scratch = chol.Batch(flat.clone(), offs, orders, rhs.clone(), roffs)
        best, tune_ms = chol.batched_autotune(src, scratch)
        del scratch
        work = chol.Batch(flat.clone(), offs, orders, rhs.clone(), roffs)
        stream = torch.cuda.Stream(dev)

        def step():
            work.flat.copy_(src.flat)
            work.rhs_flat.copy_(src.rhs_flat)
            chol.posv_batched(work, best, stream=stream)

        with torch.cuda.stream(stream):
            step()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            step()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.batched_steps + 1)]
        with torch.cuda.stream(stream):  # replay() launches on the current stream
            for _ in range(2):
                graph.replay()
            torch.cuda.synchronize()
            for k in range(args.batched_steps):
                ev[k].record(stream)
                graph.replay()
            ev[-1].record(stream)
        torch.cuda.synchronize()
        step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.batched_steps)]
        ms = sum(step_ms) / len(step_ms)
        bad = int((work.info != 0).sum().item())
        berr = 0.0
        for m in range(0, len(orders), max(1, len(orders) // 16)):
            A = src.matrix(m).to(torch.float64)
            b = src.rhs(m).to(torch.float64)
            x = work.rhs(m).to(torch.float64)
            r = b - A @ x
            berr = max(berr, float(r.abs().max() / (A.abs().sum(1).max() * x.abs().max() + b.abs().max())))
        out[name] = {"ms": round(ms, 3), "ms_stat": stat(step_ms, 3), "gflops": round(flops / ms / 1e6, 1),
                     "matrices_per_s": round(len(orders) / ms * 1e3, 1), "failed": bad,
                     "backward_error_sample_max": berr,
                     "autotuned": {"workers_per_sm": best.workers_per_sm, "lpt_order": best.lpt_order,
                                   "wide_panel_min_n": best.wide_panel_min_n if name == "f64" else None,
                                   "tuning_ms_best": round(tune_ms, 3)}}
        del src, work, flat, rhs, graph
        torch.cuda.empty_cache()
    return out


def run_adjoint(args, chol, dev):
    """The differentiation configuration: --adj-batch FP64 SPD matrices of order --adj-n
    (A = sym(G G^T)/n + I), loss = sum(w * x) with x = A^-1 b and w, b ~ N(0,1). One step =
    for every matrix the forward pass (factor + solve) and the backward pass (solve adjoint,
    then Cholesky adjoint) through the library's entry points, timed with CUDA events. The
    matrices are independent: they go round-robin to --adj-streams streams, and each factor
    runs with --adj-workers workers and tile --adj-nb (16 and 64: measured on the GB300
    against tiles 32-256, 8-64 workers and 4-32 streams; a tile-64 factor of order 1024 has
    at most 120 ready tasks, each one short), so several factorizations share the GPU. Flops per matrix: n^3/3 + 2n^2 forward; backward
    n^3/3 for L^T Lbar on the lower tiles, 2n^3 for the two triangular solves with n
    right-hand sides, O(n^2) for the rest."""
    import torch
    import synth
    n, m, ns = args.adj_n, args.adj_batch, max(1, args.adj_streams)
    As = [chol.colmajor(synth.gram_spd(n, seed=args.seed + 100 + i, device=dev)) for i in range(m)]
    bw = synth.rhs(n, 2 * m, seed=args.seed + 11, device=dev)
    bs = [chol.colmajor(bw[:, i:i + 1]) for i in range(m)]
    ws = [chol.colmajor(bw[:, m + i:m + i + 1]) for i in range(m)]
    o = chol.opts(nb=args.adj_nb, num_workers=args.adj_workers)
    main = torch.cuda.current_stream(dev)
    streams = [torch.cuda.Stream(dev) for _ in range(ns)]
    Fs = [torch.empty_like(As[0]) for _ in range(ns)]
    Xs = [torch.empty_like(bs[0]) for _ in range(ns)]
    fworks = [torch.empty(chol.workspace_size(n, o), dtype=torch.uint8, device=dev) for _ in range(ns)]
    sworks = [torch.empty(chol.solve_workspace_size(n, 1), dtype=torch.uint8, device=dev) for _ in range(ns)]
    infos = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in range(ns)]
    grads = [None] * m

    def step():
        start = torch.cuda.Event()
        start.record(main)
        for st in streams:
            st.wait_event(start)
        for i in range(m):
            k = i % ns
            st, F, X = streams[k], Fs[k], Xs[k]
            with torch.cuda.stream(st):
                F.copy_(As[i])
                X.copy_(bs[i])
                chol.factor(F, o, work=fworks[k], info=infos[k], stream=st)
                chol.solve(F, X, work=sworks[k], info=infos[k], stream=st)
                _, Lbar = chol.solve_backward(F, X, ws[i], stream=st)
                grads[i] = chol.cholesky_backward(F, Lbar, stream=st)
        for st in streams:
            done = torch.cuda.Event()
            done.record(st)
            main.wait_event(done)

    step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.adj_steps + 1)]
    for k in range(args.adj_steps):
        ev[k].record(main)
        step()
    ev[-1].record(main)
    torch.cuda.synchronize()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.adj_steps)]
    ms = sum(step_ms) / len(step_ms)
    flops = m * (n ** 3 / 3.0 + 2.0 * n * n + n ** 3 / 3.0 + 2.0 * n ** 3)
    bad = sum(int(x.item()) != 0 for x in infos)
    # check (outside the timed region): Abar = -(lam x^T + x lam^T)/2 with lam = A^-1 w
    worst = 0.0
    for i in (0, m // 2, m - 1):
        x = torch.linalg.solve(As[i], bs[i])
        lam = torch.linalg.solve(As[i], ws[i])
        ref = -0.5 * (lam @ x.T + x @ lam.T)
        worst = max(worst, float(torch.linalg.norm(grads[i] - ref) / torch.linalg.norm(ref)))
    return {"workload": "%d FP64 SPD matrices n=%d (A = sym(G G^T)/n + I), loss = sum(w * x), x = A^-1 b; "
                        "forward factor + solve and backward solve + Cholesky adjoints per matrix, tile %d, "
                        "%d streams, %d factor workers per matrix" % (m, n, args.adj_nb, ns, args.adj_workers),
            "ms": round(ms, 2), "ms_stat": stat(step_ms, 2), "ms_per_matrix": round(ms / m, 3),
            "flops_per_step": flops,
            "gflops": round(flops / ms / 1e6, 1), "frac_of_fp64_peak": round(flops / ms / 1e6 / FP64_PEAK_GFLOPS, 4),
            "nonzero_info": bad, "grad_rel_diff_vs_closed_form": worst}


def run_e2e(args, chol, A0, B0, o, dev):
    """Same metric through chol_posv_host with pinned host buffers: every step copies A and B
    to the device, factors, solves and copies L and X back inside the timed region."""
    import torch
    n, nrhs = args.n, args.nrhs
    hA0 = A0.cpu().numpy()   # Fortran-ordered (column-major) host copy
    hB0 = B0.cpu().numpy()
    pA = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()  # column-major pinned
    pB = torch.empty((nrhs, n), dtype=torch.float64, pin_memory=True).t()
    hA = pA.numpy()
    hB = pB.numpy()
    stage = torch.empty(chol.lib.chol_posv_host_stage_size(n, nrhs, __import__("ctypes").byref(o)),
                        dtype=torch.uint8, device=dev)
    tt = 0.0
    step_ms = []
    for _ in range(max(1, args.e2e_steps)):
        hA[...] = hA0
        hB[...] = hB0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = chol.posv_host(hA, hB, o, stage=stage)
        dt = time.perf_counter() - t0
        tt += dt
        step_ms.append(dt * 1e3)
        if info != 0:
            raise RuntimeError("posv_host info %d" % info)
    steps = max(1, args.e2e_steps)
    del stage
    return {"value": round(step_flops(n, nrhs) * steps / tt / 1e9, 2), "unit": "GFLOP/s",
            "h2d_bytes_per_step": n * n * 8 + n * nrhs * 8, "d2h_bytes_per_step": n * n * 8 + n * nrhs * 8 + 4,
            "steps": steps, "step_ms": stat(step_ms, 2), "api": "chol_posv_host (pinned host buffers)"}


if __name__ == "__main__":
    main()
