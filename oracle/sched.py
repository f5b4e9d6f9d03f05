"""One activate operation of the paper's two list-scheduling policies, on identical workers.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Setting (Section 3): the paper schedules on m CPUs and k GPUs with per-task processing
times p_i^CPU and p_i^GPU. Here every worker is one of a single kind (persistent thread
blocks of one GPU), so each task has one processing time p_i, the speedup S_i is 1 for all
tasks, and the CPU-only / GPU-only extraction steps of the dual approximation are empty.

Inputs of one activation: the list LR of newly ready tasks, each with
  p      processing time (integer ns)
  prio   bottom-level (integer ns) -- the priority of the original HEFT rule, which the
         paper names next to its speedup rule; with S_i = 1 for all tasks the speedup sort
         orders nothing, so the bottom-level order is used
  aff    the worker that last wrote the tile the task modifies, or -1
  score  the affinity score: bytes of that tile (the paper scores a (task, resource) pair
         by the amount of data the task updates on that resource, Section 3.2 "Affinity")
  tid    task id, the final tie-break (lower first)
and load[w] >= 0: the predicted time until worker w has finished the work already queued
on it (Section 2.3: a shared time-stamp per processor of its predicted completion date).

Ties between workers go to the lowest worker index.
"""


def heft(LR, load):
    """Algorithm 1. Returns a list of (tid, worker) in push order."""
    load = list(load)
    order = sorted(LR, key=lambda t: (-t["prio"], t["tid"]))
    out = []
    for t in order:
        best_w, best_f = -1, None
        for w, l in enumerate(load):
            f = l + t["p"]
            if best_f is None or f < best_f:
                best_w, best_f = w, f
        load[best_w] = best_f
        out.append((t["tid"], best_w))
    return out


def _dada_trial(LR, load0, alpha, lam):
    load = list(load0)
    placed = {}
    # local affinity phase: each task with an affinity worker goes there while that worker's
    # load is still below alpha * lambda (the last task placed may cross the threshold)
    for t in sorted([t for t in LR if t["aff"] >= 0], key=lambda t: (-t["score"], -t["prio"], t["tid"])):
        w = t["aff"]
        if float(load[w]) < alpha * float(lam):
            placed[t["tid"]] = w
            load[w] += t["p"]
    # global balance phase: the rest by decreasing processing time, each on the worker that
    # finishes it first
    rest = [t for t in LR if t["tid"] not in placed]
    for t in sorted(rest, key=lambda t: (-t["p"], -t["prio"], t["tid"])):
        best_w, best_f = -1, None
        for w, l in enumerate(load):
            f = l + t["p"]
            if best_f is None or f < best_f:
                best_w, best_f = w, f
        placed[t["tid"]] = best_w
        load[best_w] = best_f
    fits = float(max(load)) <= (2.0 + alpha) * float(lam)
    return placed, fits


def dada(LR, load, alpha, eps_frac=0.01, max_iter=16):
    """Algorithm 2. Binary search on the makespan guess lambda between lower = 0 and
    upper = sum_i p_i + max_w load_w; keep the last schedule that fits in (2 + alpha) lambda.
    The bisection stops when upper - lower <= eps (1% of the first upper) or after max_iter
    halvings. Returns (list of (tid, worker) in push order, number of halvings)."""
    if not LR:
        return [], 0
    lower = 0
    upper = sum(t["p"] for t in LR) + max(load)
    eps = int(upper * eps_frac)
    best, fits = _dada_trial(LR, load, alpha, upper)
    assert fits
    it = 0
    while upper - lower > eps and it < max_iter:
        lam = (upper + lower) // 2
        placed, fits = _dada_trial(LR, load, alpha, lam)
        if fits:
            upper = lam
            best = placed
        else:
            lower = lam
        it += 1
    order = sorted(LR, key=lambda t: (-t["prio"], t["tid"]))
    return [(t["tid"], best[t["tid"]]) for t in order], it


# ----------------------------------------------------------------------------------------
# Communication prediction (DADA(alpha)+CP, Section 4.1 "Methodology"; HEFT always counts
# transfers in its earliest finish time). On one GPU a "transfer" is the cost of bringing a
# task's input tiles to a worker that did not last write them: each task lists the workers
# owning its input tiles (own, up to three) and a per-tile cost comm (ns); on worker w the
# task then costs p + comm * (number of its input tiles not owned by w).

def _cost_on(t, w):
    own = [o for o in t.get("own", []) if o >= 0]
    nin = t.get("nin", 0)
    return t["p"] + t.get("comm", 0) * (nin - sum(1 for o in own if o == w))


def _eft(t, load):
    best_w, best_f = -1, None
    for w, l in enumerate(load):
        f = l + _cost_on(t, w)
        if best_f is None or f < best_f:
            best_w, best_f = w, f
    return best_w, best_f


def heft_cp(LR, load):
    """Algorithm 1 with transfer time in the finish time."""
    load = list(load)
    out = []
    for t in sorted(LR, key=lambda t: (-t["prio"], t["tid"])):
        w, f = _eft(t, load)
        load[w] = f
        out.append((t["tid"], w))
    return out


def _dada_cp_trial(LR, load0, alpha, lam):
    load = list(load0)
    placed = {}
    for t in sorted([t for t in LR if t["aff"] >= 0], key=lambda t: (-t["score"], -t["prio"], t["tid"])):
        w = t["aff"]
        if float(load[w]) < alpha * float(lam):
            placed[t["tid"]] = w
            load[w] += _cost_on(t, w)
    rest = [t for t in LR if t["tid"] not in placed]
    for t in sorted(rest, key=lambda t: (-t["p"], -t["prio"], t["tid"])):
        w, f = _eft(t, load)
        placed[t["tid"]] = w
        load[w] = f
    return placed, float(max(load)) <= (2.0 + alpha) * float(lam)


def dada_cp(LR, load, alpha, eps_frac=0.01, max_iter=16):
    """Algorithm 2 with communication prediction: task costs depend on the worker as above;
    upper = sum_i (p_i + comm_i * nin_i) + max_w load_w."""
    if not LR:
        return [], 0
    lower = 0
    upper = sum(t["p"] + t.get("comm", 0) * t.get("nin", 0) for t in LR) + max(load)
    eps = int(upper * eps_frac)
    best, fits = _dada_cp_trial(LR, load, alpha, upper)
    assert fits
    it = 0
    while upper - lower > eps and it < max_iter:
        lam = (upper + lower) // 2
        placed, fits = _dada_cp_trial(LR, load, alpha, lam)
        if fits:
            upper = lam
            best = placed
        else:
            lower = lam
        it += 1
    order = sorted(LR, key=lambda t: (-t["prio"], t["tid"]))
    return [(t["tid"], best[t["tid"]]) for t in order], it
