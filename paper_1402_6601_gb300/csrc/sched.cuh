// The activate operation: placement of newly ready tasks on workers (Section 2.2).
//
// Workers are identical (thread blocks of one GPU), so each task has one processing time p
// and the speedup S_i = p_CPU / p_GPU of the paper is 1 for every task.
//
//  HEFT (Algorithm 1): the ready list is taken in decreasing priority -- the bottom level,
//  i.e. the upward rank of the original HEFT rule, since sorting by S_i orders nothing here
//  -- and each task goes to the worker with the earliest finish time; that worker's
//  predicted completion time-stamp grows by p (Section 2.3).
//
//  DADA (Algorithm 2): binary search on a makespan guess lambda between 0 and
//  sum(p) + max(load). For each guess, a local affinity phase puts every task that has an
//  affinity worker (the worker that last wrote the tile the task modifies; score = bytes
//  of that tile, Section 3.2) on that worker while the worker's load is still below
//  alpha * lambda (the last task placed may overreach it), then a global balance phase
//  places the rest by decreasing p on the earliest-finishing worker. A guess is accepted
//  when every load fits in (2 + alpha) * lambda; the last accepted schedule is pushed.
//  The search stops when upper - lower <= eps * (first upper) or after max_iter halvings.
//
//  Communication prediction (DADA(alpha)+CP, and HEFT's transfer-aware finish time): a task
//  costs p plus `comm` for each input tile the worker did not write last (cost_on); the
//  finish times of both algorithms and DADA's loads then use that cost.
//
// The same code runs on the host (Exec = HostExec, one thread) and on the device inside
// the persistent kernel (Exec = WarpExec: all 32 lanes of one warp execute it in lockstep,
// the leader lane performs the sequential writes, and the worker scans are warp-parallel).
// Ties between workers go to the lowest index in both, so both give the same placement.
#pragma once
#include <stdint.h>
#include "dag.cuh"

namespace chol {

enum Policy { P_HEFT = 0, P_DADA = 1, P_STEAL = 2, P_STATIC = 3 };

struct ReadyTask {
  int tid;        // task id (lower wins ties)
  int aff;        // affinity worker or -1
  int64_t p;      // processing time, ns
  int64_t prio;   // bottom level, ns
  int64_t score;  // affinity score, bytes
  int64_t comm;   // communication prediction: cost of one input tile not owned by the worker
  int own[3];     // workers that last wrote the task's input tiles (-1: none)
  int nin;        // number of input tiles (1..3)
};

// Cost of task t on worker w; with communication prediction every input tile that w did
// not write last adds t.comm.
CHOL_HD int64_t cost_on(const ReadyTask &t, int w, bool cp) {
  if (!cp) return t.p;
  const int cnt = (t.own[0] == w) + (t.own[1] == w) + (t.own[2] == w);
  return t.p + t.comm * (t.nin - cnt);
}

struct HostExec {
  static constexpr bool WARP = false;
  CHOL_HD static bool leader() { return true; }
  CHOL_HD static void sync() {}
  CHOL_HD static int lane() { return 0; }
  CHOL_HD static int width() { return 1; }
  // argmin of load[w] over w, ties to the lowest w
  CHOL_HD static int argmin(const int64_t *load, int W) {
    int best = 0;
    for (int w = 1; w < W; ++w)
      if (load[w] < load[best]) best = w;
    return best;
  }
  CHOL_HD static int64_t maxval(const int64_t *load, int W) {
    int64_t m = load[0];
    for (int w = 1; w < W; ++w) m = load[w] > m ? load[w] : m;
    return m;
  }
  CHOL_HD static int64_t sum_p(const ReadyTask *LR, int m, bool cp) {
    int64_t s = 0;
    for (int i = 0; i < m; ++i) s += LR[i].p + (cp ? LR[i].comm * LR[i].nin : 0);
    return s;
  }
};

#ifdef __CUDACC__
struct WarpExec {
  static constexpr bool WARP = true;
  __device__ static bool leader() { return (threadIdx.x & 31) == 0; }
  __device__ static void sync() { __syncwarp(); }
  __device__ static int lane() { return threadIdx.x & 31; }
  __device__ static int width() { return 32; }
  __device__ static int argmin(const int64_t *load, int W) {
    const int l = threadIdx.x & 31;
    int64_t bv = INT64_MAX;
    int bw = 0x7fffffff;
    for (int w = l; w < W; w += 32) {
      const int64_t v = load[w];
      if (v < bv) { bv = v; bw = w; }  // w increases per lane: first minimum kept
    }
    for (int o = 16; o > 0; o >>= 1) {
      const int64_t ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int ow = __shfl_xor_sync(0xffffffffu, bw, o);
      if (ov < bv || (ov == bv && ow < bw)) { bv = ov; bw = ow; }
    }
    return bw;
  }
  __device__ static int64_t maxval(const int64_t *load, int W) {
    const int l = threadIdx.x & 31;
    int64_t m = INT64_MIN;
    for (int w = l; w < W; w += 32) m = load[w] > m ? load[w] : m;
    for (int o = 16; o > 0; o >>= 1) {
      const int64_t om = __shfl_xor_sync(0xffffffffu, m, o);
      m = om > m ? om : m;
    }
    return m;
  }
  __device__ static int64_t sum_p(const ReadyTask *LR, int m, bool cp) {
    const int l = threadIdx.x & 31;
    int64_t s = 0;
    for (int i = l; i < m; i += 32) s += LR[i].p + (cp ? LR[i].comm * LR[i].nin : 0);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
  }
};
#endif

// Scratch the placement needs: three orderings of the ready list, two assignments and a
// trial copy of the loads.
struct PlaceScratch {
  int *ord_prio;   // m: push order (decreasing priority, then lower tid)
  int *ord_aff;    // m: affinity phase order (decreasing score, priority, lower tid)
  int *ord_lpt;    // m: balance phase order (decreasing p, priority, lower tid)
  int *assign;     // m: output worker per ready-list index
  int *trial;      // m: worker per index in the current trial, -1 = unplaced
  int64_t *tload;  // W: loads in the current trial
};

CHOL_HD bool before_prio(const ReadyTask &a, const ReadyTask &b) {
  if (a.prio != b.prio) return a.prio > b.prio;
  return a.tid < b.tid;
}
CHOL_HD bool before_aff(const ReadyTask &a, const ReadyTask &b) {
  if (a.score != b.score) return a.score > b.score;
  return before_prio(a, b);
}
CHOL_HD bool before_lpt(const ReadyTask &a, const ReadyTask &b) {
  if (a.p != b.p) return a.p > b.p;
  return before_prio(a, b);
}

template <int KEY>
CHOL_HD bool before_key(const ReadyTask &a, const ReadyTask &b) {
  return KEY == 0 ? before_prio(a, b) : KEY == 1 ? before_aff(a, b) : before_lpt(a, b);
}

// Insertion sort of indices; m is at most T - 1 and this runs once per activation.
template <int KEY>
CHOL_HD void sort_indices(int *ord, const ReadyTask *LR, int m) {
  for (int i = 0; i < m; ++i) ord[i] = i;
  for (int i = 1; i < m; ++i) {
    const int v = ord[i];
    int j = i - 1;
    while (j >= 0) {
      const bool bef = KEY == 0 ? before_prio(LR[v], LR[ord[j]])
                     : KEY == 1 ? before_aff(LR[v], LR[ord[j]])
                                : before_lpt(LR[v], LR[ord[j]]);
      if (!bef) break;
      ord[j + 1] = ord[j];
      --j;
    }
    ord[j + 1] = v;
  }
}

// The same order from the whole warp (device): every lane ranks its tasks against all the
// others -- the comparisons are a strict total order (ties end at the task id), so the ranks
// are a permutation, the one the insertion sort produces. O(m^2 / 32) comparisons per lane
// with broadcast reads instead of O(m^2) on one lane: this sort sits on every activation,
// so on the factor's critical path.
template <int KEY, class X>
CHOL_HD void sort_ready(int *ord, const ReadyTask *LR, int m) {
  if constexpr (X::WARP) {
    for (int i = X::lane(); i < m; i += X::width()) {
      const ReadyTask t = LR[i];
      int r = 0;
      for (int j = 0; j < m; ++j) r += before_key<KEY>(LR[j], t) ? 1 : 0;
      ord[r] = i;
    }
  } else {
    sort_indices<KEY>(ord, LR, m);
  }
}

// Worker with the earliest finish time load[w] + cost_on(t, w), ties to the lowest index.
// Without communication prediction that is the least-loaded worker. With it, only the
// (at most three) workers owning input tiles can beat the least-loaded worker, so they are
// the only ones evaluated besides it.
template <class X>
CHOL_HD int eft_worker(const int64_t *load, int W, const ReadyTask &t, bool cp) {
  const int w0 = X::argmin(load, W);
  if (!cp) return w0;
  int bw = w0;
  int64_t best = load[w0] + cost_on(t, w0, cp);
  for (int a = 0; a < 3; ++a) {
    const int o = t.own[a];
    if (o < 0 || o >= W) continue;
    const int64_t v = load[o] + cost_on(t, o, cp);
    if (v < best || (v == best && o < bw)) {
      best = v;
      bw = o;
    }
  }
  return bw;
}

// One DADA trial at guess lam; returns whether all loads fit in (2 + alpha) lam.
template <class X>
CHOL_HD bool dada_trial(const ReadyTask *LR, int m, const int64_t *load, int W, double alpha,
                        int64_t lam, PlaceScratch &s, bool cp) {
  for (int w = X::lane(); w < W; w += X::width()) s.tload[w] = load[w];
  for (int i = X::lane(); i < m; i += X::width()) s.trial[i] = -1;
  X::sync();
  if (X::leader()) {
    const double thr = alpha * (double)lam;
    for (int q = 0; q < m; ++q) {
      const int i = s.ord_aff[q];
      const int w = LR[i].aff;
      if (w < 0 || w >= W) continue;
      if ((double)s.tload[w] < thr) {
        s.trial[i] = w;
        s.tload[w] += cost_on(LR[i], w, cp);
      }
    }
  }
  X::sync();
  for (int q = 0; q < m; ++q) {
    const int i = s.ord_lpt[q];
    if (s.trial[i] >= 0) continue;   // uniform: every lane reads the same shared value
    const int w = eft_worker<X>(s.tload, W, LR[i], cp);
    X::sync();
    if (X::leader()) {
      s.trial[i] = w;
      s.tload[w] += cost_on(LR[i], w, cp);
    }
    X::sync();
  }
  const int64_t mx = X::maxval(s.tload, W);
  X::sync();
  return (double)mx <= (2.0 + alpha) * (double)lam;
}

#ifdef __CUDACC__
// HEFT without communication prediction on the device: every task, in priority order, goes to
// the least-loaded worker (ties to the lowest index), as eft_worker decides. Each lane keeps
// the minimum over its own workers (w = lane, lane + 32, ...) as one key (load << 11 | w);
// after a placement only the lane owning the chosen worker rescans its workers, and a 5-step
// shuffle minimum gives the next choice, instead of a scan of all W loads per task.
// Returns false (nothing placed) if a load is negative or too large for the key.
__device__ __forceinline__ bool heft_place_warp(const ReadyTask *LR, int m, int64_t *load, int W, PlaceScratch &s) {
  const int lane = threadIdx.x & 31;
  bool bad = false;
  for (int w = lane; w < W; w += 32) bad |= load[w] < 0 || load[w] >= (int64_t(1) << 51);  // + m p < 2^51 + 2^50: keys stay below 2^63
  for (int i = lane; i < m; i += 32) bad |= LR[i].p < 0 || LR[i].p >= (int64_t(1) << 40);
  if (__any_sync(0xffffffffu, bad)) return false;
  auto local_min = [&]() {
    unsigned long long best = ~0ull;
    for (int w = lane; w < W; w += 32) {
      const unsigned long long key = ((unsigned long long)load[w] << 11) | (unsigned)w;
      best = key < best ? key : best;
    }
    return best;
  };
  unsigned long long mine = local_min();
  for (int q = 0; q < m; ++q) {
    unsigned long long k = mine;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
      k = ok < k ? ok : k;
    }
    const int w = (int)(k & 2047ull);
    const int i = s.ord_prio[q];
    if (lane == (w & 31)) {
      load[w] += LR[i].p;
      mine = local_min();
    }
    if (lane == 0) s.assign[i] = w;
  }
  __syncwarp();
  return true;
}
#endif

// Place the m ready tasks. load[W] is updated with the chosen placement. Returns the number
// of bisection steps taken (DADA) or 0.
template <class X>
CHOL_HD int place(int policy, double alpha, int max_iter, double eps, const ReadyTask *LR, int m,
                  int64_t *load, int W, PlaceScratch &s, bool cp = false) {
  if (m <= 0) return 0;
  sort_ready<0, X>(s.ord_prio, LR, m);
  X::sync();
  int iters = 0;
  if (policy == P_HEFT) {
#ifdef __CUDA_ARCH__
    if constexpr (X::WARP) {
      if (!cp && W <= 2048 && heft_place_warp(LR, m, load, W, s)) return 0;
    }
#endif
    for (int q = 0; q < m; ++q) {
      const int i = s.ord_prio[q];
      const int w = eft_worker<X>(load, W, LR[i], cp);
      X::sync();
      if (X::leader()) {
        s.assign[i] = w;
        load[w] += cost_on(LR[i], w, cp);
      }
      X::sync();
    }
    return 0;
  }
  // DADA
  sort_ready<1, X>(s.ord_aff, LR, m);
  sort_ready<2, X>(s.ord_lpt, LR, m);
  X::sync();
  int64_t lower = 0;
  int64_t upper = X::sum_p(LR, m, cp) + X::maxval(load, W);
  X::sync();
  const int64_t eps_abs = (int64_t)((double)upper * eps);
  dada_trial<X>(LR, m, load, W, alpha, upper, s, cp);  // always fits: every load <= upper
  for (int i = X::lane(); i < m; i += X::width()) s.assign[i] = s.trial[i];
  X::sync();
  while (upper - lower > eps_abs && iters < max_iter) {
    const int64_t lam = (upper + lower) / 2;
    const bool fits = dada_trial<X>(LR, m, load, W, alpha, lam, s, cp);
    if (fits) {
      upper = lam;
      for (int i = X::lane(); i < m; i += X::width()) s.assign[i] = s.trial[i];
    } else {
      lower = lam;
    }
    X::sync();
    ++iters;
  }
  if (X::leader())
    for (int q = 0; q < m; ++q) load[s.assign[q]] += cost_on(LR[q], s.assign[q], cp);
  X::sync();
  return iters;
}

}  // namespace chol
