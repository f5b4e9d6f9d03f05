// Persistent data-flow kernel for the tiled Cholesky factorization.
//
// One thread block per worker (Section 2: one worker per processing unit, each with a
// local ready queue). A worker loops: pop a task from its own queue, else steal from a
// random victim (Section 2.1 "Execution flow"), run the tile body, then activate the
// successors whose dependency counters reach zero and place them on workers' queues with
// the chosen policy (Section 2.2; Algorithms 1 and 2). The predicted completion
// time-stamp of a worker (Section 2.3) is the predicted end of the task it runs plus the
// predicted times of the tasks queued on it; both are kept in device memory and updated
// with atomics, and the running task's term is corrected from the real clock when the
// task starts and ends.
//
// Ready queues are arrays of 64-bit slots (0 = empty; otherwise the priority key in the
// high word and the complemented task id in the low word). Push claims an empty slot with
// a compare-and-swap; pop and steal scan a queue with one warp and claim the slot with the
// largest key. At any time at most one task per tile is ready (the tasks writing a tile
// form a chain), so at most T(T+1)/2 tasks are queued in total; every queue has
// C >= T(T+1)/(2W) + 64 slots, and a push that finds its queue full goes to the next
// queue, so a push always finds a slot (the spill is counted in the control block).
//
// Every wait is bounded: a worker that finds no work sleeps with back-off, and if the
// count of completed tasks does not move for opts.timeout_ns (or a matching iteration
// count) it raises the abort flag and writes CHOL_INFO_TIMEOUT; all workers then return.
#include <algorithm>
#include <mutex>
#include "common.cuh"
#include "dag.cuh"
#include "dag_lu.cuh"
#include "internal.cuh"
#include "sched.cuh"
#include "tiles_f32.cuh"
#include "tiles_tc.cuh"
#include "tiles_f64.cuh"
#include "tiles_lu.cuh"

namespace chol {

constexpr int SM_SLOTS = 1024;  // %smid values tracked by the co-scheduling rule

// Control block. The counters that every task touches (done, queued, free_sms) and the words
// that idle workers poll (abort, help_open) sit on separate 128-byte lines, so that polling
// and the atomics of running workers do not queue behind one another on one line.
struct Ctrl {
  alignas(128) int done;
  alignas(128) int abort;
  int info;
  unsigned int fifo_seq;
  int spills;
  alignas(128) int queued;    // tasks in all queues
  alignas(128) int free_sms;  // SMs that host a worker and run no task
  alignas(128) int help_open; // split tasks with units not yet claimed
};

// A task cut into units that idle workers help with (one slot per worker, written by the
// worker that runs the task). `word` holds the slot's generation (bits 40..63), the number
// of units (bits 32..39) and the next unit to hand out (bits 0..31): the owner takes units
// with an atomic add, a helper with a compare-and-swap that also checks the generation, so a
// helper holding an old view of the slot can never take a unit of a later task.
struct __align__(128) HelpSlot {
  unsigned long long word;
  int done;  // units finished
  int kind, i, j, k;
  int pad[26];
};

struct FactorArgs {
  void *A;  // double or float, by the kernel instantiation
  int64_t lda;
  int n, nb, T;
  int64_t ntasks;
  int W, C;
  int policy, queue_order, steal, dada_max_iter, trace;
  double alpha, dada_eps;
  int64_t cost[4];
  int64_t timeout_ns, iter_limit;
  Ctrl *ctrl;
  int *cnt;
  int64_t *bl;
  int *owner;
  unsigned long long *slots;
  unsigned int *qhead;
  int *qcount;
  unsigned long long *qcost;   // int64 two's complement
  unsigned long long *run_end; // ns, 0 = idle
  int *sm_busy;                // per SM (by %smid, < SM_SLOTS): running tasks, hosted workers, then
                               // running critical-path tasks (P::critical)
  long long *trace_buf;
  int use_cp;       // communication prediction in the placement
  int64_t comm_ns;  // predicted cost of one input tile a worker did not write last
  unsigned char *split;  // tensor-core forms: BF16 terms of the panel tiles (nullable)
  int64_t split_tile;    // bytes per panel tile in `split`
  int *lu_piv;           // LU: pivots of GETRF(k) / TSTRF(i, k) at ((k T + i) nb), nb per tile
  double *lu_lw;         // LU: L11 blocks of TSTRF(i, k) at ((k T + i) LU_IB nb)
  HelpSlot *board;       // one help slot per worker
  int split_mode;        // 0 off, 1 the next panel's TRSM and SYRK, 2 every TRSM and SYRK
  int keep_next;         // the finishing worker runs the most urgent task it made ready
};

struct Resolved {
  int prec, lu, nb, T, policy, queue_order, steal, wps, W, max_iter, trace;
  double alpha, eps;
  int64_t cost[4];
  int64_t timeout_ns;
  int64_t hold_task;
  int use_cp;
  int64_t comm_ns;
  int split;
  int keep_next;
};

struct Layout {
  size_t ctrl, trace, zero_begin, qhead, qcount, qcost, run_end, sm_busy, board, slots, zero_end, cnt, owner, bl,
      split, total;
  size_t split_tile;
  int C;
  int64_t ntasks;
};

static size_t sched_smem_bytes(int T, int W) {
  size_t b = align_up((size_t)T * sizeof(ReadyTask), 16);
  b += align_up((size_t)T * 4 * 5, 16);
  b += (size_t)W * 8 * 2;
  return b;
}



static Layout make_layout(int n, const Resolved &r, int W) {
  Layout L;
  const int T = r.T;
  L.ntasks = r.lu ? LuGraph::count(T) : CholGraph::count(T);
  {
    const int64_t ready = r.lu ? LuGraph::max_ready(T) : CholGraph::max_ready(T);
    const int64_t need = (ready + W - 1) / W + 64;
    L.C = (int)std::max<int64_t>(128, (need + 31) / 32 * 32);
  }
  size_t o = 0;
  // the trace comes first so that its offset does not depend on the worker count
  L.ctrl = o; o += align_up(sizeof(Ctrl), 256);
  L.trace = o;
  if (r.trace) o += align_up((size_t)L.ntasks * 32, 256);
  L.zero_begin = o;
  L.qhead = o; o += align_up((size_t)W * 4, 256);
  L.qcount = o; o += align_up((size_t)W * 4, 256);
  L.qcost = o; o += align_up((size_t)W * 8, 256);
  L.run_end = o; o += align_up((size_t)W * 8, 256);
  L.sm_busy = o; o += align_up((size_t)3 * SM_SLOTS * 4, 256);
  L.board = o; o += align_up((size_t)W * sizeof(HelpSlot), 256);
  L.slots = o; o += align_up((size_t)W * L.C * 8, 256);
  L.zero_end = o;
  L.cnt = o; o += align_up((size_t)L.ntasks * 4, 256);
  L.owner = o; o += align_up((size_t)T * T * 4, 256);
  L.bl = o; o += align_up((size_t)L.ntasks * 8, 256);
  // tensor-core forms with 32-aligned tiles up to 256: the panel tiles' BF16 terms, written by
  // their TRSM and bulk-copied by the updates that use them (T (T - 1) / 2 panel tiles)
  L.split = o;
  L.split_tile = 0;
  if ((r.prec == PREC_BF16 || r.prec == PREC_BF16X3) && r.nb % 32 == 0 && r.nb <= 256) {
    L.split_tile = r.prec == PREC_BF16 ? tc::Split<1>::tile_bytes(r.nb) : tc::Split<3>::tile_bytes(r.nb);
    o += align_up((size_t)T * (T - 1) / 2 * L.split_tile, 256);
  }
  L.total = o;
  (void)n;
  return L;
}

// ------------------------------------------------------------------------------------
// device side

__device__ __forceinline__ unsigned long long make_entry(uint32_t key, int64_t tid) {
  return ((unsigned long long)key << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)tid);
}
__device__ __forceinline__ int64_t entry_tid(unsigned long long e) {
  return (int64_t)(0xFFFFFFFFu - (uint32_t)(e & 0xFFFFFFFFull));
}
__device__ __forceinline__ uint32_t prio_key(int64_t bl) {
  int64_t k = bl >> 8;
  if (k > 0xFFFFFFFEll) k = 0xFFFFFFFEll;
  if (k < 0) k = 0;
  return (uint32_t)k + 1u;
}

__device__ __forceinline__ int tile_dim(const FactorArgs &a, int t) {
  return min(a.nb, a.n - t * a.nb);
}
template <class T>
__device__ __forceinline__ T *tile_ptr(const FactorArgs &a, int i, int j) {
  return static_cast<T *>(a.A) + (int64_t)j * a.nb * a.lda + (int64_t)i * a.nb;
}

// Push by a single thread onto queue w, or onto the next queue with a free slot if w is
// full. Returns the queue used, or -1 if every queue is full (cannot happen, see above).
__device__ int push_task(const FactorArgs &a, int w, unsigned long long entry) {
  for (int hop = 0; hop < a.W; ++hop) {
    const int q = (w + hop) % a.W;
    unsigned long long *s = a.slots + (size_t)q * a.C;
    unsigned int idx = atomicAdd(&a.qhead[q], 1u) % (unsigned)a.C;
    for (int probe = 0; probe < a.C; ++probe) {
      if (atomicCAS(&s[idx], 0ull, entry) == 0ull) {
        atomicAdd(&a.qcount[q], 1);
        atomicAdd(&a.ctrl->queued, 1);
        if (hop) atomicAdd(&a.ctrl->spills, 1);
        return q;
      }
      if (++idx == (unsigned)a.C) idx = 0;
    }
  }
  return -1;
}

// Pop the highest-key entry of queue q; called by all lanes of one warp.
__device__ int64_t try_pop(const FactorArgs &a, int q) {
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  if (lane == 0) cnt = ld_volatile(&a.qcount[q]);
  cnt = __shfl_sync(0xffffffffu, cnt, 0);
  if (cnt <= 0) return -1;
  unsigned long long *s = a.slots + (size_t)q * a.C;
  for (int attempt = 0; attempt < 8; ++attempt) {
    unsigned long long best = 0ull;
    int bslot = -1;
    // C is a multiple of 32: batches of four loads per lane are issued before any compare
    for (int i0 = 0; i0 < a.C; i0 += 128) {
      unsigned long long v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + 32 * u + lane;
        v[u] = i < a.C ? ld_volatile(&s[i]) : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (v[u] > best) { best = v[u]; bslot = i0 + 32 * u + lane; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int os = __shfl_xor_sync(0xffffffffu, bslot, o);
      if (ov > best) { best = ov; bslot = os; }
    }
    if (best == 0ull) return -1;
    int ok = 0;
    if (lane == 0) ok = atomicCAS(&s[bslot], best, 0ull) == best;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
      if (lane == 0) {
        atomicSub(&a.qcount[q], 1);
        atomicSub(&a.ctrl->queued, 1);
      }
      return entry_tid(best);
    }
  }
  return -1;
}

__device__ __forceinline__ uint32_t xorshift32(uint32_t x) {
  x ^= x << 13; x ^= x >> 17; x ^= x << 5;
  return x;
}

__device__ __forceinline__ void raise_abort(const FactorArgs &a, int info) {
  atomicCAS(&a.ctrl->info, 0, info);
  atomicExch(&a.ctrl->abort, 1);
}

constexpr int64_t HELP_ID = -3;  // acquire's answer when the worker is to run a unit of a split task

__device__ __forceinline__ unsigned long long help_word(unsigned long long gen, int units, int next) {
  return (gen << 40) | ((unsigned long long)units << 32) | (unsigned long long)(unsigned)next;
}

// Take the next unit of slot h, whose word was last seen as w; -1 if none is left or the slot
// has moved on to another task (generation changed).
__device__ int help_claim(HelpSlot *h, unsigned long long w) {
  const unsigned long long gen = w >> 40;
  while (true) {
    if ((w >> 40) != gen) return -1;
    const int units = (int)((w >> 32) & 0xffull), next = (int)(w & 0xffffffffull);
    if (next >= units) return -1;
    const unsigned long long old = atomicCAS(&h->word, w, w + 1ull);
    if (old == w) return next;
    w = old;
  }
}

// One warp scans the help board for a split task with units left and takes one.
__device__ bool help_scan(const FactorArgs &a, int &slot, int &unit) {
  const int lane = threadIdx.x & 31;
  for (int q0 = 0; q0 < a.W; q0 += 32) {
    const int q = q0 + lane;
    unsigned long long w = 0;
    bool open = false;
    if (q < a.W) {
      w = ld_volatile(&a.board[q].word);
      open = (w >> 40) != 0 && (int)((w >> 32) & 0xffull) > (int)(w & 0xffffffffull);
    }
    unsigned m = __ballot_sync(0xffffffffu, open);
    while (m) {
      const int src = __ffs(m) - 1;
      int got = -1;
      if (lane == src) got = help_claim(&a.board[q], w);
      got = __shfl_sync(0xffffffffu, got, src);
      if (got >= 0) {
        slot = q0 + src;
        unit = got;
        return true;
      }
      m &= m - 1;
    }
  }
  return false;
}

// Get the next task for worker wid (warp 0). Returns -1 when all tasks are done or the run
// was aborted, HELP_ID when the worker is to run unit `hunit` of the task in help slot
// `hslot`. `from` receives the queue the task came from.
__device__ int64_t acquire(const FactorArgs &a, int wid, int smid, uint32_t &rng, int &from, int &hslot,
                           int &hunit) {
  const int lane = threadIdx.x & 31;
  int last_done = -1;
  uint64_t t_last = 0;
  int64_t iters = 0;
  unsigned sleep_ns = 32;
  while (true) {
    int abort_ = 0, done_ = 0;
    unsigned long long now = 0;
    if (lane == 0) {
      abort_ = ld_volatile(&a.ctrl->abort);
      done_ = ld_volatile(&a.ctrl->done);
      now = globaltimer_ns();
    }
    abort_ = __shfl_sync(0xffffffffu, abort_, 0);
    done_ = __shfl_sync(0xffffffffu, done_, 0);
    now = __shfl_sync(0xffffffffu, now, 0);
    if (abort_ || done_ >= a.ntasks) return -1;
    // units of split tasks come first: those tasks are on the critical path
    if (a.split_mode) {
      int open = 0;
      if (lane == 0) open = ld_volatile(&a.ctrl->help_open);
      open = __shfl_sync(0xffffffffu, open, 0);
      if (open > 0 && help_scan(a, hslot, hunit)) return HELP_ID;
    }
    // while the SM's other worker runs a task, take one only if the queued work exceeds what
    // the SMs with no running task can start: two tasks on one SM each run at about half
    // speed, which lengthens the critical path when work is scarce
    int yield_ = 0;
    if (lane == 0 && smid >= 0 && ld_volatile(&a.sm_busy[smid]) > 0)
      yield_ = ld_volatile(&a.ctrl->queued) <= ld_volatile(&a.ctrl->free_sms) ||
               ld_volatile(&a.sm_busy[2 * SM_SLOTS + smid]) > 0;
    yield_ = __shfl_sync(0xffffffffu, yield_, 0);
    int64_t id = yield_ ? -1 : try_pop(a, wid);
    if (id >= 0) { from = wid; return id; }
    if (!yield_ && a.steal && a.W > 1) {
      for (int t = 0; t < 4; ++t) {
        rng = xorshift32(rng);
        int v = (int)(rng % (uint32_t)(a.W - 1));
        if (v >= wid) ++v;
        id = try_pop(a, v);
        if (id >= 0) { from = v; return id; }
      }
    }
    if (done_ != last_done) {
      last_done = done_;
      t_last = now;
      iters = 0;
    } else if (now - t_last > (uint64_t)a.timeout_ns || ++iters > a.iter_limit) {
      if (lane == 0) raise_abort(a, CHOL_INFO_TIMEOUT);
      return -1;
    }
    __nanosleep(sleep_ns);
    sleep_ns = sleep_ns < 2048 ? sleep_ns * 2 : 2048;
  }
}

// Largest entry in queue q (0 if it is empty); all lanes of one warp.
__device__ unsigned long long queue_top(const FactorArgs &a, int q) {
  const int lane = threadIdx.x & 31;
  const unsigned long long *s = a.slots + (size_t)q * a.C;
  unsigned long long best = 0ull;
  for (int i0 = 0; i0 < a.C; i0 += 128) {
    unsigned long long v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + 32 * u + lane;
      v[u] = i < a.C ? ld_volatile(&s[i]) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) best = v[u] > best ? v[u] : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
    best = ov > best ? ov : best;
  }
  return best;
}

// Activate the successors of a finished task and place the ready ones (warp 0). With
// keep_next, the most urgent of the newly ready tasks is not placed when it outranks every
// task queued on this worker: the worker, free at this moment, runs it next (*s_next, else
// -1). Under HEFT's own rule this worker is then the earliest-finishing one for that task,
// since a queue is served in priority order and the task would be taken from it first.
template <class G>
__device__ void complete(const FactorArgs &a, int wid, int smid, const TaskDesc &d, unsigned char *smem_raw,
                         int *s_nready, long long *s_next) {
  const int lane = threadIdx.x & 31;
  const int T = a.T;
  ReadyTask *LR = reinterpret_cast<ReadyTask *>(smem_raw);
  size_t off = align_up((size_t)T * sizeof(ReadyTask), 16);
  PlaceScratch ps;
  int *ints = reinterpret_cast<int *>(smem_raw + off);
  ps.ord_prio = ints;
  ps.ord_aff = ints + T;
  ps.ord_lpt = ints + 2 * T;
  ps.assign = ints + 3 * T;
  ps.trial = ints + 4 * T;
  off += align_up((size_t)T * 4 * 5, 16);
  int64_t *load = reinterpret_cast<int64_t *>(smem_raw + off);
  ps.tload = load + a.W;

  if (lane == 0) {
    int ti, tj;
    G::rw(d, ti, tj);
    *(volatile int *)&a.owner[ti * T + tj] = wid;
    *(volatile unsigned long long *)&a.run_end[wid] = 0ull;
    *s_nready = 0;
    *s_next = -1;
  }
  __syncwarp();
  const int ns = G::nsucc(T, d);
  for (int s = lane; s < ns; s += 32) {
    const int64_t sid = G::succ(T, d, s);
    if (atomicSub(&a.cnt[sid], 1) == 1) {
      const int pos = atomicAdd(s_nready, 1);
      LR[pos].tid = (int)sid;
    }
  }
  __syncwarp();
  __threadfence();
  int m = *(volatile int *)s_nready;
  // keep a task only on an SM that runs nothing else (this worker's own task still counts in
  // sm_busy): next to a running task it would run at half speed, and the co-scheduling rule
  // would not have let this worker take it
  bool alone = true;
  if (a.keep_next && m > 0 && smid >= 0) {
    int b = 0;
    if (lane == 0) b = ld_volatile(&a.sm_busy[smid]);
    alone = __shfl_sync(0xffffffffu, b, 0) <= 1;
  }
  if (m > 0 && a.keep_next && alone) {
    // the most urgent ready task: highest bottom level, then lowest id (warp argmax)
    int bi = -1;
    int64_t bp = 0;
    int bt = 0;
    for (int i = lane; i < m; i += 32) {
      const int t = LR[i].tid;
      const int64_t p = a.bl[t];
      if (bi < 0 || p > bp || (p == bp && t < bt)) { bi = i; bp = p; bt = t; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const int64_t op = __shfl_xor_sync(0xffffffffu, bp, o);
      const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
      if (oi >= 0 && (bi < 0 || op > bp || (op == bp && ot < bt))) { bi = oi; bp = op; bt = ot; }
    }
    const unsigned long long top = queue_top(a, wid);
    if (make_entry(prio_key(bp), bt) > top) {
      if (lane == 0) {
        *s_next = bt;
        LR[bi].tid = LR[m - 1].tid;  // the rest are placed as usual
      }
      __syncwarp();
      m -= 1;
    }
  }
  if (m > 0) {
    for (int i = lane; i < m; i += 32) {
      const TaskDesc sd = G::desc(T, LR[i].tid);
      int ti, tj;
      G::rw(sd, ti, tj);
      LR[i].p = a.cost[sd.kind];
      LR[i].prio = a.queue_order == 0 ? a.bl[LR[i].tid] : 0;
      const int aff = ld_volatile(&a.owner[ti * T + tj]);
      LR[i].aff = aff;
      LR[i].score = aff >= 0 ? (int64_t)min(a.nb, a.n - ti * a.nb) * min(a.nb, a.n - tj * a.nb) * 8 : 0;
      // communication prediction: the workers holding the task's input tiles
      LR[i].comm = a.comm_ns;
      LR[i].own[0] = LR[i].own[1] = LR[i].own[2] = -1;
      if (a.use_cp) {
        int ii[3], jj[3];
        const int nin = G::inputs(sd, ii, jj);
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q < nin) LR[i].own[q] = ld_volatile(&a.owner[ii[q] * T + jj[q]]);
        LR[i].nin = nin;
      } else {
        LR[i].nin = 0;
      }
    }
    __syncwarp();
    const bool model = a.policy == P_HEFT || a.policy == P_DADA;
    if (model) {
      unsigned long long now = 0;
      if (lane == 0) now = globaltimer_ns();
      now = __shfl_sync(0xffffffffu, now, 0);
      for (int w = lane; w < a.W; w += 32) {
        const unsigned long long re = ld_volatile(&a.run_end[w]);
        const int64_t rem = re > now ? (int64_t)(re - now) : 0;
        int64_t q = (int64_t)ld_volatile(&a.qcost[w]);
        load[w] = rem + (q > 0 ? q : 0);
      }
      __syncwarp();
      place<WarpExec>(a.policy, a.alpha, a.dada_max_iter, a.dada_eps, LR, m, load, a.W, ps, a.use_cp != 0);
    } else {
      for (int i = lane; i < m; i += 32) {
        if (a.policy == P_STEAL) {
          ps.assign[i] = wid;
        } else {
          const TaskDesc sd = G::desc(T, LR[i].tid);
          int ti, tj;
          G::rw(sd, ti, tj);
          ps.assign[i] = (ti + tj * T) % a.W;
        }
        ps.ord_prio[i] = i;
      }
    }
    __syncwarp();
    unsigned int seq0 = 0;
    if (a.queue_order == 1) {
      if (lane == 0) seq0 = atomicAdd(&a.ctrl->fifo_seq, (unsigned)m);
      seq0 = __shfl_sync(0xffffffffu, seq0, 0);
    }
    for (int q = lane; q < m; q += 32) {
      const int i = ps.ord_prio[q];
      const uint32_t key = a.queue_order == 1 ? (0xFFFFFFFFu - ((seq0 + (unsigned)q) & 0x7FFFFFFFu))
                                              : prio_key(LR[i].prio);
      const int w = push_task(a, ps.assign[i], make_entry(key, LR[i].tid));
      if (w < 0) raise_abort(a, CHOL_INFO_QUEUE_FULL);
      else atomicAdd(&a.qcost[w], (unsigned long long)LR[i].p);
    }
  }
  __syncwarp();
  if (lane == 0) atomicAdd(&a.ctrl->done, 1);
}

// Tile bodies per precision of the factored matrix.
struct TilesF64 {
  using T = double;
  using Graph = CholGraph;
  static constexpr bool CAN_SPLIT = true;  // TRSM, SYRK and GEMM tasks can be cut into units
  static constexpr int UPD_UNIT = 64;       // SYRK / GEMM units: the update's 64 x 64 blocks
  static constexpr bool SPLIT_TRSM = true, SPLIT_SYRK = true, SPLIT_GEMM = true;
  static constexpr bool SPLIT_EVERY_TRSM = false;
  __device__ static bool critical(int) { return false; }
  static constexpr int SMEM = TILE_SMEM_BYTES;
  static constexpr int MIN_BLOCKS = 2;  // two workers per SM share the FP64 pipe
  __device__ static int potrf(T *G, int64_t ld, int nk, T *s) { return potrf_tile(G, ld, nk, s); }
  __device__ static void trsm(T *B, int64_t ldb, const T *L, int64_t ldl, int mb, int nk, T *s, unsigned char *) {
    trsm_tile(B, ldb, L, ldl, mb, nk, s);
  }
  // rows [r0, r0 + rows) of the panel tile B (a unit of a split TRSM)
  __device__ static void trsm_rows(T *B, int64_t ldb, const T *L, int64_t ldl, int r0, int rows, int nk, T *s,
                                   unsigned char *) {
    trsm_tile(B + r0, ldb, L, ldl, rows, nk, s);
  }
  __device__ static int update(T *C, int64_t ldc, const T *A, int64_t lda, const T *B, int64_t ldb, int M,
                               int N, int K, bool lower, T *s, const unsigned char *, const unsigned char *) {
    update_nt(C, ldc, A, lda, B, ldb, M, N, K, lower, s);
    return 0;
  }
  // one block of a split SYRK, with the body the whole SYRK runs on
  __device__ static void syrk_part(T *C, int64_t ldc, const T *A, int64_t lda, const T *B, int64_t ldb, int M,
                                   int N, int K, bool lower, T *s) {
    update_nt(C, ldc, A, lda, B, ldb, M, N, K, lower, s);
  }
  __device__ static void begin() {}
  __device__ static void end() {}
};
struct TilesF32 {
  using T = float;
  using Graph = CholGraph;
  static constexpr bool CAN_SPLIT = true;
  static constexpr int UPD_UNIT = 128;      // the FFMA update's 128 x 128 blocks
  static constexpr bool SPLIT_TRSM = true, SPLIT_SYRK = true, SPLIT_GEMM = true;
  // a whole FP32 TRSM is its 64-row bands one after another, so every TRSM is handed out band
  // by band (mode 1): same work, and no long TRSM lands on a critical path
  static constexpr bool SPLIT_EVERY_TRSM = true;
  __device__ static bool critical(int) { return false; }
  static_assert(f32::TRSM_BAND_SMEM_BYTES <= (f32::PANEL_SMEM_BYTES > f32::TILE_SMEM_BYTES ? f32::PANEL_SMEM_BYTES
                                                                                         : f32::TILE_SMEM_BYTES),
                "the band TRSM must fit the FP32 bodies' shared memory");
  static constexpr int SMEM = f32::PANEL_SMEM_BYTES > f32::TILE_SMEM_BYTES ? f32::PANEL_SMEM_BYTES
                                                                            : f32::TILE_SMEM_BYTES;
  static constexpr int MIN_BLOCKS = 1;  // the 8x8 register tiles need more than 128 registers
  // POTRF and TRSM lie on the critical path: for tiles up to 256 they run latency-lean bodies
  __device__ static int potrf(T *G, int64_t ld, int nk, T *s) {
    return nk <= f32::PANEL_MAX_N ? f32::potrf_tile_smem(G, ld, nk, s) : f32::potrf_tile(G, ld, nk, s);
  }
  // bands of 64 rows (f32::trsm_band); a split TRSM hands the bands to helpers
  __device__ static void trsm(T *B, int64_t ldb, const T *L, int64_t ldl, int mb, int nk, T *s, unsigned char *) {
    if (nk <= f32::PANEL_MAX_N) {
      for (int r0 = 0; r0 < mb; r0 += f32::BAND_ROWS)
        f32::trsm_band(B + r0, ldb, L, ldl, min(f32::BAND_ROWS, mb - r0), nk, s);
    } else {
      f32::trsm_tile(B, ldb, L, ldl, mb, nk, s);
    }
  }
  __device__ static void trsm_rows(T *B, int64_t ldb, const T *L, int64_t ldl, int r0, int rows, int nk, T *s,
                                   unsigned char *) {
    if (nk <= f32::PANEL_MAX_N) f32::trsm_band(B + r0, ldb, L, ldl, rows, nk, s);
    else f32::trsm_tile(B + r0, ldb, L, ldl, rows, nk, s);
  }
  __device__ static int update(T *C, int64_t ldc, const T *A, int64_t lda, const T *B, int64_t ldb, int M,
                               int N, int K, bool lower, T *s, const unsigned char *, const unsigned char *) {
    f32::update_nt(C, ldc, A, lda, B, ldb, M, N, K, lower, s);
    return 0;
  }
  // one block of a split SYRK: FFMA, also in the three-term tensor-core form (whose SYRKs run
  // on this body)
  __device__ static void syrk_part(T *C, int64_t ldc, const T *A, int64_t lda, const T *B, int64_t ldb, int M,
                                   int N, int K, bool lower, T *s) {
    f32::update_nt(C, ldc, A, lda, B, ldb, M, N, K, lower, s);
  }
  __device__ static void begin() {}
  __device__ static void end() {}
};
// FP32 storage and FP32 POTRF/TRSM; GEMM (and, with one term, SYRK) updates on the tensor
// cores with NTERM BF16 operand terms. The accumulators (all 512 TMEM columns) are held by the
// worker for the whole launch.
template <int NTERM>
struct TilesTC : TilesF32 {
  // split units: TRSM bands, and the SYRKs that run on the FFMA body (three-term form); the
  // tensor-core updates are one MMA tile each
  static constexpr bool SPLIT_TRSM = true, SPLIT_SYRK = NTERM > 1, SPLIT_GEMM = false;
  static constexpr int EMIT_OFF = (f32::TRSM_BAND_SMEM_BYTES + 127) / 128 * 128;
  static constexpr int SMEM0 = tc::Cfg<NTERM>::SMEM > TilesF32::SMEM ? tc::Cfg<NTERM>::SMEM : TilesF32::SMEM;
  static constexpr int SMEM = SMEM0 > EMIT_OFF + tc::SplitEmitBand<NTERM>::BYTES ? SMEM0
                                                                                 : EMIT_OFF + tc::SplitEmitBand<NTERM>::BYTES;
  static_assert(EMIT_OFF + tc::SplitEmitBand<NTERM>::BYTES <= SMEM, "TRSM split buffers must fit");
  // one worker per SM: a second one would wait in tcgen05.alloc for columns the first holds
  static_assert(2 * SMEM > 228 * 1024, "tensor-core workers must not share an SM");
  __device__ static tc::State &state() {
    __shared__ tc::State st;
    return st;
  }
  // with a side buffer the TRSM also writes the tile's BF16 terms, and the updates bulk-copy
  // them; without one the updates split their FP32 operands themselves
  __device__ static void trsm(T *B, int64_t ldb, const T *L, int64_t ldl, int mb, int nk, T *s,
                              unsigned char *split) {
    if (split && nk <= f32::PANEL_MAX_N) {
      for (int r0 = 0; r0 < mb; r0 += f32::BAND_ROWS) trsm_rows(B, ldb, L, ldl, r0, min(f32::BAND_ROWS, mb - r0), nk, s, split);
    } else {
      TilesF32::trsm(B, ldb, L, ldl, mb, nk, s, nullptr);
    }
  }
  // one band of 64 rows, its BF16 terms staged past the band body's shared memory
  __device__ static void trsm_rows(T *B, int64_t ldb, const T *L, int64_t ldl, int r0, int rows, int nk, T *s,
                                   unsigned char *split) {
    if (split && nk <= f32::PANEL_MAX_N)
      f32::trsm_band(B + r0, ldb, L, ldl, rows, nk, s,
                     tc::SplitEmitBand<NTERM>{split, reinterpret_cast<unsigned char *>(s) + EMIT_OFF, r0});
    else
      TilesF32::trsm_rows(B, ldb, L, ldl, r0, rows, nk, s, nullptr);
  }
  // SYRK updates (C -= A A^T on a diagonal tile, rows of A that lie close together in the
  // matrix) add products that mostly share one sign, and the errors of the tensor cores' FP32
  // accumulation then pile up in one direction: a bias in the Schur complements that the
  // refinement removes only slowly. Measured at n = 16384, kappa = 1e6 (four matrices): with
  // the SYRKs on the tensor cores it contracts ~50x per step and needs five steps to 1e-14;
  // with them in FFMA (round to nearest) ~80x and four steps for every matrix. The multi-term
  // form therefore runs its SYRKs on the FFMA body and only the GEMMs, whose products take
  // both signs, on the tensor cores. (Recomputing only the diagonal entries in FFMA does not
  // help; keeping each tile's last SYRK on the tensor cores saves 3 ms of factor time but
  // leaves half of those matrices just above 1e-14 after four steps.)
  __device__ static int update(T *C, int64_t ldc, const T *A, int64_t lda, const T *B, int64_t ldb, int M,
                               int N, int K, bool lower, T *s, const unsigned char *sa, const unsigned char *sb) {
    if (NTERM > 1 && lower) return TilesF32::update(C, ldc, A, lda, B, ldb, M, N, K, true, s, sa, sb);
    unsigned char *sm = reinterpret_cast<unsigned char *>(s);
    if (sa && sb) return tc::update_nt_split<NTERM>(C, ldc, sa, sb, M, N, K, lower, sm, state());
    return tc::update_nt<NTERM>(C, ldc, A, lda, B, ldb, M, N, K, lower, sm, state());
  }
  __device__ static void begin() { tc::begin(state()); }
  __device__ static void end() { tc::end(state()); }
};

// BF16 terms of panel tile (i, k), i > k, in the side buffer (nullptr without one)
__device__ __forceinline__ unsigned char *split_ptr(const FactorArgs &a, int i, int k) {
  return a.split ? a.split + ((int64_t)i * (i - 1) / 2 + k) * a.split_tile : nullptr;
}

// LU with incremental pivoting, FP64 (tile bodies in tiles_lu.cuh).
struct LuF64 {
  using T = double;
  using Graph = LuGraph;
  static constexpr bool CAN_SPLIT = false;  // (the LU graph has its own runner)
  static constexpr int UPD_UNIT = 64;
  static constexpr bool SPLIT_TRSM = false, SPLIT_SYRK = false, SPLIT_GEMM = false;
  static constexpr bool SPLIT_EVERY_TRSM = false;
  // the panel factorizations form the graph's longest chain (TSTRF(i, k) -> TSTRF(i + 1, k),
  // and on to step k + 1): while one runs, its SM's other worker takes no new task, so the
  // chain gets the whole FP64 pipe instead of half of it and no dependent FP64 operation
  // waits behind a neighbour's update
  __device__ static bool critical(int kind) { return kind == K_GETRF || kind == K_TSTRF; }
  static constexpr int SMEM = LU_SMEM_BYTES;
  static constexpr int MIN_BLOCKS = 2;
  __device__ static void begin() {}
  __device__ static void end() {}
};

// Run one tile task with the whole block. Returns 0 or a 1-based failing global column.
template <class P>
struct Runner {
  __device__ static int run(const FactorArgs &a, const TaskDesc &d, typename P::T *smem, int wid, bool starving);
  __device__ static void unit(const FactorArgs &a, const TaskDesc &d, int u, typename P::T *smem);
};

// Split tasks (FP64 bodies): a TRSM is cut into bands of 64 rows of the panel tile (the rows
// of X L^T = B are independent), a SYRK into the 64 x 64 blocks of the lower triangle of its
// diagonal tile, a GEMM into the 64 x 64 blocks of its tile. Every element is computed by the
// same operations in the same order as in the whole-task bodies, so the factor is bitwise the
// same with and without splitting.
constexpr int SPLIT_ROWS = 64;  // rows of a TRSM unit (FP32 updates use 128 x 128 units)

template <class P>
__device__ __forceinline__ int split_units(const FactorArgs &a, const TaskDesc &d) {
  if (d.kind == K_TRSM) return (tile_dim(a, d.i) + SPLIT_ROWS - 1) / SPLIT_ROWS;
  const int nbi = (tile_dim(a, d.i) + P::UPD_UNIT - 1) / P::UPD_UNIT;
  if (d.kind == K_SYRK) return nbi * (nbi + 1) / 2;
  return nbi * ((tile_dim(a, d.j) + P::UPD_UNIT - 1) / P::UPD_UNIT);
}

// Mode 1: the TRSMs of tile rows k + 1 and k + 2 and the SYRK of tile row k + 1 -- the chain
// POTRF(k) -> TRSM(k+1, k) -> SYRK(k+1, k) -> POTRF(k+1), and the path POTRF(k) -> TRSM(k+2, k)
// -> GEMM(k+2, k+1, k) -> TRSM(k+2, k+1) beside it, which is as long once the chain's own tasks
// are split -- and any TRSM, SYRK or GEMM that starts while SMs run no task and no queued task
// is left for them (`starving`: the end of the factor, or small matrices). Mode 2: every TRSM,
// SYRK and GEMM.
template <class P>
__device__ __forceinline__ bool should_split(const FactorArgs &a, const TaskDesc &d, bool starving) {
  if (!a.split_mode || d.kind == K_POTRF) return false;
  if ((d.kind == K_TRSM && !P::SPLIT_TRSM) || (d.kind == K_SYRK && !P::SPLIT_SYRK) ||
      (d.kind == K_GEMM && !P::SPLIT_GEMM))
    return false;
  if (split_units<P>(a, d) < 2 || split_units<P>(a, d) > 255) return false;
  if (a.split_mode == 2) return true;
  if ((d.kind == K_TRSM && (d.i <= d.k + 2 || P::SPLIT_EVERY_TRSM)) || (d.kind == K_SYRK && d.i == d.k + 1))
    return true;
  return starving;
}

template <class P>
__device__ __noinline__ void Runner<P>::unit(const FactorArgs &a, const TaskDesc &d, int u, typename P::T *smem) {
  if constexpr (P::CAN_SPLIT) {
    using T = typename P::T;
    const int mi = tile_dim(a, d.i), nk = tile_dim(a, d.k);
    constexpr int U = P::UPD_UNIT;
    if (d.kind == K_TRSM) {
      const int r0 = SPLIT_ROWS * u;
      P::trsm_rows(tile_ptr<T>(a, d.i, d.k), a.lda, tile_ptr<T>(a, d.k, d.k), a.lda, r0, min(SPLIT_ROWS, mi - r0),
                   nk, smem, split_ptr(a, d.i, d.k));
    } else if (d.kind == K_GEMM) {
      const int mj = tile_dim(a, d.j), nbj = (mj + U - 1) / U;
      const int r0 = U * (u / nbj), c0 = U * (u % nbj);
      P::update(tile_ptr<T>(a, d.i, d.j) + (int64_t)c0 * a.lda + r0, a.lda, tile_ptr<T>(a, d.i, d.k) + r0, a.lda,
                tile_ptr<T>(a, d.j, d.k) + c0, a.lda, min(U, mi - r0), min(U, mj - c0), nk, false, smem, nullptr,
                nullptr);
    } else {
      int bm = (int)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
      while (bm * (bm + 1) / 2 > u) --bm;
      while ((bm + 1) * (bm + 2) / 2 <= u) ++bm;
      const int bn = u - bm * (bm + 1) / 2;
      const int r0 = U * bm, c0 = U * bn;
      const T *A = tile_ptr<T>(a, d.i, d.k);
      P::syrk_part(tile_ptr<T>(a, d.i, d.i) + (int64_t)c0 * a.lda + r0, a.lda, A + r0, a.lda, A + c0, a.lda,
                   min(U, mi - r0), min(U, mi - c0), nk, bm == bn, smem);
    }
  }
}

// Run task d as units: publish it on this worker's help slot, take units until none is
// left, then wait (bounded) for the units other workers took. Returns 0 or CHOL_INFO_TIMEOUT.
template <class P>
__device__ __noinline__ int run_split(const FactorArgs &a, const TaskDesc &d, typename P::T *smem, int wid) {
  __shared__ int s_unit;
  HelpSlot *h = a.board + wid;
  const int units = split_units<P>(a, d);
  if (threadIdx.x == 0) {
    const unsigned long long gen = (ld_volatile(&h->word) >> 40) + 1ull;
    h->kind = d.kind;
    h->i = d.i;
    h->j = d.j;
    h->k = d.k;
    h->done = 0;
    __threadfence();
    atomicExch(&h->word, help_word(gen, units, 0));
    atomicAdd(&a.ctrl->help_open, 1);
  }
  while (true) {
    if (threadIdx.x == 0) {
      const unsigned long long old = atomicAdd(&h->word, 1ull);
      const int next = (int)(old & 0xffffffffull);
      s_unit = next < units ? next : -1;
    }
    __syncthreads();
    const int u = s_unit;
    __syncthreads();
    if (u < 0) break;
    Runner<P>::unit(a, d, u, smem);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&h->done, 1);
  }
  if (threadIdx.x == 0) {
    atomicSub(&a.ctrl->help_open, 1);
    // the units other workers took: they run tile bodies only, with no waits
    int fail = 0;
    const uint64_t t0 = globaltimer_ns();
    int64_t spins = 0;
    unsigned slp = 32;
    while (ld_volatile(&h->done) < units) {
      if (ld_volatile(&a.ctrl->abort)) break;
      if (globaltimer_ns() - t0 > (uint64_t)a.timeout_ns || ++spins > a.iter_limit) {
        fail = CHOL_INFO_TIMEOUT;
        break;
      }
      __nanosleep(slp);
      slp = slp < 256 ? slp * 2 : 256;
    }
    __threadfence();
    s_unit = fail;
  }
  __syncthreads();
  return s_unit;
}

template <class P>
__device__ int Runner<P>::run(const FactorArgs &a, const TaskDesc &d, typename P::T *smem, int wid,
                              bool starving) {
  using T = typename P::T;
  if constexpr (P::CAN_SPLIT) {
    if (should_split<P>(a, d, starving)) return run_split<P>(a, d, smem, wid);
  }
  switch (d.kind) {
    case K_POTRF: {
      const int f = P::potrf(tile_ptr<T>(a, d.k, d.k), a.lda, tile_dim(a, d.k), smem);
      return f ? d.k * a.nb + f : 0;
    }
    case K_TRSM:
      P::trsm(tile_ptr<T>(a, d.i, d.k), a.lda, tile_ptr<T>(a, d.k, d.k), a.lda, tile_dim(a, d.i),
              tile_dim(a, d.k), smem, split_ptr(a, d.i, d.k));
      return 0;
    case K_SYRK:  // a nonzero return is an expired wait inside the tile update
      return P::update(tile_ptr<T>(a, d.i, d.i), a.lda, tile_ptr<T>(a, d.i, d.k), a.lda,
                       tile_ptr<T>(a, d.i, d.k), a.lda, tile_dim(a, d.i), tile_dim(a, d.i), tile_dim(a, d.k),
                       true, smem, split_ptr(a, d.i, d.k), split_ptr(a, d.i, d.k))
                 ? CHOL_INFO_TIMEOUT
                 : 0;
    default:
      return P::update(tile_ptr<T>(a, d.i, d.j), a.lda, tile_ptr<T>(a, d.i, d.k), a.lda,
                       tile_ptr<T>(a, d.j, d.k), a.lda, tile_dim(a, d.i), tile_dim(a, d.j), tile_dim(a, d.k),
                       false, smem, split_ptr(a, d.i, d.k), split_ptr(a, d.j, d.k))
                 ? CHOL_INFO_TIMEOUT
                 : 0;
  }
}

__device__ __forceinline__ int *lu_piv_ptr(const FactorArgs &a, int i, int k) {
  return a.lu_piv + ((int64_t)k * a.T + i) * a.nb;
}
__device__ __forceinline__ double *lu_lw_ptr(const FactorArgs &a, int i, int k) {
  return a.lu_lw + ((int64_t)k * a.T + i) * LU_IB * a.nb;
}

template <>
__device__ int Runner<LuF64>::run(const FactorArgs &a, const TaskDesc &d, double *smem, int, bool) {
  const int64_t ld = a.lda;
  switch (d.kind) {
    case K_GETRF: {
      const int f = lu_getrf_tile(tile_ptr<double>(a, d.k, d.k), ld, tile_dim(a, d.k), lu_piv_ptr(a, d.k, d.k), smem);
      return f ? d.k * a.nb + f : 0;
    }
    case K_GESSM:
      lu_gessm_tile(tile_ptr<double>(a, d.k, d.j), ld, tile_dim(a, d.k), tile_dim(a, d.j),
                    tile_ptr<double>(a, d.k, d.k), lu_piv_ptr(a, d.k, d.k), smem);
      return 0;
    case K_TSTRF: {
      const int f = lu_tstrf_tile(tile_ptr<double>(a, d.k, d.k), tile_ptr<double>(a, d.i, d.k), ld, tile_dim(a, d.k),
                                  tile_dim(a, d.i), lu_piv_ptr(a, d.i, d.k), lu_lw_ptr(a, d.i, d.k), smem);
      return f ? d.k * a.nb + f : 0;
    }
    default:
      lu_ssssm_tile(tile_ptr<double>(a, d.k, d.j), tile_ptr<double>(a, d.i, d.j), ld, tile_ptr<double>(a, d.i, d.k),
                    tile_dim(a, d.k), tile_dim(a, d.i), tile_dim(a, d.j), lu_piv_ptr(a, d.i, d.k),
                    lu_lw_ptr(a, d.i, d.k), smem);
      return 0;
  }
}

template <class P>
__global__ void __launch_bounds__(NT, P::MIN_BLOCKS) factor_kernel(const __grid_constant__ FactorArgs a) {
  using G = typename P::Graph;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typename P::T *smem = reinterpret_cast<typename P::T *>(smem_raw);
  __shared__ long long s_id;
  __shared__ int s_from;
  __shared__ int s_nready;
  __shared__ int s_hslot, s_hunit;
  __shared__ long long s_next;
  __shared__ int s_starving;
  const int wid = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t rng = 0x9E3779B9u ^ ((uint32_t)wid * 0x85EBCA6Bu + 1u);
  int smid = -1;
  {
    unsigned v;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
    if (a.W > 1 && v < (unsigned)SM_SLOTS) smid = (int)v;
  }
  if (smid >= 0 && threadIdx.x == 0 && atomicAdd(&a.sm_busy[SM_SLOTS + smid], 1) == 0)
    atomicAdd(&a.ctrl->free_sms, 1);
  P::begin();
  if (wid == 0 && threadIdx.x == 0) {
    const uint32_t key = a.queue_order == 1 ? 0xFFFFFFFFu : prio_key(a.bl[0]);
    atomicAdd(&a.qcost[0], (unsigned long long)a.cost[G::KIND0]);
    if (push_task(a, 0, make_entry(key, 0)) < 0) raise_abort(a, CHOL_INFO_QUEUE_FULL);
  }
  if (threadIdx.x == 0) s_next = -1;
  __syncthreads();
  while (true) {
    if (warp == 0) {
      int from = -1, hs = -1, hu = -1;
      const long long kept = s_next;  // a task this worker made ready and keeps (not queued)
      int64_t id;
      if (kept >= 0) {
        id = ld_volatile(&a.ctrl->abort) ? -1 : kept;
        from = wid;
      } else {
        id = acquire(a, wid, smid, rng, from, hs, hu);
      }
      if (id >= 0 && lane == 0 && smid >= 0 && atomicAdd(&a.sm_busy[smid], 1) == 0)
        atomicSub(&a.ctrl->free_sms, 1);
      if (id >= 0 && lane == 0) {
        const TaskDesc d = G::desc(a.T, id);
        if (smid >= 0 && P::critical(d.kind)) atomicAdd(&a.sm_busy[2 * SM_SLOTS + smid], 1);
        const int64_t c = a.cost[d.kind];
        if (kept < 0) atomicAdd(&a.qcost[from], (unsigned long long)(-c));
        *(volatile unsigned long long *)&a.run_end[wid] = globaltimer_ns() + (uint64_t)c;
      }
      if (lane == 0) {
        s_id = id;
        s_from = from;
        s_hslot = hs;
        s_hunit = hu;
        s_starving = a.split_mode && id >= 0 && ld_volatile(&a.ctrl->free_sms) > ld_volatile(&a.ctrl->queued);
      }
    }
    __syncthreads();
    const int64_t id = s_id;
    if (id == HELP_ID) {
      // one unit of another worker's split task
      __threadfence();
      const HelpSlot *h = a.board + s_hslot;
      TaskDesc hd;
      hd.kind = ld_volatile(&h->kind);
      hd.i = ld_volatile(&h->i);
      hd.j = ld_volatile(&h->j);
      hd.k = ld_volatile(&h->k);
      if (threadIdx.x == 0) {
        // busy for about one unit's share of the task: the placement's load model must not
        // take a helping worker for an idle one
        const int units = (int)((ld_volatile(&h->word) >> 32) & 0xffull);
        const uint64_t c = (uint64_t)a.cost[hd.kind] / (uint64_t)(units > 0 ? units : 1);
        *(volatile unsigned long long *)&a.run_end[wid] = globaltimer_ns() + c;
      }
      Runner<P>::unit(a, hd, s_hunit, smem);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        *(volatile unsigned long long *)&a.run_end[wid] = 0ull;
        atomicAdd(&a.board[s_hslot].done, 1);
      }
      continue;
    }
    if (id < 0) break;
    __threadfence();
    const TaskDesc d = G::desc(a.T, id);
    unsigned long long t0 = 0;
    if (a.trace && threadIdx.x == 0) t0 = globaltimer_ns();
    const int fail = Runner<P>::run(a, d, smem, wid, s_starving != 0);
    __threadfence();
    __syncthreads();
    if (warp == 0) {
      // the end time is taken before the successors are activated, so a successor's start
      // time is never earlier than it
      unsigned long long t1 = 0;
      if (a.trace && lane == 0) t1 = globaltimer_ns();
      if (fail) {
        if (lane == 0) {
          raise_abort(a, fail);
          s_next = -1;
        }
      } else {
        complete<G>(a, wid, smid, d, smem_raw, &s_nready, &s_next);
      }
      if (lane == 0 && smid >= 0 && P::critical(d.kind)) atomicSub(&a.sm_busy[2 * SM_SLOTS + smid], 1);
      if (lane == 0 && smid >= 0 && atomicSub(&a.sm_busy[smid], 1) == 1) atomicAdd(&a.ctrl->free_sms, 1);
      if (a.trace && lane == 0) {
        long long *tr = a.trace_buf + 4 * id;
        tr[0] = wid;
        tr[1] = s_from;
        tr[2] = (long long)t0;
        tr[3] = (long long)t1;
      }
    }
  }
  P::end();
}

template <class G>
__global__ void init_kernel(int T, int64_t ntasks, int *cnt, int *owner, int64_t hold_task) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < ntasks; id += stride)
    cnt[id] = G::initial(G::desc(T, id)) + (id == hold_task ? 1 : 0);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)T * T; t += stride)
    owner[t] = -1;
}

// Bottom levels as order-preserving unsigned keys, so the per-step maxima can be taken with
// shared-memory atomicMax; BL_ZERO is the key of 0, the start of every maximum (a task
// without successors has bottom level = its cost).
constexpr unsigned long long BL_SIGN = 0x8000000000000000ull;
constexpr unsigned long long BL_ZERO = BL_SIGN;
__device__ __forceinline__ unsigned long long bl_key(int64_t v) { return (unsigned long long)v ^ BL_SIGN; }
__device__ __forceinline__ int64_t bl_val(unsigned long long k) { return (int64_t)(k ^ BL_SIGN); }

__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Bottom levels of the Cholesky graph by steps k = T-1 .. 0 (one block). Each SYRK(i, k) and
// GEMM(i, j, k) has its one successor in step k+1 (already known); one warp takes tile row
// i of the step (SYRK(i, k) and the GEMM(i, j, k), a lane each) and folds the values into
// the maxima, in shared memory, of the TRSMs they follow: TRSM(i, k) precedes SYRK(i, k),
// GEMM(i, *, k) and GEMM(*, i, k). The TRSMs then fold theirs into the POTRF's maximum and
// POTRF(k) closes the step. tmax[b][t] holds TRSM(k+1+t, k)'s maximum and tmax[b][m] the
// POTRF's; the two buffers alternate with the parity of k and the next step's buffer is
// cleared behind the last barrier of this one. The row maxima are reduced across the warp
// first, so no two lanes of a warp update one entry at once.
__global__ void __launch_bounds__(1024) bottom_level_kernel(int T, int64_t c0, int64_t c1, int64_t c2,
                                                            int64_t c3, int64_t *bl) {
  __shared__ unsigned long long tmax[2][1025];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int t = threadIdx.x; t < 2 * 1025; t += blockDim.x) (&tmax[0][0])[t] = BL_ZERO;
  __syncthreads();
  for (int k = T - 1; k >= 0; --k) {
    unsigned long long *mx = tmax[k & 1];
    const int64_t base = step_offset(T, k);
    const int m = T - 1 - k;
    for (int ip = warp; ip < m; ip += nwarps) {
      const int i = k + 1 + ip;
      unsigned long long rowkey = BL_ZERO;
      for (int t0 = 0; t0 <= ip; t0 += 32) {
        const int t = t0 + lane;
        if (t <= ip) {
          int64_t id, sid, c;
          if (t == 0) {  // SYRK(i, k) -> POTRF(i) or SYRK(i, k+1)
            id = task_id(T, K_SYRK, i, i, k);
            sid = ip == 0 ? task_id(T, K_POTRF, i, i, i) : task_id(T, K_SYRK, i, i, k + 1);
            c = c2;
          } else {  // GEMM(i, j, k) -> TRSM(i, j) or GEMM(i, j, k+1)
            const int j = k + t;
            id = task_id(T, K_GEMM, i, j, k);
            sid = j == k + 1 ? task_id(T, K_TRSM, i, j, j) : task_id(T, K_GEMM, i, j, k + 1);
            c = c3;
          }
          const int64_t sv = bl[sid];
          const int64_t v = c + (sv > 0 ? sv : 0);
          bl[id] = v;
          const unsigned long long key = bl_key(v);
          rowkey = key > rowkey ? key : rowkey;
          if (t > 0) atomicMax(&mx[t - 1], key);  // GEMM(i, j, k) also follows TRSM(j, k)
        }
      }
      rowkey = warp_max_key(rowkey);
      if (lane == 0) atomicMax(&mx[ip], rowkey);
    }
    __syncthreads();
    for (int t0 = warp * 32; t0 < m; t0 += blockDim.x) {
      const int t = t0 + lane;
      unsigned long long key = BL_ZERO;
      if (t < m) {
        const int64_t v = c1 + bl_val(mx[t]);
        bl[base + 1 + t] = v;
        key = bl_key(v);
      }
      key = warp_max_key(key);
      if (lane == 0) atomicMax(&mx[m], key);
    }
    __syncthreads();
    if (threadIdx.x == 0) bl[base] = c0 + bl_val(mx[m]);
    unsigned long long *nx = tmax[(k - 1) & 1];
    for (int t = threadIdx.x; t <= m; t += blockDim.x) nx[t] = BL_ZERO;
    __syncthreads();
  }
}

// Bottom levels of the LU graph by steps k = T-1 .. 0 (one block). In step k the SSSSMs of
// tile column j form a chain down the rows (SSSSM(i, j, k) precedes SSSSM(i+1, j, k) and the
// next writer of tile (i, j) in step k+1), so one thread per column walks i = T-1 .. k+1:
// S(i) = c3 + max(0, next writer, S(i+1)); it then writes GESSM(k, j) (successor SSSSM(k+1,
// j, k)). Each S(i) goes into row i's maximum (reduced across the warp first: the lanes of a
// warp walk the same row together) and GESSM(k, j) into GETRF(k)'s. The TSTRF chain,
// TSTRF(i, k) = c2 + max(row i's maximum, TSTRF(i+1, k)), and GETRF(k) = c0 + max(GESSMs,
// TSTRF(k+1, k)) are then taken by one thread from shared memory. rmax[b][t] holds row
// k+1+t's maximum, rmax[b][m] GETRF(k)'s; the buffers alternate with the parity of k.
__global__ void __launch_bounds__(1024) lu_bottom_level_kernel(int T, int64_t c0, int64_t c1, int64_t c2,
                                                               int64_t c3, int64_t *bl) {
  __shared__ unsigned long long rmax[2][1025];
  const int lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < 2 * 1025; t += blockDim.x) (&rmax[0][0])[t] = BL_ZERO;
  __syncthreads();
  for (int k = T - 1; k >= 0; --k) {
    unsigned long long *mx = rmax[k & 1];
    const int m = T - 1 - k;
    // warps with at least one column walk the rows together (m <= 1023 < 1024 threads)
    if ((threadIdx.x & ~31) < m) {
      const int jj = threadIdx.x;
      const bool act = jj < m;
      const int j = k + 1 + jj;
      int64_t S = 0;
      // the next writer of tile (i, j) is in step k+1: its value is loaded one row ahead
      int64_t nv_next = act ? bl[LuGraph::succ(T, TaskDesc{K_SSSSM, T - 1, j, k}, 0)] : 0;
      for (int i = T - 1; i > k; --i) {
        unsigned long long key = 0;  // below every key: no contribution
        if (act) {
          const int64_t nv = nv_next;
          if (i - 1 > k) nv_next = bl[LuGraph::succ(T, TaskDesc{K_SSSSM, i - 1, j, k}, 0)];
          int64_t best = nv > 0 ? nv : 0;
          if (i + 1 < T && S > best) best = S;
          S = c3 + best;
          bl[LuGraph::id(T, K_SSSSM, i, j, k)] = S;
          key = bl_key(S);
        }
        key = warp_max_key(key);
        if (lane == 0) atomicMax(&mx[i - k - 1], key);
      }
      unsigned long long gkey = 0;
      if (act) {
        const int64_t g = c1 + (S > 0 ? S : 0);
        bl[LuGraph::id(T, K_GESSM, k, j, k)] = g;
        gkey = bl_key(g);
      }
      gkey = warp_max_key(gkey);
      if (lane == 0) atomicMax(&mx[m], gkey);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t R = 0;
      for (int i = T - 1; i > k; --i) {
        int64_t best = bl_val(mx[i - k - 1]);
        if (i + 1 < T && R > best) best = R;
        R = c2 + best;
        bl[LuGraph::id(T, K_TSTRF, i, k, k)] = R;
      }
      int64_t best = bl_val(mx[m]);
      if (m > 0 && R > best) best = R;
      bl[LuGraph::id(T, K_GETRF, k, k, k)] = c0 + best;
    }
    unsigned long long *nx = rmax[(k - 1) & 1];
    for (int t = threadIdx.x; t <= m; t += blockDim.x) nx[t] = BL_ZERO;
    __syncthreads();
  }
}

chol_status bottom_levels_device(bool lu, int T, const int64_t *cost, int64_t *dBl, cudaStream_t s) {
  if (T < 1 || T > 1024) return CHOL_ERR_INVALID_ARG;
  if (lu) lu_bottom_level_kernel<<<1, 1024, 0, s>>>(T, cost[0], cost[1], cost[2], cost[3], dBl);
  else bottom_level_kernel<<<1, 1024, 0, s>>>(T, cost[0], cost[1], cost[2], cost[3], dBl);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

__global__ void copy_info_kernel(const Ctrl *ctrl, int *dInfo) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dInfo = ctrl->info;
}

// ------------------------------------------------------------------------------------
// host side

static size_t tile_smem_bytes(int prec) {
  switch (prec) {
    case PREC_F64: return TilesF64::SMEM;
    case PREC_LU_F64: return LuF64::SMEM;
    case PREC_F32: return TilesF32::SMEM;
    case PREC_BF16: return TilesTC<1>::SMEM;
    default: return TilesTC<3>::SMEM;
  }
}

static size_t factor_smem_bytes(int prec, int T, int W) { return std::max(tile_smem_bytes(prec), sched_smem_bytes(T, W)); }

// dynamic shared memory the factor kernel of each precision may request
static int smem_limit(int prec) {
  switch (prec) {
    case PREC_F64: return 96 * 1024;
    case PREC_LU_F64: return 112 * 1024;
    default: return 200 * 1024;
  }
}

static const void *kernel_for(int prec) {
  switch (prec) {
    case PREC_F64: return (const void *)factor_kernel<TilesF64>;
    case PREC_LU_F64: return (const void *)factor_kernel<LuF64>;
    case PREC_F32: return (const void *)factor_kernel<TilesF32>;
    case PREC_BF16: return (const void *)factor_kernel<TilesTC<1>>;
    default: return (const void *)factor_kernel<TilesTC<3>>;
  }
}

static bool resolve(int n, const chol_opts *opts, Resolved &r, int prec = PREC_F64) {
  chol_opts o;
  chol_opts_default(&o);
  if (opts) o = *opts;
  r.prec = prec;
  r.lu = prec == PREC_LU_F64 ? 1 : 0;
  // automatic tile: FP64 factors of mid-size matrices are bound by the POTRF -> TRSM -> SYRK
  // chain of each step, whose tile bodies run on one SM, so a smaller tile shortens it
  // (fraction of the FP64 peak at 128 vs 256: 0.76 vs 0.41 at n = 8192, 0.94 vs 0.84 at
  // 16384, 0.971 vs 0.964 at 32768); larger orders keep 256 (fewer tasks, T <= 1024)
  r.nb = o.nb > 0 ? o.nb : (n <= 32768 ? 128 : 256);
  if (r.nb < 16 || r.nb > 1024) return false;
  if (r.lu && r.nb > LU_NB_MAX) return false;
  r.T = n > 0 ? (n + r.nb - 1) / r.nb : 1;
  if (r.T > 1024) return false;
  if (o.policy < 0 || o.policy > 3) return false;
  r.policy = o.policy;
  if (!(o.alpha >= 0.0 && o.alpha <= 1.0)) return false;
  r.alpha = o.alpha;
  r.steal = o.steal ? 1 : 0;
  r.wps = o.workers_per_sm > 0 ? o.workers_per_sm : 2;
  if (r.wps > 2) return false;
  r.W = o.num_workers;
  if (r.W < 0 || r.W > 1024) return false;
  r.queue_order = o.queue_order ? 1 : 0;
  r.max_iter = o.dada_max_iter > 0 ? o.dada_max_iter : 16;
  r.eps = o.dada_eps > 0.0 ? o.dada_eps : 0.01;
  const double nb = (double)r.nb;
  // predicted rate per SM of each kind (GFLOP/s = flop per ns), from the tile bodies' measured
  // times: FP64 DFMA bodies ~7.5 for every Cholesky kind; the FP32 forms' POTRF and TRSM are dependent
  // chains (~40 and ~60), FFMA SYRK ~140, FFMA GEMM ~250, tensor-core updates ~1000 (one BF16
  // term, SYRK and GEMM) and ~730 (three terms, GEMM only: its SYRKs run on FFMA). Equal
  // predictions for TRSM and SYRK would tie the bottom levels of the critical TRSM(k+1, k) and
  // the previous step's SYRK(k+1, k-1), and the tie would go to the older task.
  double per_sm[4];
  if (prec == PREC_F64) {
    for (int k = 0; k < 4; ++k) per_sm[k] = 7.5;
  } else if (prec == PREC_LU_F64) {
    // GETRF / GESSM / TSTRF / SSSSM at tile 128, measured per task in a trace of the n = 8192
    // factor: the panel factorizations are dependent chains, their transformations less so
    per_sm[0] = 3.4;
    per_sm[1] = 6.6;
    per_sm[2] = 4.2;
    per_sm[3] = 7.0;
  } else {
    per_sm[0] = 40.0;
    per_sm[1] = 60.0;
    per_sm[2] = prec == PREC_BF16 ? 1000.0 : 140.0;
    per_sm[3] = prec == PREC_F32 ? 250.0 : prec == PREC_BF16 ? 1000.0 : 730.0;
  }
  // per kind: POTRF/TRSM/SYRK/GEMM, or GETRF/GESSM/TSTRF/SSSSM
  const double chol_flops[4] = {nb * nb * nb / 3.0, nb * nb * nb, nb * nb * nb, 2.0 * nb * nb * nb};
  const double lu_flops[4] = {2.0 * nb * nb * nb / 3.0, nb * nb * nb, nb * nb * nb, 2.0 * nb * nb * nb};
  const double *flops = r.lu ? lu_flops : chol_flops;
  for (int k = 0; k < 4; ++k) {
    if (o.cost_ns[k] < 0) return false;
    const double rate = per_sm[k] / (double)r.wps;
    r.cost[k] = o.cost_ns[k] > 0 ? o.cost_ns[k] : std::max<int64_t>(1, (int64_t)(flops[k] / rate));
  }
  r.timeout_ns = o.timeout_ns > 0 ? o.timeout_ns : 10000000000ll;
  r.trace = o.trace ? 1 : 0;
  r.hold_task = o.hold_task;
  r.use_cp = o.use_cp ? 1 : 0;
  {
    const double gbs = o.cp_gbs > 0.0 ? o.cp_gbs : 40.0;  // GB/s = bytes per ns
    const double tile_bytes = nb * nb * (prec == PREC_F64 ? 8.0 : 4.0);
    r.comm_ns = std::max<int64_t>(1, (int64_t)(tile_bytes / gbs));
  }
  if (r.hold_task >= (r.lu ? LuGraph::count(r.T) : CholGraph::count(r.T))) return false;
  if (o.split < 0 || o.split > 2) return false;
  r.keep_next = o.keep_next ? 1 : 0;
  r.split = r.lu ? 0 : o.split;  // the Cholesky tile bodies can be cut into units
  return true;
}

// Workers that will be launched: all SMs x workers per SM, limited by occupancy.
static int launch_workers(const Resolved &r, const DeviceInfo &di) {
  if (di.sms <= 0) return 1024;
  // a failure shows in the occupancy query below and again, checked, in factor_impl
  (void)set_smem_attr(kernel_for(r.prec), smem_limit(r.prec));
  const size_t smem = factor_smem_bytes(r.prec, r.T, 2 * di.sms);
  int per_sm = 0;
  const void *fn = kernel_for(r.prec);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem) != cudaSuccess)
    per_sm = 1;
  per_sm = std::max(1, std::min(per_sm, r.wps));
  int W = di.sms * per_sm;
  if (r.W > 0) W = std::min(W, r.W);
  return W;
}

}  // namespace chol

using namespace chol;

extern "C" size_t chol_factor_lowp_workspace_size(int precision, int n, const chol_opts *opts) {
  const int prec = precision == CHOL_F32 ? PREC_F32
                   : precision == CHOL_BF16 ? PREC_BF16
                   : precision == CHOL_BF16X3 ? PREC_BF16X3
                                              : -1;
  Resolved r;
  if (prec < 0 || n < 0 || !resolve(n, opts, r, prec)) return 0;
  const DeviceInfo di = current_device_info();
  const int W = launch_workers(r, di);
  return make_layout(n, r, W).total;
}

extern "C" size_t chol_factor_workspace_size(int n, const chol_opts *opts) {
  // the same workspace serves the FP64 and FP32 factors (the tensor-core forms also keep the
  // panel tiles' BF16 terms: chol_factor_lowp_workspace_size)
  size_t best = 0;
  for (int prec = PREC_F64; prec <= PREC_F32; ++prec) {
    Resolved r;
    if (n < 0 || !resolve(n, opts, r, prec)) return 0;
    const DeviceInfo di = current_device_info();
    const int W = launch_workers(r, di);
    best = std::max(best, make_layout(n, r, W).total);
  }
  return best;
}

extern "C" long long chol_factor_trace_offset(int n, const chol_opts *opts) {
  Resolved r;
  if (n < 0 || !resolve(n, opts, r) || !r.trace) return -1;
  const DeviceInfo di = current_device_info();
  const int W = launch_workers(r, di);
  return (long long)make_layout(n, r, W).trace;
}

extern "C" int chol_num_workers(const chol_opts *opts) {
  Resolved r;
  if (!resolve(1, opts, r)) return 0;
  const DeviceInfo di = current_device_info();
  if (di.sms <= 0) return 0;
  return launch_workers(r, di);
}

namespace chol {

chol_status factor_impl(int prec, int n, void *dA, int lda, const chol_opts *opts, void *dWork,
                        size_t work_bytes, int *dInfo, void *stream, int *lu_piv, double *lu_lw) {
  Resolved r;
  if (n < 0 || !dInfo || !resolve(n, opts, r, prec)) return CHOL_ERR_INVALID_ARG;
  if (lda < std::max(1, n) || (n > 0 && !dA)) return CHOL_ERR_INVALID_ARG;
  if (r.lu && n > 0 && (!lu_piv || !lu_lw)) return CHOL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    CHOL_CUDA_TRY(cudaMemsetAsync(dInfo, 0, sizeof(int), s));
    return CHOL_OK;
  }
  const DeviceInfo di = current_device_info();
  if (di.sms <= 0) return CHOL_ERR_CUDA;
  if (di.cc_major != 10 || di.cc_minor != 3) return CHOL_ERR_UNSUPPORTED;
  const int W = launch_workers(r, di);
  const Layout L = make_layout(n, r, W);
  if (!dWork || work_bytes < L.total || ((uintptr_t)dWork & 255)) return CHOL_ERR_WORKSPACE;
  unsigned char *ws = static_cast<unsigned char *>(dWork);

  FactorArgs a;
  a.A = dA; a.lda = lda; a.n = n; a.nb = r.nb; a.T = r.T; a.ntasks = L.ntasks;
  a.W = W; a.C = L.C;
  a.policy = r.policy; a.queue_order = r.queue_order; a.steal = r.steal;
  a.dada_max_iter = r.max_iter; a.trace = r.trace;
  a.alpha = r.alpha; a.dada_eps = r.eps;
  for (int k = 0; k < 4; ++k) a.cost[k] = r.cost[k];
  a.timeout_ns = r.timeout_ns;
  a.use_cp = r.use_cp;
  a.comm_ns = r.comm_ns;
  a.iter_limit = std::max<int64_t>(100000, r.timeout_ns / 256);
  a.ctrl = reinterpret_cast<Ctrl *>(ws + L.ctrl);
  a.cnt = reinterpret_cast<int *>(ws + L.cnt);
  a.bl = reinterpret_cast<int64_t *>(ws + L.bl);
  a.owner = reinterpret_cast<int *>(ws + L.owner);
  a.slots = reinterpret_cast<unsigned long long *>(ws + L.slots);
  a.qhead = reinterpret_cast<unsigned int *>(ws + L.qhead);
  a.qcount = reinterpret_cast<int *>(ws + L.qcount);
  a.qcost = reinterpret_cast<unsigned long long *>(ws + L.qcost);
  a.run_end = reinterpret_cast<unsigned long long *>(ws + L.run_end);
  a.sm_busy = reinterpret_cast<int *>(ws + L.sm_busy);
  a.trace_buf = r.trace ? reinterpret_cast<long long *>(ws + L.trace) : nullptr;
  a.split = L.split_tile ? ws + L.split : nullptr;
  a.split_tile = (int64_t)L.split_tile;
  a.lu_piv = lu_piv;
  a.lu_lw = lu_lw;
  a.board = reinterpret_cast<HelpSlot *>(ws + L.board);
  a.split_mode = r.split;
  a.keep_next = r.keep_next && r.queue_order == 0 && (r.policy == P_HEFT || r.policy == P_DADA);

  CHOL_CUDA_TRY(cudaMemsetAsync(ws + L.ctrl, 0, sizeof(Ctrl), s));
  CHOL_CUDA_TRY(cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_end - L.zero_begin, s));
  if (r.trace) CHOL_CUDA_TRY(cudaMemsetAsync(ws + L.trace, 0xff, (size_t)L.ntasks * 32, s));
  {
    const int64_t work = std::max<int64_t>(L.ntasks, (int64_t)r.T * r.T);
    const int blocks = (int)std::min<int64_t>((work + 255) / 256, (int64_t)di.sms * 8);
    if (r.lu) init_kernel<LuGraph><<<blocks, 256, 0, s>>>(r.T, L.ntasks, a.cnt, a.owner, r.hold_task);
    else init_kernel<CholGraph><<<blocks, 256, 0, s>>>(r.T, L.ntasks, a.cnt, a.owner, r.hold_task);
    CHOL_CUDA_TRY(cudaGetLastError());
  }
  if (r.queue_order == 0) {
    const chol_status bs = bottom_levels_device(r.lu, r.T, r.cost, a.bl, s);
    if (bs != CHOL_OK) return bs;
  }
  const size_t smem = factor_smem_bytes(prec, r.T, W);
  void *args[] = {(void *)&a};
  const void *fn = kernel_for(prec);
  if (smem > (size_t)smem_limit(prec)) return CHOL_ERR_UNSUPPORTED;
  CHOL_CUDA_TRY(set_smem_attr(fn, smem_limit(prec)));
  CHOL_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(W), dim3(NT), args, smem, s));
  copy_info_kernel<<<1, 32, 0, s>>>(a.ctrl, dInfo);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

}  // namespace chol

extern "C" chol_status chol_factor(int n, double *dA, int lda, const chol_opts *opts, void *dWork,
                                   size_t work_bytes, int *dInfo, void *stream) {
  return factor_impl(PREC_F64, n, dA, lda, opts, dWork, work_bytes, dInfo, stream);
}

extern "C" chol_status chol_factor_lowp(int precision, int n, float *dA, int lda, const chol_opts *opts,
                                        void *dWork, size_t work_bytes, int *dInfo, void *stream) {
  const int prec = precision == CHOL_F32 ? PREC_F32
                   : precision == CHOL_BF16 ? PREC_BF16
                   : precision == CHOL_BF16X3 ? PREC_BF16X3
                                              : -1;
  if (prec < 0) return CHOL_ERR_INVALID_ARG;
  return factor_impl(prec, n, dA, lda, opts, dWork, work_bytes, dInfo, stream);
}

extern "C" chol_status chol_factor_f32(int n, float *dA, int lda, const chol_opts *opts, void *dWork,
                                       size_t work_bytes, int *dInfo, void *stream) {
  return factor_impl(PREC_F32, n, dA, lda, opts, dWork, work_bytes, dInfo, stream);
}

// ------------------------------------------------------------------------------------
// LU with incremental pivoting on the same persistent kernel

namespace chol {

int lu_tile_size(int n, const chol_opts *opts) {
  Resolved r;
  if (n < 0 || !resolve(n, opts, r, PREC_LU_F64)) return 0;
  return r.nb;
}

}  // namespace chol

extern "C" size_t chol_lu_workspace_size(int n, const chol_opts *opts) {
  Resolved r;
  if (n < 0 || !resolve(n, opts, r, PREC_LU_F64)) return 0;
  const DeviceInfo di = current_device_info();
  const int W = launch_workers(r, di);
  return make_layout(n, r, W).total;
}

extern "C" chol_status chol_lu_aux_size(int n, const chol_opts *opts, long long *piv_count, long long *lw_count) {
  const int nb = lu_tile_size(n, opts);
  if (nb <= 0) return CHOL_ERR_INVALID_ARG;
  const long long T = n > 0 ? (n + nb - 1) / nb : 0;
  if (piv_count) *piv_count = T * T * nb;
  if (lw_count) *lw_count = T * T * (long long)LU_IB * nb;
  return CHOL_OK;
}

extern "C" chol_status chol_lu_factor(int n, double *dA, int lda, int *dPiv, double *dLw, const chol_opts *opts,
                                      void *dWork, size_t work_bytes, int *dInfo, void *stream) {
  return factor_impl(PREC_LU_F64, n, dA, lda, opts, dWork, work_bytes, dInfo, stream, dPiv, dLw);
}
