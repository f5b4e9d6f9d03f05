// Tile task graph of the right-looking lower Cholesky (PLASMA DPOTRF, Section 4.1).
//
// Tasks are numbered step by step: step k holds POTRF(k), then TRSM(i,k) for i = k+1..T-1,
// then SYRK(i,k) for i = k+1..T-1, then GEMM(i,j,k) for k < j < i < T with the pair index
// (i', j') = (i-k-1, j-k-1) enumerated as i'(i'-1)/2 + j'. Successors and dependency counts
// are arithmetic in (kind, i, j, k); nothing about the graph is stored.
//
// Dependencies (each task waits for the last writer of every tile it touches, Section 2):
//   POTRF(k)   <- SYRK(k, k-1)
//   TRSM(i,k)  <- POTRF(k), GEMM(i, k, k-1)
//   SYRK(i,k)  <- TRSM(i,k), SYRK(i, k-1)
//   GEMM(i,j,k)<- TRSM(i,k), TRSM(j,k), GEMM(i, j, k-1)
// (the k-1 terms exist for k > 0).
#pragma once
#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define CHOL_HD __host__ __device__ __forceinline__
#else
#define CHOL_HD inline
#endif

namespace chol {

enum TaskKind { K_POTRF = 0, K_TRSM = 1, K_SYRK = 2, K_GEMM = 3 };

struct TaskDesc {
  int kind, i, j, k;
};

// Number of tasks of a step whose trailing tile count is m = T-1-k.
CHOL_HD int64_t step_size(int64_t m) { return 1 + 2 * m + m * (m - 1) / 2; }

// sum_{m'=0}^{M-1} step_size(m') = M + M(M-1) + M(M-1)(M-2)/6
CHOL_HD int64_t steps_prefix(int64_t M) { return M + M * (M - 1) + M * (M - 1) * (M - 2) / 6; }

CHOL_HD int64_t task_count(int T) { return steps_prefix(T); }

// First task id of step k.
CHOL_HD int64_t step_offset(int T, int k) { return steps_prefix(T) - steps_prefix(T - k); }

CHOL_HD int64_t edge_count(int T) {
  // per step with m trailing tiles: POTRF m, TRSM m*m, SYRK m, GEMM m(m-1)/2
  int64_t e = 0;
  for (int k = 0; k < T; ++k) {
    int64_t m = T - 1 - k;
    e += 2 * m + m * m + m * (m - 1) / 2;
  }
  return e;
}

CHOL_HD int64_t task_id(int T, int kind, int i, int j, int k) {
  const int64_t base = step_offset(T, k);
  const int64_t m = T - 1 - k;
  switch (kind) {
    case K_POTRF: return base;
    case K_TRSM: return base + (i - k);
    case K_SYRK: return base + m + (i - k);
    default: {
      const int64_t ip = i - k - 1, jp = j - k - 1;
      return base + 1 + 2 * m + ip * (ip - 1) / 2 + jp;
    }
  }
}

CHOL_HD TaskDesc task_desc(int T, int64_t id) {
  // step k: largest k with step_offset(T,k) <= id (binary search, offsets increase with k)
  int lo = 0, hi = T - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (step_offset(T, mid) <= id) lo = mid; else hi = mid - 1;
  }
  const int k = lo;
  const int64_t r = id - step_offset(T, k);
  const int64_t m = T - 1 - k;
  TaskDesc d;
  d.k = k;
  if (r == 0) { d.kind = K_POTRF; d.i = k; d.j = k; }
  else if (r <= m) { d.kind = K_TRSM; d.i = k + (int)r; d.j = k; }
  else if (r <= 2 * m) { d.kind = K_SYRK; d.i = k + (int)(r - m); d.j = d.i; }
  else {
    const int64_t g = r - 2 * m - 1;
    // largest ip with ip(ip-1)/2 <= g
    int64_t ip = (int64_t)((1.0 + sqrt(1.0 + 8.0 * (double)g)) * 0.5);
    while (ip * (ip - 1) / 2 > g) --ip;
    while ((ip + 1) * ip / 2 <= g) ++ip;
    const int64_t jp = g - ip * (ip - 1) / 2;
    d.kind = K_GEMM; d.i = k + 1 + (int)ip; d.j = k + 1 + (int)jp;
  }
  return d;
}

CHOL_HD int initial_count(const TaskDesc &d) {
  switch (d.kind) {
    case K_POTRF: return d.k > 0 ? 1 : 0;
    case K_TRSM: return d.k > 0 ? 2 : 1;
    case K_SYRK: return d.k > 0 ? 2 : 1;
    default: return d.k > 0 ? 3 : 2;
  }
}

CHOL_HD int num_successors(int T, const TaskDesc &d) {
  switch (d.kind) {
    case K_POTRF: return T - 1 - d.k;
    case K_TRSM: return T - 1 - d.k;
    case K_SYRK: return d.k + 1 < d.i ? 1 : 1;  // SYRK(i,k+1) or POTRF(i)
    default: return 1;                           // GEMM(i,j,k+1) or TRSM(i,j)
  }
}

// s-th successor of task d, 0 <= s < num_successors.
CHOL_HD int64_t successor(int T, const TaskDesc &d, int s) {
  switch (d.kind) {
    case K_POTRF: return task_id(T, K_TRSM, d.k + 1 + s, d.k, d.k);
    case K_TRSM: {
      // s = 0: SYRK(i,k); then GEMM(i, j, k) for j = k+1..i-1; then GEMM(m, i, k), m = i+1..T-1
      if (s == 0) return task_id(T, K_SYRK, d.i, d.i, d.k);
      const int a = s - 1;
      const int left = d.i - d.k - 1;
      if (a < left) return task_id(T, K_GEMM, d.i, d.k + 1 + a, d.k);
      return task_id(T, K_GEMM, d.i + 1 + (a - left), d.i, d.k);
    }
    case K_SYRK:
      if (d.k + 1 == d.i) return task_id(T, K_POTRF, d.i, d.i, d.i);
      return task_id(T, K_SYRK, d.i, d.i, d.k + 1);
    default:
      if (d.k + 1 == d.j) return task_id(T, K_TRSM, d.i, d.j, d.j);
      return task_id(T, K_GEMM, d.i, d.j, d.k + 1);
  }
}

// The tile a task modifies (row, column in tiles).
CHOL_HD void rw_tile(const TaskDesc &d, int &ti, int &tj) {
  switch (d.kind) {
    case K_POTRF: ti = d.k; tj = d.k; break;
    case K_TRSM: ti = d.i; tj = d.k; break;
    case K_SYRK: ti = d.i; tj = d.i; break;
    default: ti = d.i; tj = d.j; break;
  }
}

// Bottom level of task d given the bottom levels of all its successors.
CHOL_HD int64_t bottom_level_of(int T, const TaskDesc &d, const int64_t *cost, const int64_t *bl) {
  int64_t best = 0;
  const int ns = num_successors(T, d);
  for (int s = 0; s < ns; ++s) {
    const int64_t v = bl[successor(T, d, s)];
    best = v > best ? v : best;
  }
  return cost[d.kind] + best;
}

}  // namespace chol

namespace chol {

// The Cholesky graph behind the interface the persistent kernel runs any tile graph through.
struct CholGraph {
  static constexpr int KIND0 = K_POTRF;
  CHOL_HD static int64_t count(int T) { return task_count(T); }
  CHOL_HD static TaskDesc desc(int T, int64_t id) { return task_desc(T, id); }
  CHOL_HD static int initial(const TaskDesc &d) { return initial_count(d); }
  CHOL_HD static int nsucc(int T, const TaskDesc &d) { return num_successors(T, d); }
  CHOL_HD static int64_t succ(int T, const TaskDesc &d, int s) { return successor(T, d, s); }
  CHOL_HD static void rw(const TaskDesc &d, int &ti, int &tj) { rw_tile(d, ti, tj); }
  // at most one ready task per tile of the lower triangle (the writers of a tile form a chain)
  CHOL_HD static int64_t max_ready(int T) { return (int64_t)T * (T + 1) / 2; }
  // tiles a task reads or updates, for the communication prediction
  CHOL_HD static int inputs(const TaskDesc &d, int *ti, int *tj) {
    switch (d.kind) {
      case K_POTRF: ti[0] = d.k; tj[0] = d.k; return 1;
      case K_TRSM: ti[0] = d.k; tj[0] = d.k; ti[1] = d.i; tj[1] = d.k; return 2;
      case K_SYRK: ti[0] = d.i; tj[0] = d.k; ti[1] = d.i; tj[1] = d.i; return 2;
      default:
        ti[0] = d.i; tj[0] = d.k; ti[1] = d.j; tj[1] = d.k; ti[2] = d.i; tj[2] = d.j;
        return 3;
    }
  }
};

}  // namespace chol
