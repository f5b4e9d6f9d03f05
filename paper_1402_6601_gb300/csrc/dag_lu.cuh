// Tile task graph of the LU factorization with incremental pivoting (PLASMA DGETRF, the
// paper's second workload, Section 4.1), in the interface of CholGraph.
//
// Step k holds GETRF(k), then GESSM(k, j) for j = k+1..T-1, then TSTRF(i, k) for
// i = k+1..T-1, then SSSSM(i, j, k) for i, j in k+1..T-1 (i-major). Task descriptors use
// (kind, i, j, k) = GETRF (0, k, k, k), GESSM (1, k, j, k), TSTRF (2, i, k, k),
// SSSSM (3, i, j, k). Every successor has a larger id than its predecessor.
//
// Dependencies, from the tiles each kernel reads and writes (Section 2: a task waits for the
// last writer of what it touches). A diagonal tile is two regions: the unit lower factor of
// GETRF, which GESSM reads, and the upper factor, which the TSTRF chain of the step updates.
//   GETRF(k)      <- SSSSM(k, k, k-1)
//   GESSM(k, j)   <- GETRF(k), SSSSM(k, j, k-1)
//   TSTRF(i, k)   <- GETRF(k) (i = k+1) or TSTRF(i-1, k); SSSSM(i, k, k-1)
//   SSSSM(i,j,k)  <- TSTRF(i, k); GESSM(k, j) (i = k+1) or SSSSM(i-1, j, k); SSSSM(i, j, k-1)
// (the k-1 terms exist for k > 0).
#pragma once
#include "dag.cuh"

namespace chol {

enum LuKind { K_GETRF = 0, K_GESSM = 1, K_TSTRF = 2, K_SSSSM = 3 };

struct LuGraph {
  static constexpr int KIND0 = K_GETRF;
  // tasks of a step with m = T-1-k trailing tile rows: 1 + 2m + m^2
  CHOL_HD static int64_t step_size(int64_t m) { return 1 + 2 * m + m * m; }
  // sum_{m'=0}^{M-1} step_size(m')
  CHOL_HD static int64_t steps_prefix(int64_t M) { return M + M * (M - 1) + (M - 1) * M * (2 * M - 1) / 6; }
  CHOL_HD static int64_t count(int T) { return steps_prefix(T); }
  CHOL_HD static int64_t step_offset(int T, int k) { return steps_prefix(T) - steps_prefix(T - k); }

  CHOL_HD static int64_t id(int T, int kind, int i, int j, int k) {
    const int64_t base = step_offset(T, k);
    const int64_t m = T - 1 - k;
    switch (kind) {
      case K_GETRF: return base;
      case K_GESSM: return base + (j - k);
      case K_TSTRF: return base + m + (i - k);
      default: return base + 1 + 2 * m + (int64_t)(i - k - 1) * m + (j - k - 1);
    }
  }

  CHOL_HD static TaskDesc desc(int T, int64_t id) {
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
    if (r == 0) { d.kind = K_GETRF; d.i = k; d.j = k; }
    else if (r <= m) { d.kind = K_GESSM; d.i = k; d.j = k + (int)r; }
    else if (r <= 2 * m) { d.kind = K_TSTRF; d.i = k + (int)(r - m); d.j = k; }
    else {
      const int64_t g = r - 2 * m - 1;
      d.kind = K_SSSSM;
      d.i = k + 1 + (int)(g / m);
      d.j = k + 1 + (int)(g % m);
    }
    return d;
  }

  CHOL_HD static int initial(const TaskDesc &d) {
    const int prev = d.k > 0 ? 1 : 0;
    switch (d.kind) {
      case K_GETRF: return prev;
      case K_GESSM: return 1 + prev;
      case K_TSTRF: return 1 + prev;
      default: return 2 + prev;
    }
  }

  CHOL_HD static int nsucc(int T, const TaskDesc &d) {
    const int m = T - 1 - d.k;
    switch (d.kind) {
      case K_GETRF: return m + (m > 0 ? 1 : 0);  // GESSM(k, j) for all j, TSTRF(k+1, k)
      case K_GESSM: return 1;                    // SSSSM(k+1, j, k)
      case K_TSTRF: return m + (d.i + 1 < T ? 1 : 0);  // SSSSM(i, j, k) for all j, TSTRF(i+1, k)
      default: return 1 + (d.i + 1 < T ? 1 : 0);  // next writer of A_ij, SSSSM(i+1, j, k)
    }
  }

  // s-th successor, 0 <= s < nsucc
  CHOL_HD static int64_t succ(int T, const TaskDesc &d, int s) {
    const int k = d.k;
    const int m = T - 1 - k;
    switch (d.kind) {
      case K_GETRF:
        return s < m ? id(T, K_GESSM, k, k + 1 + s, k) : id(T, K_TSTRF, k + 1, k, k);
      case K_GESSM:
        return id(T, K_SSSSM, k + 1, d.j, k);
      case K_TSTRF:
        return s < m ? id(T, K_SSSSM, d.i, k + 1 + s, k) : id(T, K_TSTRF, d.i + 1, k, k);
      default: {
        if (s == 1) return id(T, K_SSSSM, d.i + 1, d.j, k);
        // the writer of A_ij in step k+1
        const int i = d.i, j = d.j, k1 = k + 1;
        if (i == k1 && j == k1) return id(T, K_GETRF, k1, k1, k1);
        if (i == k1) return id(T, K_GESSM, k1, j, k1);
        if (j == k1) return id(T, K_TSTRF, i, k1, k1);
        return id(T, K_SSSSM, i, j, k1);
      }
    }
  }

  // the tile whose multipliers or factor the task produces (its affinity tile)
  CHOL_HD static void rw(const TaskDesc &d, int &ti, int &tj) {
    switch (d.kind) {
      case K_GETRF: ti = d.k; tj = d.k; break;
      case K_GESSM: ti = d.k; tj = d.j; break;
      case K_TSTRF: ti = d.i; tj = d.k; break;
      default: ti = d.i; tj = d.j; break;
    }
  }

  // at most one ready task per tile (the writers of each tile form a chain)
  CHOL_HD static int64_t max_ready(int T) { return (int64_t)T * T; }

  CHOL_HD static int inputs(const TaskDesc &d, int *ti, int *tj) {
    switch (d.kind) {
      case K_GETRF: ti[0] = d.k; tj[0] = d.k; return 1;
      case K_GESSM: ti[0] = d.k; tj[0] = d.k; ti[1] = d.k; tj[1] = d.j; return 2;
      case K_TSTRF: ti[0] = d.k; tj[0] = d.k; ti[1] = d.i; tj[1] = d.k; return 2;
      default:
        ti[0] = d.i; tj[0] = d.k; ti[1] = d.k; tj[1] = d.j; ti[2] = d.i; tj[2] = d.j;
        return 3;
    }
  }

  // bottom level of d from its successors' bottom levels
  CHOL_HD static int64_t bottom_level_of(int T, const TaskDesc &d, const int64_t *cost, const int64_t *bl) {
    int64_t best = 0;
    const int ns = nsucc(T, d);
    for (int s = 0; s < ns; ++s) {
      const int64_t v = bl[succ(T, d, s)];
      best = v > best ? v : best;
    }
    return cost[d.kind] + best;
  }
};

}  // namespace chol
