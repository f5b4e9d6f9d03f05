// FP64 tile kernels of the LU factorization with incremental pivoting (PLASMA DGETRF,
// Section 4.1), executed by one 256-thread block (one worker), and the pieces the LU solve
// shares with them.
//
// Every kernel works on inner blocks of LU_IB columns. For one block the elimination is an
// LU with partial pivoting of a panel of rows held in shared memory (lu_panel); the panel's
// rows are numbered by positions (0 .. w-1: the rows the block's pivots end up in; w ..: the
// rows below them) and the pivot of column j is the position interchanged with position j.
// The block's transformation of any rows [X1; X2] laid out the same way (lu_apply_block)
// is: the interchanges in order, X1 <- L11^{-1} X1 with the panel's unit lower L11, and
// X2 <- X2 - L21 X1 with its multipliers L21 (a DFMA tile update). Multipliers of earlier
// blocks are not interchanged by later blocks.
//
//   GETRF(k)      panels of the diagonal tile; the right part of the tile transformed
//   GESSM(k, j)   GETRF(k)'s blocks applied to A_kj
//   TSTRF(i, k)   panels [rows of U_kk (upper part); A_ik]; U_kk and A_ik transformed; the
//                 unit lower L11 of each block goes to Lw(i, k), since U_kk's strict lower
//                 triangle holds GETRF(k)'s multipliers
//   SSSSM(i,j,k)  TSTRF(i, k)'s blocks applied to [A_kj; A_ij]
//
// Storage: pivots of GETRF(k) / TSTRF(i, k) are one int per column of tile k (positions
// relative to the block); Lw(i, k) is LU_IB x nk, column-major, block b's L11 (strict lower
// part, zeros elsewhere) in columns b*LU_IB ...
#pragma once
#include <stdint.h>
#include "tiles_f64.cuh"

namespace chol {

constexpr int LU_IB = 32;
constexpr int LU_NB_MAX = 256;                               // tile size limit of the LU kernels
constexpr int LU_PANEL_DOUBLES = (LU_IB + LU_NB_MAX) * LU_IB;  // TSTRF panel: (w + mi) x w
static_assert(LU_PANEL_DOUBLES >= STAGE_DOUBLES, "the tile update's staging must fit the panel area");
static_assert(LU_IB * LU_NB_MAX <= LU_PANEL_DOUBLES, "the apply scratch must fit the panel area");
// shared memory: panel / apply scratch / update staging, then L11 (LU_IB x DS_LD), then the
// block's pivots
constexpr int LU_SMEM_BYTES = (LU_PANEL_DOUBLES + LU_IB * DS_LD) * 8 + LU_IB * 4;

struct LuSmem {
  double *work;  // LU_PANEL_DOUBLES
  double *l11;   // LU_IB x DS_LD, row-major
  int *piv;      // LU_IB
};

__device__ __forceinline__ LuSmem lu_smem(double *smem) {
  LuSmem s;
  s.work = smem;
  s.l11 = smem + LU_PANEL_DOUBLES;
  s.piv = reinterpret_cast<int *>(smem + LU_PANEL_DOUBLES + LU_IB * DS_LD);
  return s;
}

// LU with partial pivoting of the m x w panel P (shared, column-major, ld ldp) in place: for
// each column the first row of largest magnitude at or below the diagonal is the pivot, the
// two rows are interchanged across the panel, the column below is divided by the pivot and
// the rest of the panel receives the rank-one update. piv[j] = pivot position of column j.
// Returns 0 or the 1-based column of the first zero pivot (that column is then left
// unscaled). Called by all threads; ends synchronised.
static __device__ __noinline__ int lu_panel(double *P, int ldp, int m, int w, int *piv) {
  __shared__ double s_val[NT / 32];
  __shared__ int s_idx[NT / 32];
  __shared__ int s_p;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int info = 0;
  const int steps = min(m, w);
  for (int j = 0; j < steps; ++j) {
    double best = -1.0;
    int bi = m;
    for (int r = j + tid; r < m; r += NT) {
      const double v = fabs(P[j * ldp + r]);
      if (v > best) { best = v; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = s_val[0];
      int p = s_idx[0];
      for (int q = 1; q < NT / 32; ++q)
        if (s_val[q] > b || (s_val[q] == b && s_idx[q] < p)) { b = s_val[q]; p = s_idx[q]; }
      if (p >= m) p = j;  // no comparable value (NaN column): keep the diagonal row
      s_p = p;
      piv[j] = p;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j && tid < w) {
      const double t = P[tid * ldp + j];
      P[tid * ldp + j] = P[tid * ldp + p];
      P[tid * ldp + p] = t;
    }
    __syncthreads();
    const double d = P[j * ldp + j];
    if (d == 0.0) {
      if (!info) info = j + 1;
    } else {
      const double rinv = 1.0 / d;
      // each thread scales its rows and updates them with the pivot row (not modified here)
      for (int r = j + 1 + tid; r < m; r += NT) {
        const double l = quot(P[j * ldp + r], d, rinv);
        P[j * ldp + r] = l;
        for (int c = j + 1; c < w; ++c) P[c * ldp + r] = fma(-l, P[c * ldp + j], P[c * ldp + r]);
      }
    }
    __syncthreads();
  }
  return info;
}

// One inner block's transformation applied to the rows [X1 (w rows); X2 (mA rows)] over
// ncols <= LU_NB_MAX columns (global, column-major): the interchanges piv[0..w) in order,
// X1 <- L11^{-1} X1 (unit lower, shared), X2 <- X2 - L21 X1 (L21 global mA x w). One thread
// per column for the first two steps (the column's X1 part staged in shared memory), then the
// DFMA tile update. Called by all threads; ends synchronised.
static __device__ __noinline__ void lu_apply_block(double *X1, int64_t ld1, double *X2, int64_t ld2, int ncols,
                                                   int w, const int *piv, const double *L11, int mA,
                                                   const double *L21, int64_t ldl, double *smem) {
  double *Xs = smem;  // w x ncols, row-major: thread c touches column c
  // X2 rows the interchanges touch: slot j holds position piv[j] if j is its first occurrence
  // (later interchanges with the same position use that slot), -1 if piv[j] is not an X2 row
  __shared__ int s_slot[LU_IB];
  if (threadIdx.x < w) {
    const int j = threadIdx.x, q = piv[j];
    int sl = -1;
    if (q != j && q >= w && q < w + mA) {
      sl = j;
      for (int jj = 0; jj < j; ++jj)
        if (piv[jj] == q) { sl = jj; break; }
    }
    s_slot[j] = sl;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncols; c += NT) {
    const double *x1 = X1 + (int64_t)c * ld1;
    for (int r = 0; r < w; ++r) Xs[r * ncols + c] = ldcg(x1 + r);
    // the touched X2 values are loaded together, interchanged in the thread's own slots, and
    // stored back once: the same sequence of interchanges without a dependent load from
    // global memory per interchange
    double *x2c = X2 + (int64_t)c * ld2;
    double c2[LU_IB];
    for (int j = 0; j < w; ++j)
      if (s_slot[j] == j) c2[j] = ldcg(x2c + (piv[j] - w));
    for (int j = 0; j < w; ++j) {
      const int q = piv[j];
      if (q == j || q < 0 || q >= w + mA) continue;  // positions outside the rows: not a pivot
      if (q < w) {
        const double t = Xs[j * ncols + c];
        Xs[j * ncols + c] = Xs[q * ncols + c];
        Xs[q * ncols + c] = t;
      } else {
        const int sl = s_slot[j];
        const double t = c2[sl];
        c2[sl] = Xs[j * ncols + c];
        Xs[j * ncols + c] = t;
      }
    }
    for (int j = 0; j < w; ++j)
      if (s_slot[j] == j) stcg(x2c + (piv[j] - w), c2[j]);
    for (int r = 1; r < w; ++r) {
      double t = Xs[r * ncols + c];
      for (int j = 0; j < r; ++j) t = fma(-L11[r * DS_LD + j], Xs[j * ncols + c], t);
      Xs[r * ncols + c] = t;
    }
    double *y1 = X1 + (int64_t)c * ld1;
    for (int r = 0; r < w; ++r) stcg(y1 + r, Xs[r * ncols + c]);
  }
  __syncthreads();
  if (mA > 0 && ncols > 0) update_core<true>(X2, ld2, L21, ldl, X1, ld1, mA, ncols, w, false, smem);
  __syncthreads();
}

// L11 of a block from the strict lower part of a w x w block (global, column-major, ld),
// zero elsewhere. Ends synchronised.
__device__ __forceinline__ void lu_load_l11(const double *B, int64_t ld, int w, double *L11) {
  for (int e = threadIdx.x; e < LU_IB * LU_IB; e += NT) {
    const int r = e & (LU_IB - 1), c = e >> 5;
    L11[r * DS_LD + c] = (r < w && c < r) ? ldcg(B + (int64_t)c * ld + r) : 0.0;
  }
  __syncthreads();
}

// GETRF on the nk x nk diagonal tile G (in place); ipiv receives nk pivot positions.
// Returns 0 or the 1-based column (inside the tile) of the first zero pivot.
static __device__ __noinline__ int lu_getrf_tile(double *G, int64_t ld, int nk, int *ipiv, double *smem) {
  const LuSmem s = lu_smem(smem);
  int info = 0;
  for (int c0 = 0; c0 < nk; c0 += LU_IB) {
    const int w = min(LU_IB, nk - c0), m = nk - c0, c1 = c0 + w;
    double *P = s.work;  // m x w, ld m
    for (int e = threadIdx.x; e < m * w; e += NT) {
      const int c = e / m, r = e - c * m;
      P[c * m + r] = ldcg(G + (int64_t)(c0 + c) * ld + c0 + r);
    }
    __syncthreads();
    const int f = lu_panel(P, m, m, w, s.piv);
    if (f && !info) info = c0 + f;
    for (int e = threadIdx.x; e < m * w; e += NT) {
      const int c = e / m, r = e - c * m;
      stcg(G + (int64_t)(c0 + c) * ld + c0 + r, P[c * m + r]);
    }
    for (int e = threadIdx.x; e < LU_IB * LU_IB; e += NT) {
      const int r = e & (LU_IB - 1), c = e >> 5;
      s.l11[r * DS_LD + c] = (r < w && c < r) ? P[c * m + r] : 0.0;
    }
    if (threadIdx.x < w) ipiv[c0 + threadIdx.x] = s.piv[threadIdx.x];
    __syncthreads();
    if (c1 < nk)
      lu_apply_block(G + (int64_t)c1 * ld + c0, ld, G + (int64_t)c1 * ld + c1, ld, nk - c1, w, s.piv, s.l11,
                     nk - c1, G + (int64_t)c0 * ld + c1, ld, s.work);
  }
  __syncthreads();
  return info;
}

// GESSM: GETRF(k)'s transformation (diagonal tile Akk of order nk, pivots ipiv) applied to
// the nk x nj tile Akj in place.
static __device__ __noinline__ void lu_gessm_tile(double *Akj, int64_t ld, int nk, int nj, const double *Akk,
                                                  const int *ipiv, double *smem) {
  const LuSmem s = lu_smem(smem);
  for (int c0 = 0; c0 < nk; c0 += LU_IB) {
    const int w = min(LU_IB, nk - c0), c1 = c0 + w;
    if (threadIdx.x < w) s.piv[threadIdx.x] = ipiv[c0 + threadIdx.x];
    lu_load_l11(Akk + (int64_t)c0 * ld + c0, ld, w, s.l11);
    lu_apply_block(Akj + c0, ld, Akj + c1, ld, nj, w, s.piv, s.l11, nk - c1, Akk + (int64_t)c0 * ld + c1, ld,
                   s.work);
  }
}

// TSTRF: LU with partial pivoting of [U_kk; A_ik] in place (U_kk nk x nk upper part, A_ik
// mi x nk); ipiv receives nk positions, Lw (LU_IB x nk, ld LU_IB) the blocks' L11. Returns 0
// or the 1-based column of the first zero pivot.
static __device__ __noinline__ int lu_tstrf_tile(double *Ukk, double *Aik, int64_t ld, int nk, int mi, int *ipiv,
                                                 double *Lw, double *smem) {
  const LuSmem s = lu_smem(smem);
  int info = 0;
  for (int c0 = 0; c0 < nk; c0 += LU_IB) {
    const int w = min(LU_IB, nk - c0), m = w + mi, c1 = c0 + w;
    double *P = s.work;  // m x w, ld m
    for (int e = threadIdx.x; e < m * w; e += NT) {
      const int c = e / m, r = e - c * m;
      double v;
      if (r < w) v = c >= r ? ldcg(Ukk + (int64_t)(c0 + c) * ld + c0 + r) : 0.0;
      else v = ldcg(Aik + (int64_t)(c0 + c) * ld + (r - w));
      P[c * m + r] = v;
    }
    __syncthreads();
    const int f = lu_panel(P, m, m, w, s.piv);
    if (f && !info) info = c0 + f;
    for (int e = threadIdx.x; e < m * w; e += NT) {
      const int c = e / m, r = e - c * m;
      const double v = P[c * m + r];
      if (r >= w) stcg(Aik + (int64_t)(c0 + c) * ld + (r - w), v);
      else if (c >= r) stcg(Ukk + (int64_t)(c0 + c) * ld + c0 + r, v);
    }
    for (int e = threadIdx.x; e < LU_IB * LU_IB; e += NT) {
      const int r = e & (LU_IB - 1), c = e >> 5;
      const double v = (r < w && c < w && c < r) ? P[c * m + r] : 0.0;
      s.l11[r * DS_LD + c] = v;
      if (c < w) stcg(Lw + (int64_t)(c0 + c) * LU_IB + r, v);
    }
    if (threadIdx.x < w) ipiv[c0 + threadIdx.x] = s.piv[threadIdx.x];
    __syncthreads();
    if (c1 < nk)
      lu_apply_block(Ukk + (int64_t)c1 * ld + c0, ld, Aik + (int64_t)c1 * ld, ld, nk - c1, w, s.piv, s.l11, mi,
                     Aik + (int64_t)c0 * ld, ld, s.work);
  }
  __syncthreads();
  return info;
}

// SSSSM: TSTRF(i, k)'s transformation (multipliers in Aik, mi x nk; pivots ipiv; L11 blocks
// in Lw) applied to [A_kj (nk x nj); A_ij (mi x nj)] in place.
static __device__ __noinline__ void lu_ssssm_tile(double *Akj, double *Aij, int64_t ld, const double *Aik, int nk,
                                                  int mi, int nj, const int *ipiv, const double *Lw,
                                                  double *smem) {
  const LuSmem s = lu_smem(smem);
  for (int c0 = 0; c0 < nk; c0 += LU_IB) {
    const int w = min(LU_IB, nk - c0);
    if (threadIdx.x < w) s.piv[threadIdx.x] = ipiv[c0 + threadIdx.x];
    lu_load_l11(Lw + (int64_t)c0 * LU_IB, LU_IB, w, s.l11);
    lu_apply_block(Akj + c0, ld, Aij, ld, nj, w, s.piv, s.l11, mi, Aik + (int64_t)c0 * ld, ld, s.work);
  }
}

}  // namespace chol
