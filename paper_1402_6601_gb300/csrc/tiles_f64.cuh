// FP64 tile task bodies, executed by one 256-thread block (one worker) at a time.
//
// On sm_103 the FP64 units retire two fused multiply-adds per clock per SM, and the FP64
// mma.sync shapes run slower than plain DFMA, so the contraction is a register-tiled DFMA
// update fed through shared memory: every operand byte is reused 32 times from shared
// memory and 4 times from registers, far more than the FP64 rate needs, and the tile
// bodies stay bound by the FP64 pipe.
//
// Global memory is read with ld.global.cg and written with st.global.cg: tiles written by
// one worker are read by others after the dependency counters say so, and L2 is the point
// where all SMs see the same bytes.
#pragma once
#include <stdint.h>

namespace chol {

constexpr int NT = 256;  // threads per worker
constexpr int BM = 64, BN = 64, BK = 32;
constexpr int IB = 32;   // inner block of the POTRF and TRSM bodies
constexpr int DS_LD = IB + 1;

// shared memory: staging [2][BK][BM] + [2][BK][BN] doubles, then the 32 x 33 diagonal block
// and the reciprocals of its diagonal
constexpr int STAGE_DOUBLES = 2 * BK * BM + 2 * BK * BN;
constexpr int TILE_SMEM_BYTES = (STAGE_DOUBLES + IB * DS_LD + IB) * 8;

__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(double *p, double v) { __stcg(p, v); }

// One 32-deep k chunk of the 4 x 4 register tile: acc[i][j] += a[i] b[j] with a[i] the rows
// tx + 16 i, b[j] the columns ty + 16 j of the block. DIAG (a diagonal block of a lower
// update): rows tx + 16 i and columns ty + 16 j with i < j never meet row >= column (tx, ty <
// 16), so those six chains are left out -- their values would not be stored -- and the FP64
// pipe, which a predicated-off instruction would still occupy, does 10 of 16 FMAs per step.
// NI, NJ: the 16-row / 16-column groups of the block that hold rows < M / columns < N (the
// last block of a ragged update has fewer); the chains of the other groups are left out too.
template <bool DIAG, int NI, int NJ>
__device__ __forceinline__ void mac_chunk(double (&acc)[4][4], const double *as, const double *bs, int tx, int ty) {
#pragma unroll 8
  for (int kk = 0; kk < BK; ++kk) {
    double a[4], b[4];
#pragma unroll
    for (int i = 0; i < NI; ++i) a[i] = as[kk * BM + tx + 16 * i];
#pragma unroll
    for (int j = 0; j < NJ; ++j) b[j] = bs[kk * BN + ty + 16 * j];
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        if (!DIAG || i >= j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

// mac_chunk for the block's live groups (block-uniform: no divergence)
template <bool DIAG>
__device__ __forceinline__ void mac_chunk_live(double (&acc)[4][4], const double *as, const double *bs, int tx,
                                               int ty, int ni, int nj) {
#define CHOL_MAC_NJ(NI)                                                          \
  switch (nj) {                                                                  \
    case 1: mac_chunk<DIAG, NI, 1>(acc, as, bs, tx, ty); break;                  \
    case 2: mac_chunk<DIAG, NI, 2>(acc, as, bs, tx, ty); break;                  \
    case 3: mac_chunk<DIAG, NI, 3>(acc, as, bs, tx, ty); break;                  \
    default: mac_chunk<DIAG, NI, 4>(acc, as, bs, tx, ty); break;                 \
  }
  switch (ni) {
    case 1: CHOL_MAC_NJ(1) break;
    case 2: CHOL_MAC_NJ(2) break;
    case 3: CHOL_MAC_NJ(3) break;
    default: CHOL_MAC_NJ(4) break;
  }
#undef CHOL_MAC_NJ
}

// C[M x N] -= A[M x K] * op(B), column-major: op(B) = B^T with B N x K (B_KN = false), or
// op(B) = B with B K x N (B_KN = true, the form of the LU updates). With `lower`, only
// elements with row >= column (relative to C) are written and blocks wholly above the
// diagonal skipped. Called by all NT threads; ends with the block synchronised.
template <bool B_KN>
static __device__ __noinline__ void update_core(double *C, int64_t ldc, const double *A, int64_t lda,
                                                const double *B, int64_t ldb, int M, int N, int K,
                                                bool lower, double *smem) {
  double *As = smem;
  double *Bs = smem + 2 * BK * BM;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int lrow = tid & 63, lk = tid >> 6;  // loader: row lrow, k columns lk + 4q
  const int kk_b = tid & 31, ncol_b = tid >> 5;  // K x N loader of B: k = kk_b, columns ncol_b + 8q
  for (int bn = 0; bn < N; bn += BN) {
    for (int bm = 0; bm < M; bm += BM) {
      if (lower && bm + BM <= bn) continue;
      double acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
      double ra[8], rb[8];
      const bool arow = bm + lrow < M, brow = bn + lrow < N;
      const int ni = min(4, (M - bm + 15) / 16), nj = min(4, (N - bn + 15) / 16);  // live groups
      const double *Ap = A + bm + lrow;
      const double *Bp = B_KN ? B + (int64_t)(bn + ncol_b) * ldb + kk_b : B + bn + lrow;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int kk = lk + 4 * q;
        ra[q] = (arow && kk < K) ? ldcg(Ap + (int64_t)kk * lda) : 0.0;
        if (B_KN)
          rb[q] = (bn + ncol_b + 8 * q < N && kk_b < K) ? ldcg(Bp + (int64_t)(8 * q) * ldb) : 0.0;
        else
          rb[q] = (brow && kk < K) ? ldcg(Bp + (int64_t)kk * ldb) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        As[(lk + 4 * q) * BM + lrow] = ra[q];
        if (B_KN) Bs[kk_b * BN + ncol_b + 8 * q] = rb[q];
        else Bs[(lk + 4 * q) * BN + lrow] = rb[q];
      }
      __syncthreads();
      int buf = 0;
      for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int kk = k0 + BK + lk + 4 * q;
            ra[q] = (arow && kk < K) ? ldcg(Ap + (int64_t)kk * lda) : 0.0;
            if (B_KN)
              rb[q] = (bn + ncol_b + 8 * q < N && k0 + BK + kk_b < K)
                          ? ldcg(Bp + (int64_t)(8 * q) * ldb + k0 + BK) : 0.0;
            else
              rb[q] = (brow && kk < K) ? ldcg(Bp + (int64_t)kk * ldb) : 0.0;
          }
        }
        const double *as = As + buf * BK * BM;
        const double *bs = Bs + buf * BK * BN;
        if (lower && bm == bn) mac_chunk_live<true>(acc, as, bs, tx, ty, ni, nj);  // uniform over the block
        else mac_chunk_live<false>(acc, as, bs, tx, ty, ni, nj);
        if (more) {
          double *an = As + (buf ^ 1) * BK * BM;
          double *bnx = Bs + (buf ^ 1) * BK * BN;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            an[(lk + 4 * q) * BM + lrow] = ra[q];
            if (B_KN) bnx[kk_b * BN + ncol_b + 8 * q] = rb[q];
            else bnx[(lk + 4 * q) * BN + lrow] = rb[q];
          }
        }
        __syncthreads();
        buf ^= 1;
      }
      // loads of C before any store, so that they overlap instead of each waiting for the
      // previous (possibly aliasing) store
      double cv[4][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = bn + ty + 16 * j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = bm + tx + 16 * i;
          cv[i][j] = (c < N && r < M && (!lower || r >= c)) ? ldcg(C + (int64_t)c * ldc + r) : 0.0;
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = bn + ty + 16 * j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = bm + tx + 16 * i;
          if (c < N && r < M && (!lower || r >= c)) stcg(C + (int64_t)c * ldc + r, cv[i][j] - acc[i][j]);
        }
      }
    }
  }
  __syncthreads();
}

// C[M x N] -= A[M x K] * B[N x K]^T (the Cholesky updates)
static __device__ __forceinline__ void update_nt(double *C, int64_t ldc, const double *A, int64_t lda,
                                                 const double *B, int64_t ldb, int M, int N, int K,
                                                 bool lower, double *smem) {
  update_core<false>(C, ldc, A, lda, B, ldb, M, N, K, lower, smem);
}

// Quotient b / d from the correctly rounded reciprocal r = RN(1/d) with one correction step
// (Markstein, 1990): x = RN(b r); e = b - x d is exact with a fused multiply-add; RN(x + e r)
// is the correctly rounded quotient outside overflow and underflow. Three dependent
// operations instead of a full division on the substitution's critical chain; exact
// quotients (integer data) are recovered exactly.
__device__ __forceinline__ double quot(double b, double d, double r) {
  const double x = b * r;
  const double e = fma(-x, d, b);
  return fma(e, r, x);
}

// Forward substitution of one row against the pb x pb lower block D (shared, ld DS_LD):
// x D^T = b. Column-oriented: x_c = (b_c - sum_{m<c} x_m d_cm) / d_cc with the sum built up
// in increasing m as the x_m become known, so each x_c is at the end of a short chain.
// Row r of the panel P (column-major). Rinv holds 1/d_cc.
__device__ __forceinline__ void row_solve_lt(double *P, int64_t ldp, int r, int pb, const double *Ds,
                                             const double *Rinv) {
  double x[IB];
#pragma unroll
  for (int c = 0; c < IB; ++c) x[c] = c < pb ? ldcg(P + (int64_t)c * ldp + r) : 0.0;
#pragma unroll
  for (int c = 0; c < IB; ++c) {
    if (c < pb) {
      x[c] = quot(x[c], Ds[c * DS_LD + c], Rinv[c]);
#pragma unroll
      for (int m = c + 1; m < IB; ++m)
        if (m < pb) x[m] = fma(-x[c], Ds[m * DS_LD + c], x[m]);
    }
  }
#pragma unroll
  for (int c = 0; c < IB; ++c)
    if (c < pb) stcg(P + (int64_t)c * ldp + r, x[c]);
}

// Load the lower part of the pb x pb block at G (column-major, ld) into Ds (row-major).
__device__ __forceinline__ void load_diag_block(const double *G, int64_t ld, int pb, double *Ds) {
  for (int e = threadIdx.x; e < IB * IB; e += NT) {
    const int r = e & (IB - 1), c = e >> 5;
    Ds[r * DS_LD + c] = (r < pb && c < pb && r >= c) ? ldcg(G + (int64_t)c * ld + r) : 0.0;
  }
}

// POTRF on the nk x nk diagonal tile G (in place, lower). Returns 0, or the 1-based column
// inside the tile whose pivot is not positive (or NaN). Called by all threads.
//
// pw (32 or 64) is the width of the panel whose update of the trailing matrix is applied at
// once: 32-column blocks are factored and solved in turn, the later columns of the same panel
// updated right away, and the columns past the panel updated once per panel with K = pw, so
// with pw = 64 the trailing matrix is read and written half as often and the update runs two
// 32-deep chunks double-buffered. The same products are formed; only the order in which the
// two 32-column halves of a panel are subtracted from the trailing matrix changes.
static __device__ __noinline__ int potrf_tile(double *G, int64_t ld, int nk, double *smem, int pw = IB) {
  double *Ds = smem + STAGE_DOUBLES;
  double *Rinv = Ds + IB * DS_LD;
  __shared__ int s_fail;
  __shared__ int s_dfail[2];
  const int tid = threadIdx.x;
  for (int p = 0; p < nk; p += IB) {
    const int pb = min(IB, nk - p);
    const int pend = min(nk, (p / pw) * pw + pw);  // end of this block's panel
    double *Gpp = G + (int64_t)p * ld + p;
    load_diag_block(Gpp, ld, pb, Ds);
    if (tid == 0) s_fail = 0;
    __syncthreads();
    // unblocked right-looking factor of the pb x pb block by warps 0-3 (one per SM
    // sub-partition), lane r owns row r. Column j: warp j % 4 takes the square root and the
    // quotients l_rj; after a barrier of the four warps each updates the columns c = w mod 4
    // it owns with l_rj l_cj, so the 496 FMA instructions of the rank-one updates are spread
    // over four FP64 pipes instead of one. Every entry sees the same operations in the same
    // order as with one warp. The owner's failure flag is double-buffered by column parity,
    // so a warp that reads it late never sees the next column's.
    if (tid < 128) {
      const int r = tid & 31, w = tid >> 5;
      int fail = 0;
      for (int j = 0; j < pb; ++j) {
        if (w == (j & 3)) {
          const double s = Ds[j * DS_LD + j];
          int f = 0;
          if (!(s > 0.0)) {
            f = p + j + 1;
          } else {
            const double ljj = sqrt(s);
            if (r > j && r < pb) Ds[r * DS_LD + j] = Ds[r * DS_LD + j] / ljj;
            if (r == j) Ds[j * DS_LD + j] = ljj;
          }
          if (r == 0) s_dfail[j & 1] = f;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        fail = s_dfail[j & 1];
        if (fail) break;
        if (r > j && r < pb) {
          const double lrj = Ds[r * DS_LD + j];
          for (int c = j + 1 + ((w - j - 1) & 3); c <= r; c += 4)
            Ds[r * DS_LD + c] = fma(-lrj, Ds[c * DS_LD + j], Ds[r * DS_LD + c]);
        }
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (tid == 0) s_fail = fail;
      if (!fail && tid < pb) Rinv[tid] = 1.0 / Ds[tid * DS_LD + tid];
    }
    __syncthreads();
    if (s_fail) return s_fail;
    for (int e = tid; e < IB * IB; e += NT) {
      const int r = e & (IB - 1), c = e >> 5;
      if (r < pb && c < pb && r >= c) stcg(Gpp + (int64_t)c * ld + r, Ds[r * DS_LD + c]);
    }
    // panel below the diagonal block: rows p+pb..nk-1 of columns p..p+pb-1
    const int rows = nk - p - pb;
    double *Pn = G + (int64_t)p * ld + p + pb;
    for (int r0 = 0; r0 < rows; r0 += NT) {
      const int r = r0 + tid;
      if (r < rows) row_solve_lt(Pn, ld, r, pb, Ds, Rinv);
    }
    __syncthreads();
    // the panel's later columns now; the columns past the panel once the panel is complete
    const int pcols = pend - p - pb;
    if (rows > 0 && pcols > 0) {
      double *Gt = G + (int64_t)(p + pb) * ld + p + pb;
      update_nt(Gt, ld, Pn, ld, Pn, ld, rows, pcols, pb, true, smem);
    }
    if (p + pb == pend && nk > pend) {
      const int P0 = pend - ((pend - 1) % pw + 1);  // first column of the panel
      const int trail = nk - pend;
      double *Gt = G + (int64_t)pend * ld + pend;
      const double *Pp = G + (int64_t)P0 * ld + pend;
      update_nt(Gt, ld, Pp, ld, Pp, ld, trail, trail, pend - P0, true, smem);
    }
  }
  __syncthreads();
  return 0;
}

// TRSM: X L^T = B in place on B (mb x nk), L the nk x nk lower factor tile.
static __device__ __noinline__ void trsm_tile(double *B, int64_t ldb, const double *L, int64_t ldl,
                                       int mb, int nk, double *smem) {
  double *Ds = smem + STAGE_DOUBLES;
  double *Rinv = Ds + IB * DS_LD;
  const int tid = threadIdx.x;
  for (int p = 0; p < nk; p += IB) {
    const int pb = min(IB, nk - p);
    load_diag_block(L + (int64_t)p * ldl + p, ldl, pb, Ds);
    if (tid < pb) Rinv[tid] = 1.0 / ldcg(L + (int64_t)(p + tid) * ldl + p + tid);
    __syncthreads();
    double *Bp = B + (int64_t)p * ldb;
    for (int r0 = 0; r0 < mb; r0 += NT) {
      const int r = r0 + tid;
      if (r < mb) row_solve_lt(Bp, ldb, r, pb, Ds, Rinv);
    }
    __syncthreads();
    const int rest = nk - p - pb;
    if (rest > 0)
      update_nt(B + (int64_t)(p + pb) * ldb, ldb, Bp, ldb, L + (int64_t)p * ldl + p + pb, ldl, mb,
                rest, pb, false, smem);
  }
  __syncthreads();
}

}  // namespace chol
