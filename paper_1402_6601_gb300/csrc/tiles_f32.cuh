// FP32 tile task bodies (the low-precision factor of the mixed-precision solver), executed
// by one 256-thread block at a time, like the FP64 bodies.
//
// FP32 FMA runs 64 times faster than FP64 on sm_103 (128 vs 2 per clock per SM), so here the
// contraction must reuse operands much harder: 128 x 128 output blocks, an 8 x 8 register
// tile per thread (two 4-wide strips in each direction, read from shared memory as float4),
// 16-deep k chunks double-buffered through registers. Per k step a warp issues 64 FFMA
// against 4 shared-memory vector loads.
#pragma once
#include <stdint.h>

namespace chol {
namespace f32 {

constexpr int NT = 256;
constexpr int BM = 128, BN = 128, BK = 16;
constexpr int IB = 32;
constexpr int DS_LD = IB + 1;
constexpr int STAGE_FLOATS = 2 * BK * BM + 2 * BK * BN;
constexpr int TILE_SMEM_BYTES = (STAGE_FLOATS + IB * DS_LD + IB) * 4;

__device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(float *p, float v) { __stcg(p, v); }

// C[M x N] -= A[M x K] * B[N x K]^T, column-major; `lower` writes only row >= column.
static __device__ __noinline__ void update_nt(float *C, int64_t ldc, const float *A, int64_t lda, const float *B,
                                       int64_t ldb, int M, int N, int K, bool lower, float *smem) {
  float *As = smem;
  float *Bs = smem + 2 * BK * BM;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int lrow = tid & 127, lk = tid >> 7;  // loader: row lrow, k = lk + 2q
  for (int bn = 0; bn < N; bn += BN) {
    for (int bm = 0; bm < M; bm += BM) {
      if (lower && bm + BM <= bn) continue;
      float acc[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
      float ra[8], rb[8];
      const bool arow = bm + lrow < M, brow = bn + lrow < N;
      const float *Ap = A + bm + lrow;
      const float *Bp = B + bn + lrow;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int kk = lk + 2 * q;
        ra[q] = (arow && kk < K) ? ldcg(Ap + (int64_t)kk * lda) : 0.f;
        rb[q] = (brow && kk < K) ? ldcg(Bp + (int64_t)kk * ldb) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        As[(lk + 2 * q) * BM + lrow] = ra[q];
        Bs[(lk + 2 * q) * BN + lrow] = rb[q];
      }
      __syncthreads();
      int buf = 0;
      for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int kk = k0 + BK + lk + 2 * q;
            ra[q] = (arow && kk < K) ? ldcg(Ap + (int64_t)kk * lda) : 0.f;
            rb[q] = (brow && kk < K) ? ldcg(Bp + (int64_t)kk * ldb) : 0.f;
          }
        }
        const float *as = As + buf * BK * BM;
        const float *bs = Bs + buf * BK * BN;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          const float4 a0 = *reinterpret_cast<const float4 *>(as + kk * BM + tx * 4);
          const float4 a1 = *reinterpret_cast<const float4 *>(as + kk * BM + 64 + tx * 4);
          const float4 b0 = *reinterpret_cast<const float4 *>(bs + kk * BN + ty * 4);
          const float4 b1 = *reinterpret_cast<const float4 *>(bs + kk * BN + 64 + ty * 4);
          const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
          float *an = As + (buf ^ 1) * BK * BM;
          float *bnx = Bs + (buf ^ 1) * BK * BN;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            an[(lk + 2 * q) * BM + lrow] = ra[q];
            bnx[(lk + 2 * q) * BN + lrow] = rb[q];
          }
        }
        __syncthreads();
        buf ^= 1;
      }
      // all loads of C first, then the stores: interleaved, every read would wait for the
      // previous store (possible aliasing) and the epilogue would cost 64 L2 round trips
      float cv[8][8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = bn + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = bm + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
          cv[i][j] = (c < N && r < M && (!lower || r >= c)) ? ldcg(C + (int64_t)c * ldc + r) : 0.f;
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = bn + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = bm + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
          if (c < N && r < M && (!lower || r >= c)) stcg(C + (int64_t)c * ldc + r, cv[i][j] - acc[i][j]);
        }
      }
    }
  }
  __syncthreads();
}

// b / d from r = RN(1/d) with one Markstein correction step.
__device__ __forceinline__ float quot(float b, float d, float r) {
  const float x = b * r;
  const float e = fmaf(-x, d, b);
  return fmaf(e, r, x);
}

// One row of X D^T = P against the pb x pb lower block D (shared), column-oriented.
__device__ __forceinline__ void row_solve_lt(float *P, int64_t ldp, int r, int pb, const float *Ds,
                                             const float *Rinv) {
  float x[IB];
#pragma unroll
  for (int c = 0; c < IB; ++c) x[c] = c < pb ? ldcg(P + (int64_t)c * ldp + r) : 0.f;
#pragma unroll
  for (int c = 0; c < IB; ++c) {
    if (c < pb) {
      x[c] = quot(x[c], Ds[c * DS_LD + c], Rinv[c]);
#pragma unroll
      for (int m = c + 1; m < IB; ++m)
        if (m < pb) x[m] = fmaf(-x[c], Ds[m * DS_LD + c], x[m]);
    }
  }
#pragma unroll
  for (int c = 0; c < IB; ++c)
    if (c < pb) stcg(P + (int64_t)c * ldp + r, x[c]);
}

__device__ __forceinline__ void load_diag_block(const float *G, int64_t ld, int pb, float *Ds) {
  for (int e = threadIdx.x; e < IB * IB; e += NT) {
    const int r = e & (IB - 1), c = e >> 5;
    Ds[r * DS_LD + c] = (r < pb && c < pb && r >= c) ? ldcg(G + (int64_t)c * ld + r) : 0.f;
  }
}

// POTRF on the nk x nk diagonal tile (FP32); returns 0 or the failing 1-based column.
static __device__ __noinline__ int potrf_tile(float *G, int64_t ld, int nk, float *smem) {
  float *Ds = smem + STAGE_FLOATS;
  float *Rinv = Ds + IB * DS_LD;
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  for (int p = 0; p < nk; p += IB) {
    const int pb = min(IB, nk - p);
    float *Gpp = G + (int64_t)p * ld + p;
    load_diag_block(Gpp, ld, pb, Ds);
    if (tid == 0) s_fail = 0;
    __syncthreads();
    if (tid < 32) {
      // lane r keeps row r of the block in registers (rows/columns past pb form an identity),
      // the pivot column is scaled in place and broadcast by shuffles for the rank-1 update
      const int r = tid;
      float x[IB];
#pragma unroll
      for (int c = 0; c < IB; ++c) x[c] = (r < pb && c <= r) ? Ds[r * DS_LD + c] : (r == c ? 1.f : 0.f);
      int fail = 0;
#pragma unroll
      for (int j = 0; j < IB; ++j) {
        const float s = __shfl_sync(0xffffffffu, x[j], j);
        if (!fail && !(s > 0.f)) fail = p + j + 1;  // the same s on every lane
        const float ljj = sqrtf(s > 0.f ? s : 1.f);
        const float lrj = r == j ? ljj : (r > j ? x[j] / ljj : x[j]);
        x[j] = lrj;
#pragma unroll
        for (int c = j + 1; c < IB; ++c) {
          const float lcj = __shfl_sync(0xffffffffu, lrj, c);
          if (r >= c) x[c] = fmaf(-lrj, lcj, x[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < IB; ++c)
        if (r < pb && c <= r) Ds[r * DS_LD + c] = x[c];
      if (r == 0) s_fail = fail;
      if (!fail && r < pb) Rinv[r] = 1.f / x[r];
    }
    __syncthreads();
    if (s_fail) return s_fail;
    for (int e = tid; e < IB * IB; e += NT) {
      const int r = e & (IB - 1), c = e >> 5;
      if (r < pb && c < pb && r >= c) stcg(Gpp + (int64_t)c * ld + r, Ds[r * DS_LD + c]);
    }
    const int rows = nk - p - pb;
    float *Pn = G + (int64_t)p * ld + p + pb;
    for (int r0 = 0; r0 < rows; r0 += NT) {
      const int r = r0 + tid;
      if (r < rows) row_solve_lt(Pn, ld, r, pb, Ds, Rinv);
    }
    __syncthreads();
    if (rows > 0) update_nt(G + (int64_t)(p + pb) * ld + p + pb, ld, Pn, ld, Pn, ld, rows, rows, pb, true, smem);
  }
  __syncthreads();
  return 0;
}

// TRSM: X L^T = B in place on B (mb x nk).
static __device__ __noinline__ void trsm_tile(float *B, int64_t ldb, const float *L, int64_t ldl, int mb, int nk,
                                       float *smem) {
  float *Ds = smem + STAGE_FLOATS;
  float *Rinv = Ds + IB * DS_LD;
  const int tid = threadIdx.x;
  for (int p = 0; p < nk; p += IB) {
    const int pb = min(IB, nk - p);
    load_diag_block(L + (int64_t)p * ldl + p, ldl, pb, Ds);
    if (tid < pb) Rinv[tid] = 1.f / ldcg(L + (int64_t)(p + tid) * ldl + p + tid);
    __syncthreads();
    float *Bp = B + (int64_t)p * ldb;
    for (int r0 = 0; r0 < mb; r0 += NT) {
      const int r = r0 + tid;
      if (r < mb) row_solve_lt(Bp, ldb, r, pb, Ds, Rinv);
    }
    __syncthreads();
    const int rest = nk - p - pb;
    if (rest > 0)
      update_nt(B + (int64_t)(p + pb) * ldb, ldb, Bp, ldb, L + (int64_t)p * ldl + p + pb, ldl, mb, rest, pb, false,
                smem);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// Shared-memory resident POTRF for tiles of order <= PANEL_MAX_N. The diagonal tasks form
// the factorization's critical path, and the blocked version above spends its time in
// latency: after each 32-column step it re-reads and re-writes the trailing tile through L2.
// Here the lower triangle of the tile is read once into shared memory as 32 x 32 blocks, the
// right-looking factorization runs there (diagonal block in warp 0's registers, the rows
// below solved one per thread, the trailing blocks updated with 4 x 8 register tiles per
// lane), and the factor is written back once.

constexpr int PANEL_MAX_N = 256;
constexpr int NBLK_MAX = PANEL_MAX_N / IB;  // 8 block rows
constexpr int SB_LD = IB + 4;               // column-major 32 x 32 block, 16-byte aligned columns
constexpr int SB_FLOATS = IB * SB_LD;
constexpr int PANEL_SMEM_BYTES = (NBLK_MAX * (NBLK_MAX + 1) / 2 * SB_FLOATS + IB) * 4;

// lower block (i, j), i >= j, of the shared-memory tile
__device__ __forceinline__ float *sblk(float *S, int i, int j) { return S + (i * (i + 1) / 2 + j) * SB_FLOATS; }

// Factor the 32 x 32 block Db (column-major, ld SB_LD) in warp 0's registers, lane r holding
// row r; rows and columns at or past pb are an identity. Writes L and Rinv = 1 / diag(L).
// Returns 0 or the 1-based failing column offset by p. Warp 0 only.
//
// The loop is one dependent chain per column, so it is kept short: the square root and the
// correctly rounded reciprocal square root are taken side by side from the pivot, the
// column is scaled by a corrected quotient, and every lane runs the same unpredicated
// update (lanes above the diagonal compute values in the upper triangle that are never read
// or stored).
__device__ __forceinline__ int warp_diag_factor_cm(float *Db, float *Rinv, int pb, int p) {
  const int r = threadIdx.x;
  float x[IB];
#pragma unroll
  for (int c = 0; c < IB; ++c) x[c] = (r < pb && c <= r) ? Db[c * SB_LD + r] : (r == c ? 1.f : 0.f);
  int fail = 0;
#pragma unroll
  for (int j = 0; j < IB; ++j) {
    const float s = __shfl_sync(0xffffffffu, x[j], j);
    if (!fail && !(s > 0.f)) fail = p + j + 1;  // the same s on every lane
    const float sp = s > 0.f ? s : 1.f;
    const float ljj = sqrtf(sp);
    const float rj = __frsqrt_rn(sp);
    const float lrj = r == j ? ljj : quot(x[j], ljj, rj);
    x[j] = lrj;
#pragma unroll
    for (int c = j + 1; c < IB; ++c) x[c] = fmaf(-lrj, __shfl_sync(0xffffffffu, lrj, c), x[c]);
  }
#pragma unroll
  for (int c = 0; c < IB; ++c)
    if (c <= r) Db[c * SB_LD + r] = x[c];
  float d = x[0];
#pragma unroll
  for (int c = 1; c < IB; ++c) d = r == c ? x[c] : d;
  Rinv[r] = __frcp_rn(d);
  return fail;
}

// POTRF of the nk x nk tile G (nk <= PANEL_MAX_N) in shared memory; returns 0 or the failing
// 1-based column. Called by all threads.
static __device__ __noinline__ int potrf_tile_smem(float *G, int64_t ld, int nk, float *smem) {
  float *S = smem;
  float *Rinv = smem + NBLK_MAX * (NBLK_MAX + 1) / 2 * SB_FLOATS;
  __shared__ int s_fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (nk + IB - 1) / IB;
  const int nlow = nblk * (nblk + 1) / 2;
  // whole-column vectors of 4 rows can be moved as float4 when every column start is aligned
  const bool vec = ((reinterpret_cast<uintptr_t>(G) | (uintptr_t)(ld * 4)) & 15) == 0;
  // load: element (r, c) of block (i, j) is A(32i + r, 32j + c); entries outside the tile form
  // an identity, entries above the diagonal are zero
  // four vectors in flight per thread: the loads of a group are issued before any is stored
  for (int e0 = tid; e0 < nlow * IB * 8; e0 += 4 * NT) {
    float4 t[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const int e = e0 + g * NT;
      t[g] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < nlow * IB * 8) {
        const int q = e & 7, c = (e >> 3) & (IB - 1), b = e >> 8;
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= b) ++i;
        const int j = b - i * (i + 1) / 2;
        const int gr = IB * i + 4 * q, gc = IB * j + c;
        if (vec && gr + 3 < nk && gc < nk && (i > j || 4 * q >= c)) {
          t[g] = __ldcg(reinterpret_cast<const float4 *>(G + (int64_t)gc * ld + gr));
        } else {
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = gr + u;
            v[u] = (r < nk && gc < nk) ? (r >= gc ? ldcg(G + (int64_t)gc * ld + r) : 0.f) : (r == gc ? 1.f : 0.f);
          }
          t[g] = make_float4(v[0], v[1], v[2], v[3]);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const int e = e0 + g * NT;
      if (e < nlow * IB * 8) {
        const int q = e & 7, c = (e >> 3) & (IB - 1), b = e >> 8;
        *reinterpret_cast<float4 *>(S + b * SB_FLOATS + c * SB_LD + 4 * q) = t[g];
      }
    }
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; j < nblk; ++j) {
    const int pb = min(IB, nk - IB * j);
    if (warp == 0) {
      const int f = warp_diag_factor_cm(sblk(S, j, j), Rinv, pb, IB * j);
      if (lane == 0 && f) s_fail = f;
    }
    __syncthreads();
    if (s_fail) return s_fail;
    const float *D = sblk(S, j, j);
    const int below = nblk - j - 1;
    // rows of the blocks below the diagonal block: x D^T = b, one row per thread
    if (tid < below * IB) {
      float *P = sblk(S, j + 1 + (tid >> 5), j) + lane;
      float x[IB];
#pragma unroll
      for (int c = 0; c < IB; ++c) x[c] = P[c * SB_LD];
#pragma unroll
      for (int c = 0; c < IB; ++c) {
        x[c] = quot(x[c], D[c * SB_LD + c], Rinv[c]);
        // column c of D below the diagonal, four rows per (broadcast) vector load
#pragma unroll
        for (int m4 = (c + 1) & ~3; m4 < IB; m4 += 4) {
          const float4 d = *reinterpret_cast<const float4 *>(D + c * SB_LD + m4);
          if (m4 > c) x[m4] = fmaf(-x[c], d.x, x[m4]);
          if (m4 + 1 > c) x[m4 + 1] = fmaf(-x[c], d.y, x[m4 + 1]);
          if (m4 + 2 > c) x[m4 + 2] = fmaf(-x[c], d.z, x[m4 + 2]);
          x[m4 + 3] = fmaf(-x[c], d.w, x[m4 + 3]);
        }
      }
#pragma unroll
      for (int c = 0; c < IB; ++c) P[c * SB_LD] = x[c];
    }
    __syncthreads();
    // trailing blocks (i, m), j < m <= i < nblk: C -= L(i, j) L(m, j)^T, one block per warp
    // at a time; lane: rows 4 rg .. 4 rg + 3, columns 8 cg .. 8 cg + 7
    const int npair = below * (below + 1) / 2;
    const int rg = lane & 7, cg = lane >> 3;
    for (int t = warp; t < npair; t += NT / 32) {
      int ii = 0;
      while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
      const int i = j + 1 + ii, m = j + 1 + (t - ii * (ii + 1) / 2);
      const float *Ai = sblk(S, i, j) + 4 * rg;
      const float *Bm = sblk(S, m, j) + 8 * cg;
      float *C = sblk(S, i, m) + 8 * cg * SB_LD + 4 * rg;
      float acc[4][8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 v = *reinterpret_cast<const float4 *>(C + c * SB_LD);
        acc[0][c] = v.x; acc[1][c] = v.y; acc[2][c] = v.z; acc[3][c] = v.w;
      }
#pragma unroll 8
      for (int k = 0; k < IB; ++k) {
        const float4 a = *reinterpret_cast<const float4 *>(Ai + k * SB_LD);
        const float4 b0 = *reinterpret_cast<const float4 *>(Bm + k * SB_LD);
        const float4 b1 = *reinterpret_cast<const float4 *>(Bm + k * SB_LD + 4);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[u][c] = fmaf(-av[u], bv[c], acc[u][c]);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<float4 *>(C + c * SB_LD) = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
    }
    __syncthreads();
  }
  // write the factor back: the lower triangle of the tile only
  for (int e = tid; e < nlow * IB * 8; e += NT) {
    const int q = e & 7, c = (e >> 3) & (IB - 1), b = e >> 8;
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    const int j = b - i * (i + 1) / 2;
    const int gr = IB * i + 4 * q, gc = IB * j + c;
    if (gc >= nk) continue;
    const float4 t = *reinterpret_cast<const float4 *>(S + b * SB_FLOATS + c * SB_LD + 4 * q);
    if (vec && gr + 3 < nk && (i > j || 4 * q >= c)) {
      __stcg(reinterpret_cast<float4 *>(G + (int64_t)gc * ld + gr), t);
    } else {
      const float v[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (gr + u < nk && gr + u >= gc) stcg(G + (int64_t)gc * ld + gr + u, v[u]);
    }
  }
  __syncthreads();
  return 0;
}

// Receivers of the finished 32-column blocks of the band TRSM's rows (see trsm_band); the
// default does nothing.
constexpr int TR_LD = IB + 4;

struct NoEmit {
  __device__ void row(int, int, const float (&)[IB]) const {}
  __device__ void zero(int, int) const {}
  __device__ void flush(int) const {}
  __device__ void finish() const {}
};

// TRSM X L^T = B for one band of at most 64 rows of a panel tile (nk <= PANEL_MAX_N): the
// body of every FP32 TRSM, run band by band by one worker or as the units of a split task.
// Four threads per row, one part of the k range each (t = 64 part + row, so the 32 lanes of a
// warp share their part and every read of L is a broadcast): for each 32-column block j0 the
// parts accumulate sum_k X(row, k) L(j0 + c, k) over their own 8-wide chunks (chunk q goes to
// part q mod 4), parts 1..3 leave their sums in shared memory, and part 0 adds them in part
// order, subtracts from B(row, j0 + c) and solves the 32 x 32 diagonal block (right-looking,
// corrected quotients). The band's rows live in shared memory for the whole task, so the
// solved values are never read back from L2. `emit` gets every finished 32-column block
// of each row (emit.row / emit.zero for rows past `rows`, then emit.flush; emit.finish at the end).
constexpr int BAND_ROWS = 64;
constexpr int BX_LD = PANEL_MAX_N + 4;  // row stride of the band's rows (16-byte aligned)
constexpr int PS_LD = IB + 1;           // stride of the parts' partial sums (one row each)
constexpr int TRSM_BAND_SMEM_BYTES = (BAND_ROWS * BX_LD + 2 * PANEL_MAX_N * TR_LD + IB + 3 * BAND_ROWS * PS_LD) * 4;

// Columns j0 .. j0 + 31 of L (rows k < j0 + 32) into Lp[k * TR_LD + c] = L(j0 + c, k): 16-byte
// asynchronous copies (cp.async, completed with the calling thread's wait_group) for whole
// 4-column pieces inside the tile, plain stores of the identity padding past it. The strict
// upper part of the diagonal 32 x 32 block arrives as whatever the tile holds there and is
// cleared by trsm_band_fix once the copies have landed.
__device__ __forceinline__ void trsm_band_stage(float *Lp, const float *L, int64_t ldl, int j0, int nk) {
  const int jb = min(IB, nk - j0);
  for (int idx = threadIdx.x; idx < (j0 + IB) * (IB / 4); idx += NT) {
    const int k = idx >> 3, c4 = (idx & 7) * 4;
    float *dst = Lp + k * TR_LD + c4;
    const float *src = L + (int64_t)k * ldl + j0 + c4;
    // (any leading dimension and tile size are allowed: a piece that does not start on a
    // 16-byte boundary is loaded element by element)
    if (c4 + 4 <= jb && k < nk && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c4 + u;
        dst[u] = (c < jb && k <= j0 + c) ? ldcg(L + (int64_t)k * ldl + j0 + c) : (k == j0 + c ? 1.f : 0.f);
      }
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void trsm_band_fix(float *Lp, float *Rinv, int j0, int nk) {
  const int jb = min(IB, nk - j0);
  for (int e = threadIdx.x; e < IB * IB; e += NT) {
    const int c = e & (IB - 1), kr = e >> 5;  // row k = j0 + kr of the diagonal block
    if (c < kr && c < jb) Lp[(j0 + kr) * TR_LD + c] = 0.f;
  }
  if (threadIdx.x < IB) {
    const int c = threadIdx.x;
    Rinv[c] = c < jb ? __frcp_rn(Lp[(j0 + c) * TR_LD + c]) : 1.f;
  }
}

template <class Emit = NoEmit>
static __device__ __noinline__ void trsm_band(float *B, int64_t ldb, const float *L, int64_t ldl, int rows, int nk,
                                              float *smem, Emit emit = Emit()) {
  float *Xs = smem;                          // Xs[row * BX_LD + k]: B, then X as it is solved
  float *Lbuf = smem + BAND_ROWS * BX_LD;    // two Lp buffers, Lp[k * TR_LD + c] = L(j0 + c, k)
  float *Rinv = Lbuf + 2 * PANEL_MAX_N * TR_LD;
  float *Ps = Rinv + IB;                     // Ps[((part - 1) * BAND_ROWS + row) * PS_LD + c]
  const int tid = threadIdx.x, row = tid & (BAND_ROWS - 1), part = tid >> 6;
  static_assert(NT == 4 * BAND_ROWS, "four threads per row");
  const int nk32 = (nk + IB - 1) / IB * IB;  // columns past nk stay zero
  trsm_band_stage(Lbuf, L, ldl, 0, nk);
  for (int e = tid; e < BAND_ROWS * nk32; e += NT) {
    const int r = e % BAND_ROWS, c = e / BAND_ROWS;
    Xs[r * BX_LD + c] = (r < rows && c < nk) ? ldcg(B + (int64_t)c * ldb + r) : 0.f;
  }
  for (int j0 = 0; j0 < nk; j0 += IB) {
    const int jb = min(IB, nk - j0);
    float *Lp = Lbuf + ((j0 / IB) & 1) * PANEL_MAX_N * TR_LD;
    __syncthreads();  // everyone is done with the other buffer (block j0 - 32)
    if (j0 + IB < nk) {
      trsm_band_stage(Lbuf + ((j0 / IB + 1) & 1) * PANEL_MAX_N * TR_LD, L, ldl, j0 + IB, nk);
      asm volatile("cp.async.wait_group 1;" ::: "memory");  // this block's copies, not the next's
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();  // every thread's copies of this block have landed
    trsm_band_fix(Lp, Rinv, j0, nk);
    __syncthreads();
    const float *x = Xs + row * BX_LD;
    float acc[IB];
#pragma unroll
    for (int c = 0; c < IB; ++c) acc[c] = 0.f;
    for (int k0 = 8 * part; k0 < j0; k0 += 32) {
      const float4 xa = *reinterpret_cast<const float4 *>(x + k0);
      const float4 xb = *reinterpret_cast<const float4 *>(x + k0 + 4);
      const float xk[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
      for (int u = 0; u < 8; ++u) {
#pragma unroll
        for (int c4 = 0; c4 < IB; c4 += 4) {
          const float4 l = *reinterpret_cast<const float4 *>(Lp + (k0 + u) * TR_LD + c4);
          acc[c4] = fmaf(xk[u], l.x, acc[c4]);
          acc[c4 + 1] = fmaf(xk[u], l.y, acc[c4 + 1]);
          acc[c4 + 2] = fmaf(xk[u], l.z, acc[c4 + 2]);
          acc[c4 + 3] = fmaf(xk[u], l.w, acc[c4 + 3]);
        }
      }
    }
    if (part > 0) {
      float *ps = Ps + ((part - 1) * BAND_ROWS + row) * PS_LD;
#pragma unroll
      for (int c = 0; c < IB; ++c) ps[c] = acc[c];
    }
    __syncthreads();
    if (part == 0) {
      float v[IB];
#pragma unroll
      for (int c = 0; c < IB; ++c) {
        const float s = ((acc[c] + Ps[row * PS_LD + c]) + Ps[(BAND_ROWS + row) * PS_LD + c]) +
                        Ps[(2 * BAND_ROWS + row) * PS_LD + c];
        v[c] = x[j0 + c] - s;
      }
      // v D^T = b with D(c, m) = Lp[(j0 + m) * TR_LD + c]
      const float *D = Lp + j0 * TR_LD;
#pragma unroll
      for (int m = 0; m < IB; ++m) {
        v[m] = quot(v[m], D[m * TR_LD + m], Rinv[m]);
#pragma unroll
        for (int c4 = (m + 1) & ~3; c4 < IB; c4 += 4) {
          const float4 d = *reinterpret_cast<const float4 *>(D + m * TR_LD + c4);
          if (c4 > m) v[c4] = fmaf(-v[m], d.x, v[c4]);
          if (c4 + 1 > m) v[c4 + 1] = fmaf(-v[m], d.y, v[c4 + 1]);
          if (c4 + 2 > m) v[c4 + 2] = fmaf(-v[m], d.z, v[c4 + 2]);
          v[c4 + 3] = fmaf(-v[m], d.w, v[c4 + 3]);
        }
      }
      float *xw = Xs + row * BX_LD + j0;
#pragma unroll
      for (int c = 0; c < IB; ++c) xw[c] = c < jb ? v[c] : 0.f;
      if (row < rows) {
#pragma unroll
        for (int c = 0; c < IB; ++c)
          if (c < jb) stcg(B + (int64_t)(j0 + c) * ldb + row, v[c]);
        emit.row(row, j0 / IB, v);
      } else {
        emit.zero(row, j0 / IB);
      }
    }
    emit.flush(j0 / IB);
  }
  emit.finish();
  __syncthreads();
}

}  // namespace f32
}  // namespace chol
