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
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = bn + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
        if (c >= N) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = bm + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
          if (r < M && (!lower || r >= c)) {
            float *cp = C + (int64_t)c * ldc + r;
            stcg(cp, ldcg(cp) - acc[i][j]);
          }
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

}  // namespace f32
}  // namespace chol
