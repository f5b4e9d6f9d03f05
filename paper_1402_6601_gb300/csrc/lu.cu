// Solve A X = B with the factors of the tile LU with incremental pivoting (chol_lu_factor).
//
// The factorization recorded, tile column by tile column, the transformation of GETRF(k)
// and then those of TSTRF(i, k), i > k, each a sequence of inner blocks (interchanges, unit
// lower L11, multipliers L21). Applying them to B in the same order gives U X = M B with U
// the upper triangle of the tiles (diagonal tiles' upper parts and the tiles right of the
// diagonal); back substitution with U finishes the solve.
//
// One block per group of LU_SOLVE_COLS right-hand sides runs the whole sequence for its
// columns (right-hand sides are independent). The tile row being transformed (Y_k) and the
// one it is paired with (Y_i) are staged in shared memory; per inner block the interchanges
// run one thread per column, the unit lower L11 solve one warp per column (lane = row), and
// the elimination of the paired rows one thread per (row, column). The back substitution
// sums U_kj Y_j with the columns split over the threads and four partial sums per thread,
// then solves the diagonal tile's upper triangle block by block, one warp per column.
#include <algorithm>
#include <mutex>
#include "common.cuh"
#include "internal.cuh"
#include "tiles_lu.cuh"

namespace chol {

constexpr int LU_SOLVE_COLS = 16;
constexpr int LU_SOLVE_SMEM_BYTES = (2 * LU_NB_MAX * LU_SOLVE_COLS + LU_IB * DS_LD + LU_IB) * 8 + LU_IB * 4;

struct LuSolveArgs {
  int n, nb, T, nrhs;
  const double *F;
  int64_t lda;
  const int *piv;
  const double *lw;
  double *B;
  int64_t ldb;
};

struct LuSolveSmem {
  double *yk, *yi, *l11, *rinv;
  int *piv;
};

__device__ __forceinline__ LuSolveSmem lu_solve_smem(unsigned char *raw) {
  LuSolveSmem s;
  double *d = reinterpret_cast<double *>(raw);
  s.yk = d;
  s.yi = d + LU_NB_MAX * LU_SOLVE_COLS;
  s.l11 = s.yi + LU_NB_MAX * LU_SOLVE_COLS;
  s.rinv = s.l11 + LU_IB * DS_LD;
  s.piv = reinterpret_cast<int *>(s.rinv + LU_IB);
  return s;
}

constexpr int SLD = LU_NB_MAX;  // staged rows are column-major with this leading dimension

// rows [r0, r0 + m) of g columns of Y (global, ld) <-> staged rows S[c * SLD + r]
__device__ __forceinline__ void lu_stage_in(const double *Y, int64_t ldy, int r0, int m, int g, double *S) {
  for (int e = threadIdx.x; e < m * g; e += NT) {
    const int c = e / m, r = e - c * m;
    S[c * SLD + r] = ldcg(Y + (int64_t)c * ldy + r0 + r);
  }
}
__device__ __forceinline__ void lu_stage_out(double *Y, int64_t ldy, int r0, int m, int g, const double *S) {
  for (int e = threadIdx.x; e < m * g; e += NT) {
    const int c = e / m, r = e - c * m;
    stcg(Y + (int64_t)c * ldy + r0 + r, S[c * SLD + r]);
  }
}

// One inner block's transformation on staged rows: X1s (w rows), X2s (mA rows), g columns;
// piv and L11 in shared memory, L21 (mA x w) in global memory. Ends synchronised.
__device__ void lu_solve_block(double *X1s, double *X2s, int w, int mA, const int *piv, const double *L11,
                               const double *L21, int64_t ldl, int g) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < g) {
    double *x1 = X1s + tid * SLD, *x2 = X2s + tid * SLD;
    for (int j = 0; j < w; ++j) {
      const int q = piv[j];
      if (q == j || q < 0 || q >= w + mA) continue;
      double *o = q < w ? x1 + q : x2 + (q - w);
      const double t = x1[j];
      x1[j] = *o;
      *o = t;
    }
  }
  __syncthreads();
  for (int c = warp; c < g; c += NT / 32) {
    double y = lane < w ? X1s[c * SLD + lane] : 0.0;
    for (int j = 0; j + 1 < w; ++j) {
      const double yj = __shfl_sync(0xffffffffu, y, j);
      if (lane > j && lane < w) y = fma(-L11[lane * DS_LD + j], yj, y);
    }
    if (lane < w) X1s[c * SLD + lane] = y;
  }
  __syncthreads();
  for (int e = tid; e < mA * g; e += NT) {
    const int c = e / mA, r = e - c * mA;
    double t = X2s[c * SLD + r];
    // the row of L21 is loaded in groups of eight before the products that use it
#pragma unroll
    for (int j0 = 0; j0 < LU_IB; j0 += 8) {
      double l[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) l[u] = j0 + u < w ? ldcg(L21 + (int64_t)(j0 + u) * ldl + r) : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < w) t = fma(-l[u], X1s[c * SLD + j0 + u], t);
    }
    X2s[c * SLD + r] = t;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT) lu_solve_kernel(const __grid_constant__ LuSolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const LuSolveSmem s = lu_solve_smem(smem_raw);
  constexpr int G = LU_SOLVE_COLS;
  static_assert(SLD * G <= LU_NB_MAX * LU_SOLVE_COLS, "staging buffers");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g0 = blockIdx.x * G;
  const int g = min(G, a.nrhs - g0);
  double *Y = a.B + (int64_t)g0 * a.ldb;
  const int nb = a.nb, T = a.T;
  const int64_t lda = a.lda, ldb = a.ldb;
  auto tile = [&](int i, int j) { return a.F + (int64_t)j * nb * lda + (int64_t)i * nb; };
  auto dim = [&](int t) { return min(nb, a.n - t * nb); };

  // Y <- M Y: the recorded transformations in factorization order
  for (int k = 0; k < T; ++k) {
    const int nk = dim(k);
    const double *Akk = tile(k, k);
    const int *pk = a.piv + ((int64_t)k * T + k) * nb;
    lu_stage_in(Y, ldb, k * nb, nk, g, s.yk);
    for (int c0 = 0; c0 < nk; c0 += LU_IB) {
      const int w = min(LU_IB, nk - c0), c1 = c0 + w;
      if (tid < w) s.piv[tid] = pk[c0 + tid];
      lu_load_l11(Akk + (int64_t)c0 * lda + c0, lda, w, s.l11);
      lu_solve_block(s.yk + c0, s.yk + c1, w, nk - c1, s.piv, s.l11, Akk + (int64_t)c0 * lda + c1, lda, g);
    }
    for (int i = k + 1; i < T; ++i) {
      const int mi = dim(i);
      const int *pik = a.piv + ((int64_t)k * T + i) * nb;
      const double *lw = a.lw + ((int64_t)k * T + i) * LU_IB * nb;
      const double *Aik = tile(i, k);
      lu_stage_in(Y, ldb, i * nb, mi, g, s.yi);
      for (int c0 = 0; c0 < nk; c0 += LU_IB) {
        const int w = min(LU_IB, nk - c0);
        if (tid < w) s.piv[tid] = pik[c0 + tid];
        lu_load_l11(lw + (int64_t)c0 * LU_IB, LU_IB, w, s.l11);
        lu_solve_block(s.yk + c0, s.yi, w, mi, s.piv, s.l11, Aik + (int64_t)c0 * lda, lda, g);
      }
      lu_stage_out(Y, ldb, i * nb, mi, g, s.yi);
      __syncthreads();
    }
    lu_stage_out(Y, ldb, k * nb, nk, g, s.yk);
    __syncthreads();
  }
  // U X = Y by tile rows from the bottom
  double *part = s.yi;  // partial sums, [part][row][col]
  for (int k = T - 1; k >= 0; --k) {
    const int nk = dim(k);
    const double *Akk = tile(k, k);
    lu_stage_in(Y, ldb, k * nb, nk, g, s.yk);
    const int q0 = (k + 1) * nb, nq = a.n - q0;  // columns of U right of the diagonal tile
    const int pairs = nk * g;
    const int parts = pairs >= NT ? 1 : min(NT / pairs, LU_NB_MAX * G / pairs);
    if (nq > 0) {
      for (int idx = tid; idx < pairs * parts; idx += NT) {
        const int p = idx / pairs, e = idx - p * pairs;
        const int c = e / nk, r = e - c * nk;
        const double *urow = a.F + (int64_t)q0 * lda + (int64_t)k * nb + r;  // U(k nb + r, q0 + q)
        const double *ycol = Y + (int64_t)c * ldb + q0;
        // eight products in flight per thread, four partial sums
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        int q = p;
        for (; q + 7 * parts < nq; q += 8 * parts) {
          double u[8], y[8];
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            u[v] = ldcg(urow + (int64_t)(q + v * parts) * lda);
            y[v] = ldcg(ycol + q + v * parts);
          }
#pragma unroll
          for (int v = 0; v < 8; ++v) t[v & 3] = fma(u[v], y[v], t[v & 3]);
        }
        for (; q < nq; q += parts) t[0] = fma(ldcg(urow + (int64_t)q * lda), ldcg(ycol + q), t[0]);
        part[p * pairs + e] = (t[0] + t[1]) + (t[2] + t[3]);
      }
      __syncthreads();
      for (int e = tid; e < pairs; e += NT) {
        const int c = e / nk, r = e - c * nk;
        double t = 0.0;
        for (int p = 0; p < parts; ++p) t += part[p * pairs + e];
        s.yk[c * SLD + r] -= t;
      }
      __syncthreads();
    }
    for (int c0 = ((nk - 1) / LU_IB) * LU_IB; c0 >= 0; c0 -= LU_IB) {
      const int w = min(LU_IB, nk - c0);
      const double *U = Akk + (int64_t)c0 * lda + c0;
      for (int e = tid; e < LU_IB * LU_IB; e += NT) {
        const int r = e & (LU_IB - 1), c = e >> 5;
        s.l11[r * DS_LD + c] = (r < w && c < w && c >= r) ? ldcg(U + (int64_t)c * lda + r) : 0.0;
      }
      __syncthreads();
      if (tid < w) s.rinv[tid] = 1.0 / s.l11[tid * DS_LD + tid];
      __syncthreads();
      for (int c = warp; c < g; c += NT / 32) {
        double x = lane < w ? s.yk[c * SLD + c0 + lane] : 0.0;
        for (int j = w - 1; j >= 0; --j) {
          if (lane == j) x = quot(x, s.l11[j * DS_LD + j], s.rinv[j]);
          const double xj = __shfl_sync(0xffffffffu, x, j);
          if (lane < j) x = fma(-s.l11[lane * DS_LD + j], xj, x);
        }
        if (lane < w) s.yk[c * SLD + c0 + lane] = x;
      }
      __syncthreads();
      for (int e = tid; e < c0 * g; e += NT) {  // rows above the block inside the tile
        const int c = e / c0, r = e - c * c0;
        double t = s.yk[c * SLD + r];
        for (int j = 0; j < w; ++j) t = fma(-ldcg(Akk + (int64_t)(c0 + j) * lda + r), s.yk[c * SLD + c0 + j], t);
        s.yk[c * SLD + r] = t;
      }
      __syncthreads();
    }
    lu_stage_out(Y, ldb, k * nb, nk, g, s.yk);
    __syncthreads();
  }
}

}  // namespace chol

using namespace chol;

extern "C" chol_status chol_lu_solve(int n, int nrhs, const double *dF, int lda, const int *dPiv, const double *dLw,
                                     const chol_opts *opts, double *dB, int ldb, void *stream) {
  if (n < 0 || nrhs < 0) return CHOL_ERR_INVALID_ARG;
  const int nb = lu_tile_size(n, opts);
  if (nb <= 0) return CHOL_ERR_INVALID_ARG;
  if (n == 0 || nrhs == 0) return CHOL_OK;
  if (lda < n || ldb < n || !dF || !dPiv || !dLw || !dB) return CHOL_ERR_INVALID_ARG;
  const DeviceInfo di = current_device_info();
  if (di.sms <= 0) return CHOL_ERR_CUDA;
  if (di.cc_major != 10 || di.cc_minor != 3) return CHOL_ERR_UNSUPPORTED;
  CHOL_CUDA_TRY(set_smem_attr((const void *)lu_solve_kernel, LU_SOLVE_SMEM_BYTES));
  LuSolveArgs a;
  a.n = n;
  a.nb = nb;
  a.T = (n + nb - 1) / nb;
  a.nrhs = nrhs;
  a.F = dF;
  a.lda = lda;
  a.piv = dPiv;
  a.lw = dLw;
  a.B = dB;
  a.ldb = ldb;
  const int grid = (nrhs + LU_SOLVE_COLS - 1) / LU_SOLVE_COLS;
  lu_solve_kernel<<<grid, NT, LU_SOLVE_SMEM_BYTES, (cudaStream_t)stream>>>(a);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}
