// Solve A X = B with the factors of the tile LU with incremental pivoting (chol_lu_factor).
//
// The factorization recorded, tile column by tile column, the transformation of GETRF(k)
// and then those of TSTRF(i, k), i > k, each a sequence of inner blocks (interchanges, unit
// lower L11, multipliers L21). Applying them to B in the same order gives U X = M B with U
// the upper triangle of the tiles (diagonal tiles' upper parts and the tiles right of the
// diagonal); back substitution with U finishes the solve.
//
// One block per group of LU_SOLVE_COLS right-hand sides runs the whole sequence for its
// columns (right-hand sides are independent), with the block transformation and the DFMA
// tile update of the factorization's kernels.
#include <algorithm>
#include <mutex>
#include "common.cuh"
#include "internal.cuh"
#include "tiles_lu.cuh"

namespace chol {

constexpr int LU_SOLVE_COLS = 64;

struct LuSolveArgs {
  int n, nb, T, nrhs;
  const double *F;
  int64_t lda;
  const int *piv;
  const double *lw;
  double *B;
  int64_t ldb;
};

__global__ void __launch_bounds__(NT) lu_solve_kernel(const __grid_constant__ LuSolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *smem = reinterpret_cast<double *>(smem_raw);
  __shared__ double s_rinv[LU_IB];
  const LuSmem s = lu_smem(smem);
  const int tid = threadIdx.x;
  const int g0 = blockIdx.x * LU_SOLVE_COLS;
  const int g = min(LU_SOLVE_COLS, a.nrhs - g0);
  double *Y = a.B + (int64_t)g0 * a.ldb;
  const int nb = a.nb, T = a.T;
  const int64_t lda = a.lda, ldb = a.ldb;
  auto tile = [&](int i, int j) { return const_cast<double *>(a.F) + (int64_t)j * nb * lda + (int64_t)i * nb; };
  auto dim = [&](int t) { return min(nb, a.n - t * nb); };

  // Y <- M Y: the recorded transformations in factorization order
  for (int k = 0; k < T; ++k) {
    const int nk = dim(k);
    double *Akk = tile(k, k);
    double *Yk = Y + (int64_t)k * nb;
    const int *pk = a.piv + ((int64_t)k * T + k) * nb;
    for (int c0 = 0; c0 < nk; c0 += LU_IB) {
      const int w = min(LU_IB, nk - c0), c1 = c0 + w;
      if (tid < w) s.piv[tid] = pk[c0 + tid];
      lu_load_l11(Akk + (int64_t)c0 * lda + c0, lda, w, s.l11);
      lu_apply_block(Yk + c0, ldb, Yk + c1, ldb, g, w, s.piv, s.l11, nk - c1, Akk + (int64_t)c0 * lda + c1, lda,
                     s.work);
    }
    for (int i = k + 1; i < T; ++i) {
      const int mi = dim(i);
      const int *pik = a.piv + ((int64_t)k * T + i) * nb;
      const double *lw = a.lw + ((int64_t)k * T + i) * LU_IB * nb;
      double *Aik = tile(i, k);
      for (int c0 = 0; c0 < nk; c0 += LU_IB) {
        const int w = min(LU_IB, nk - c0);
        if (tid < w) s.piv[tid] = pik[c0 + tid];
        lu_load_l11(lw + (int64_t)c0 * LU_IB, LU_IB, w, s.l11);
        lu_apply_block(Yk + c0, ldb, Y + (int64_t)i * nb, ldb, g, w, s.piv, s.l11, mi, Aik + (int64_t)c0 * lda,
                       lda, s.work);
      }
    }
  }
  // U X = Y by tile rows from the bottom: Y_k -= U_kj X_j (j > k), then the diagonal tile's
  // upper triangle by inner blocks from the last
  for (int k = T - 1; k >= 0; --k) {
    const int nk = dim(k);
    double *Akk = tile(k, k);
    double *Yk = Y + (int64_t)k * nb;
    for (int j = k + 1; j < T; ++j)
      update_core<true>(Yk, ldb, tile(k, j), lda, Y + (int64_t)j * nb, ldb, nk, g, dim(j), false, s.work);
    for (int c0 = ((nk - 1) / LU_IB) * LU_IB; c0 >= 0; c0 -= LU_IB) {
      const int w = min(LU_IB, nk - c0);
      const double *U = Akk + (int64_t)c0 * lda + c0;
      for (int e = tid; e < LU_IB * LU_IB; e += NT) {
        const int r = e & (LU_IB - 1), c = e >> 5;
        s.l11[r * DS_LD + c] = (r < w && c < w && c >= r) ? ldcg(U + (int64_t)c * lda + r) : 0.0;
      }
      if (tid < w) s_rinv[tid] = 1.0 / ldcg(U + (int64_t)tid * lda + tid);
      __syncthreads();
      double *Xs = s.work;  // w x g, row-major
      for (int c = tid; c < g; c += NT) {
        double *y = Yk + (int64_t)c * ldb + c0;
        for (int r = 0; r < w; ++r) Xs[r * g + c] = ldcg(y + r);
        for (int r = w - 1; r >= 0; --r) {
          double t = Xs[r * g + c];
          for (int q = r + 1; q < w; ++q) t = fma(-s.l11[r * DS_LD + q], Xs[q * g + c], t);
          Xs[r * g + c] = quot(t, s.l11[r * DS_LD + r], s_rinv[r]);
        }
        for (int r = 0; r < w; ++r) stcg(y + r, Xs[r * g + c]);
      }
      __syncthreads();
      if (c0 > 0) update_core<true>(Yk, ldb, Akk + (int64_t)c0 * lda, lda, Yk + c0, ldb, c0, g, w, false, s.work);
    }
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
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(lu_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, LU_SMEM_BYTES);
  });
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
  lu_solve_kernel<<<grid, NT, LU_SMEM_BYTES, (cudaStream_t)stream>>>(a);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}
