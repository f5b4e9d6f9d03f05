// Reverse-mode derivatives of the Cholesky factor and of the solve (not in the paper; the
// differentiable form of its factorization).
//
// chol_backward: with S = L^-T Phi(L^T Lbar) L^-1 and Phi = lower triangle with the diagonal
// halved, Abar = (S + S^T)/2 (I. Murray, "Differentiation of the Cholesky decomposition",
// 2016). On the GPU: P = L^T Lbar on the lower 64 x 64 tiles (the k range of a tile starts at
// its first row, since L^T is upper triangular) with the FP64 DFMA tile update of the
// factorization; Phi(P)^T; two sweeps of the FP64 triangular solve with n right-hand sides
// (L^T M^T = Phi^T, L^T S = M); the symmetric part.
//
// chol_solve_backward: for X = A^-1 B, A = L L^T: Bbar = A^-1 Xbar (the FP64 solve) and
// Lbar = -tril(Bbar U^T + X V^T) with U = L^T X, V = L^T Bbar, all in O(n^2 nrhs).
#include <algorithm>
#include <mutex>
#include "common.cuh"
#include "tiles_f64.cuh"

namespace chol {

constexpr int AT = 64;  // output tile of the products

// dst(c, r) = src(r, c) for r < rows, c < cols; with mask_lower the entries with r < c (the
// strict upper triangle of src) are written as zero.
__global__ void transpose_kernel(const double *src, int64_t lds, double *dst, int64_t ldd, int rows, int cols,
                                 int mask_lower) {
  __shared__ double t[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + threadIdx.x, c = c0 + k;
    t[k][threadIdx.x] = (r < rows && c < cols && (!mask_lower || r >= c)) ? src[(int64_t)c * lds + r] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + threadIdx.x, r = r0 + k;
    if (r < rows && c < cols) dst[(int64_t)r * ldd + c] = t[threadIdx.x][k];
  }
}

// C tile (i0, j0) -= A(i0.., k0..) B(j0.., k0..)^T with the FP64 tile update; tiles wholly
// above the diagonal are skipped when `lower`, and with `ktri` the k range starts at i0.
__global__ void __launch_bounds__(NT) nt_tiles_kernel(double *C, int64_t ldc, const double *A, int64_t lda,
                                                      const double *B, int64_t ldb, int M, int N, int K,
                                                      int lower, int ktri) {
  extern __shared__ __align__(16) double smem[];
  const int i0 = blockIdx.x * AT, j0 = blockIdx.y * AT;
  if (lower && j0 > i0) return;
  const int k0 = ktri ? i0 : 0;
  if (k0 >= K) return;
  update_nt(C + (int64_t)j0 * ldc + i0, ldc, A + (int64_t)k0 * lda + i0, lda, B + (int64_t)k0 * ldb + j0, ldb,
            min(AT, M - i0), min(AT, N - j0), K - k0, lower && i0 == j0, smem);
}

// W(j, i) = Phi(P)_ij for i >= j, where C = -P on the lower tiles (W zero elsewhere).
__global__ void phi_t_kernel(const double *C, int64_t ldc, double *W, int64_t ldw, int n) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
    double v = 0.0;
    if (i > j) v = -C[(int64_t)j * ldc + i];
    else if (i == j) v = -0.5 * C[(int64_t)j * ldc + i];
    W[(int64_t)i * ldw + j] = v;
  }
}

// Out(i, j) = (S_ij + S_ji) / 2
__global__ void sym_kernel(const double *S, int64_t lds, double *Out, int64_t ldo, int n) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
    Out[(int64_t)j * ldo + i] = 0.5 * (S[(int64_t)j * lds + i] + S[(int64_t)i * lds + j]);
  }
}

// Out = scale * lower triangle of C (strict upper triangle of Out set to zero)
__global__ void lower_scaled_kernel(const double *C, int64_t ldc, double *Out, int64_t ldo, int n, double scale) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
    Out[(int64_t)j * ldo + i] = i >= j ? scale * C[(int64_t)j * ldc + i] : 0.0;
  }
}


static cudaError_t launch_transpose(const double *src, int64_t lds, double *dst, int64_t ldd, int rows, int cols,
                                    int mask, cudaStream_t s) {
  const dim3 grid((rows + 31) / 32, (cols + 31) / 32), block(32, 8);
  transpose_kernel<<<grid, block, 0, s>>>(src, lds, dst, ldd, rows, cols, mask);
  return cudaGetLastError();
}

static cudaError_t launch_nt(double *C, int64_t ldc, const double *A, int64_t lda, const double *B, int64_t ldb,
                             int M, int N, int K, int lower, int ktri, cudaStream_t s) {
  const cudaError_t e = set_smem_attr((const void *)nt_tiles_kernel, TILE_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const dim3 grid((M + AT - 1) / AT, (N + AT - 1) / AT);
  nt_tiles_kernel<<<grid, NT, TILE_SMEM_BYTES, s>>>(C, ldc, A, lda, B, ldb, M, N, K, lower, ktri);
  return cudaGetLastError();
}

static int eblocks() {
  const DeviceInfo di = current_device_info();
  return std::max(1, di.sms) * 8;
}

static size_t backward_ws(int n) {
  const size_t sq = align_up((size_t)n * n * 8, 256);
  return 3 * sq + align_up(chol_solve_workspace_size(n, n), 256);
}

static size_t solve_backward_ws(int n, int nrhs) {
  const size_t sq = align_up((size_t)n * n * 8, 256);
  const size_t pn = align_up((size_t)n * 2 * nrhs * 8, 256);
  return 2 * sq + 4 * pn;
}

}  // namespace chol

using namespace chol;

extern "C" size_t chol_backward_workspace_size(int n) {
  if (n < 0) return 0;
  return backward_ws(n);
}

extern "C" chol_status chol_backward(int n, const double *dL, int lda, double *dLbar, int ldlb, void *dWork,
                                     size_t work_bytes, void *stream) {
  if (n < 0 || lda < std::max(1, n) || ldlb < std::max(1, n)) return CHOL_ERR_INVALID_ARG;
  if (n == 0) return CHOL_OK;
  if (!dL || !dLbar) return CHOL_ERR_INVALID_ARG;
  if (!dWork || work_bytes < backward_ws(n) || ((uintptr_t)dWork & 255)) return CHOL_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t sq = align_up((size_t)n * n * 8, 256);
  unsigned char *ws = static_cast<unsigned char *>(dWork);
  double *W1 = reinterpret_cast<double *>(ws);
  double *W2 = reinterpret_cast<double *>(ws + sq);
  double *W3 = reinterpret_cast<double *>(ws + 2 * sq);
  void *swork = ws + 3 * sq;
  const size_t sbytes = chol_solve_workspace_size(n, n);
  // W3 = L^T, W2 = Lbar^T (lower triangles only)
  CHOL_CUDA_TRY(launch_transpose(dL, lda, W3, n, n, n, 1, s));
  CHOL_CUDA_TRY(launch_transpose(dLbar, ldlb, W2, n, n, n, 1, s));
  // W1 = -P on the lower tiles, P = L^T Lbar
  CHOL_CUDA_TRY(cudaMemsetAsync(W1, 0, (size_t)n * n * 8, s));
  CHOL_CUDA_TRY(launch_nt(W1, n, W3, n, W2, n, n, n, n, 1, 1, s));
  // W2 = Phi(P)^T
  phi_t_kernel<<<eblocks(), 256, 0, s>>>(W1, n, W2, n, n);
  CHOL_CUDA_TRY(cudaGetLastError());
  // L^T M^T = Phi^T  ->  W2 = M^T ;  W1 = M ;  L^T S = M  ->  W1 = S
  chol_status st = chol_trsm_sweep(1, n, n, dL, lda, W2, n, swork, sbytes, nullptr, stream);
  if (st != CHOL_OK) return st;
  CHOL_CUDA_TRY(launch_transpose(W2, n, W1, n, n, n, 0, s));
  st = chol_trsm_sweep(1, n, n, dL, lda, W1, n, swork, sbytes, nullptr, stream);
  if (st != CHOL_OK) return st;
  sym_kernel<<<eblocks(), 256, 0, s>>>(W1, n, dLbar, ldlb, n);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

extern "C" size_t chol_solve_backward_workspace_size(int n, int nrhs) {
  if (n < 0 || nrhs < 0) return 0;
  return solve_backward_ws(n, nrhs) + align_up(chol_solve_workspace_size(n, nrhs), 256);
}

extern "C" chol_status chol_solve_backward(int n, int nrhs, const double *dL, int lda, const double *dX, int ldx,
                                           const double *dXbar, int ldxb, double *dBbar, int ldbb,
                                           double *dLbar, int ldlb, void *dWork, size_t work_bytes,
                                           void *stream) {
  if (n < 0 || nrhs < 0 || lda < std::max(1, n) || ldx < std::max(1, n) || ldxb < std::max(1, n) ||
      ldbb < std::max(1, n) || ldlb < std::max(1, n))
    return CHOL_ERR_INVALID_ARG;
  if (n == 0) return CHOL_OK;
  if (!dL || !dLbar || (nrhs > 0 && (!dX || !dXbar || !dBbar))) return CHOL_ERR_INVALID_ARG;
  if (!dWork || work_bytes < chol_solve_backward_workspace_size(n, nrhs) || ((uintptr_t)dWork & 255))
    return CHOL_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (nrhs == 0) {
    CHOL_CUDA_TRY(cudaMemset2DAsync(dLbar, (size_t)ldlb * 8, 0, (size_t)n * 8, n, s));
    return CHOL_OK;
  }
  const size_t sq = align_up((size_t)n * n * 8, 256);
  const size_t pn = align_up((size_t)n * 2 * nrhs * 8, 256);
  unsigned char *ws = static_cast<unsigned char *>(dWork);
  double *LT = reinterpret_cast<double *>(ws);
  double *C = reinterpret_cast<double *>(ws + sq);
  double *P = reinterpret_cast<double *>(ws + 2 * sq);            // [Bbar | X], n x 2nrhs
  double *PT = reinterpret_cast<double *>(ws + 2 * sq + pn);      // P^T, 2nrhs x n
  double *Q = reinterpret_cast<double *>(ws + 2 * sq + 2 * pn);   // -L^T P = -[V | U]
  double *R = reinterpret_cast<double *>(ws + 2 * sq + 3 * pn);   // [X | Bbar]
  void *swork = ws + 2 * sq + 4 * pn;
  const size_t sbytes = chol_solve_workspace_size(n, nrhs);
  const size_t colb = (size_t)n * 8;
  // Bbar = A^-1 Xbar
  CHOL_CUDA_TRY(cudaMemcpy2DAsync(dBbar, (size_t)ldbb * 8, dXbar, (size_t)ldxb * 8, colb, nrhs,
                                  cudaMemcpyDeviceToDevice, s));
  chol_status st = chol_solve(n, nrhs, dL, lda, dBbar, ldbb, swork, sbytes, nullptr, stream);
  if (st != CHOL_OK) return st;
  // P = [Bbar | X], R = [X | Bbar], PT = P^T, LT = L^T (lower of L)
  CHOL_CUDA_TRY(cudaMemcpy2DAsync(P, colb, dBbar, (size_t)ldbb * 8, colb, nrhs, cudaMemcpyDeviceToDevice, s));
  CHOL_CUDA_TRY(cudaMemcpy2DAsync(P + (size_t)n * nrhs, colb, dX, (size_t)ldx * 8, colb, nrhs,
                                  cudaMemcpyDeviceToDevice, s));
  CHOL_CUDA_TRY(cudaMemcpy2DAsync(R, colb, dX, (size_t)ldx * 8, colb, nrhs, cudaMemcpyDeviceToDevice, s));
  CHOL_CUDA_TRY(cudaMemcpy2DAsync(R + (size_t)n * nrhs, colb, dBbar, (size_t)ldbb * 8, colb, nrhs,
                                  cudaMemcpyDeviceToDevice, s));
  CHOL_CUDA_TRY(launch_transpose(P, n, PT, 2 * nrhs, n, 2 * nrhs, 0, s));
  CHOL_CUDA_TRY(launch_transpose(dL, lda, LT, n, n, n, 1, s));
  // Q = -L^T P = -[V | U]  (L^T is upper triangular: k starts at the tile's first row)
  CHOL_CUDA_TRY(cudaMemsetAsync(Q, 0, (size_t)n * 2 * nrhs * 8, s));
  CHOL_CUDA_TRY(launch_nt(Q, n, LT, n, PT, 2 * nrhs, n, 2 * nrhs, n, 0, 1, s));
  // C = -R Q^T = X V^T + Bbar U^T on the lower tiles ; Lbar = -tril(C)
  CHOL_CUDA_TRY(cudaMemsetAsync(C, 0, (size_t)n * n * 8, s));
  CHOL_CUDA_TRY(launch_nt(C, n, R, n, Q, n, n, n, 2 * nrhs, 1, 0, s));
  lower_scaled_kernel<<<eblocks(), 256, 0, s>>>(C, n, dLbar, ldlb, n, -1.0);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

extern "C" chol_status chol_lower_copy(int n, const double *dSrc, int lds, double *dDst, int ldd, void *stream) {
  if (n < 0 || lds < std::max(1, n) || ldd < std::max(1, n)) return CHOL_ERR_INVALID_ARG;
  if (n == 0) return CHOL_OK;
  if (!dSrc || !dDst) return CHOL_ERR_INVALID_ARG;
  lower_scaled_kernel<<<eblocks(), 256, 0, (cudaStream_t)stream>>>(dSrc, lds, dDst, ldd, n, 1.0);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}
