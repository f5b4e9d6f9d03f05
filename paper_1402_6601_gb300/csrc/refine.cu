// Mixed-precision solve: low-precision tile Cholesky of A (FP32 FFMA, or FP32 with tensor-core
// BF16 updates of the diagonally scaled matrix), then iterative refinement whose residual
// r = b - A x and update x += d run in FP64 (classical iterative refinement: each step
// solves A d = r with the low-precision factor). Not in the paper; it reuses the paper's
// factorization (same task graph, scheduler and policies) at a lower precision.
//
// The loop runs a fixed number of steps on the device without host round trips: every
// step's kernels first read a "converged" flag and return at once when it is set, so the
// whole solve is one asynchronous sequence of launches on the caller's stream.
//
// Kernels (FP64 parts are bound by the FP64 pipe, like the factor):
//   convert_lower   A (FP64, lower) -> A32 (FP32), rows padded with zeros
//   norm kernels    ||A||_inf from the lower triangle (symmetric), once
//   symm_residual   R = B - A X, A symmetric from its lower triangle, one block per 32 rows
//   to_f32 / axpy   R32 = float(R); X += double(D32)
//   berr            eta = max_c ||r_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf)
#include <algorithm>
#include "common.cuh"
#include "blockacc.cuh"
#include "internal.cuh"

namespace chol {

struct RefineCtrl {
  int done;     // set once eta <= tol: later steps do nothing
  int iters;    // refinement steps taken (the first low-precision solve counts as one)
  double berr;  // eta after the last step taken
  double normA; // ||A||_inf
  int pad[58];
};

constexpr int RB = 32;    // rows per block of the residual
constexpr int RG = 64;    // right-hand sides per group
constexpr int RLD = RB + 1;

__device__ __forceinline__ void atomic_max_nonneg(double *p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(v));
}

// With `scale` (nullable): A32 = D^-1/2 A D^-1/2, scale_i = 1 / sqrt(a_ii) (1 where a_ii <= 0,
// which the factor then reports), computed in FP64 before rounding.
__global__ void convert_lower_kernel(const double *A, int64_t lda, float *A32, int64_t lda32, int n,
                                     const double *scale) {
  const int64_t total = lda32 * (int64_t)n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / lda32, i = e - j * lda32;
    double v = (i >= j && i < n) ? A[j * lda + i] : 0.0;
    if (scale && i < n) v *= scale[i] * scale[j];
    A32[e] = (float)v;
  }
}

__global__ void diag_scale_kernel(const double *A, int64_t lda, int n, double *scale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double d = A[(int64_t)i * lda + i];
    scale[i] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
  }
}

// Load block (I, J) of the symmetric A from its lower triangle into As[row in I][col in J]:
// (I, J) itself for J < I, (J, I)^T for J > I, the symmetric diagonal block for J = I.
__device__ __forceinline__ void load_sym_block(const double *A, int64_t lda, int I, int J, int n, double *As) {
  const int I0 = I * RB, J0 = J * RB, rows = min(RB, n - I0), jc = min(RB, n - J0);
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
    const int a = e & 31, b = e >> 5;
    double v = 0.0;
    if (J < I) {          // As[a][b] = A(I0+a, J0+b)
      if (a < rows && b < jc) v = A[(int64_t)(J0 + b) * lda + I0 + a];
      As[a * RLD + b] = v;
    } else if (J > I) {   // As[b][a] = A(J0+a, I0+b), read along a (contiguous)
      if (a < jc && b < rows) v = A[(int64_t)(I0 + b) * lda + J0 + a];
      As[b * RLD + a] = v;
    } else {
      if (a < rows && b < rows) v = a >= b ? A[(int64_t)(I0 + b) * lda + I0 + a] : A[(int64_t)(I0 + a) * lda + I0 + b];
      As[a * RLD + b] = v;
    }
  }
}

// ||A||_inf = max_i sum_j |a_ij| of the symmetric A; one block per 32 rows
__global__ void __launch_bounds__(256) rownorm_kernel(const double *A, int64_t lda, int n, RefineCtrl *ctrl) {
  __shared__ double As[RB * RLD];
  __shared__ double part[8][RB];
  const int nrb = (n + RB - 1) / RB;
  const int I = blockIdx.x;
  const int tid = threadIdx.x, rr = tid & 31, cs = tid >> 5;
  double s = 0.0;
  for (int J = 0; J < nrb; ++J) {
    load_sym_block(A, lda, I, J, n, As);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 4; ++t) s += fabs(As[rr * RLD + cs + 8 * t]);
    __syncthreads();
  }
  part[cs][rr] = s;
  __syncthreads();
  if (tid < RB && I * RB + tid < n) {
    double t = 0.0;
    for (int c = 0; c < 8; ++c) t += part[c][tid];
    atomic_max_nonneg(&ctrl->normA, t);
  }
}

// R = B - A X (FP64). Block (I, g): rows I*32.., columns g*64..; the 32 x 32 blocks of the
// symmetric A come from its lower triangle (load_sym_block); the threads share the
// products as described in blockacc.cuh.
template <int CPT>
__global__ void __launch_bounds__(256) symm_residual_kernel(const double *A, int64_t lda, const double *X,
                                                            int64_t ldx, const double *B, int64_t ldb, double *R,
                                                            int64_t ldr, int n, int nrhs, const int *skip) {
  __shared__ double As[RB * RLD];
  __shared__ double Xs[RB * RG];
  __shared__ double Red[RB * RG];
  if (skip && ld_volatile(skip)) return;
  const int nrb = (n + RB - 1) / RB;
  const int I = blockIdx.x, g = blockIdx.y;
  const int I0 = I * RB, rows = min(RB, n - I0);
  const int c0 = g * RG, cols = min(RG, nrhs - c0);
  const int tid = threadIdx.x, rr = tid & 31, warp = tid >> 5;
  const Slices<CPT> sl(cols, warp);
  double acc[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) {
    const int c = sl.col(q);
    acc[q] = (sl.kslice == 0 && rr < rows && c < cols) ? B[(int64_t)(c0 + c) * ldb + I0 + rr] : 0.0;
  }
  for (int J = 0; J < nrb; ++J) {
    const int J0 = J * RB, jc = min(RB, n - J0);
    load_sym_block(A, lda, I, J, n, As);
    for (int e = tid; e < RB * RG; e += 256) {
      const int k = e & 31, c = e >> 5;
      Xs[k * RG + c] = (k < jc && c < cols) ? X[(int64_t)(c0 + c) * ldx + J0 + k] : 0.0;
    }
    __syncthreads();
    acc_step<double, CPT>(acc, As, RLD, Xs, RG, rr, sl);
    __syncthreads();
  }
  acc_finish<double, CPT>(acc, Xs, RG, Red, rr, cols, sl);
  for (int e = tid; e < RB * cols; e += 256) {
    const int i = e & 31, c = e >> 5;
    if (i < rows) R[(int64_t)(c0 + c) * ldr + I0 + i] = Xs[i * RG + c];
  }
}

// R32 = float(D^-1/2 R) (scale nullable: no scaling)
__global__ void to_f32_kernel(const double *R, int64_t ldr, float *R32, int64_t ld32, int n, int nrhs,
                              const double *scale, const int *skip) {
  if (skip && ld_volatile(skip)) return;
  const int64_t total = (int64_t)n * nrhs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    const double r = R[c * ldr + i];
    R32[c * ld32 + i] = (float)(scale ? r * scale[i] : r);
  }
}

// X += D^-1/2 double(D32) (scale nullable)
__global__ void axpy_kernel(double *X, int64_t ldx, const float *D, int64_t ldd, int n, int nrhs,
                            const double *scale, const int *skip) {
  if (skip && ld_volatile(skip)) return;
  const int64_t total = (int64_t)n * nrhs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    const double d = (double)D[c * ldd + i];
    X[c * ldx + i] += scale ? d * scale[i] : d;
  }
}

// eta_c per right-hand side (one block per column)
__global__ void berr_cols_kernel(const double *R, int64_t ldr, const double *X, int64_t ldx, const double *B,
                                 int64_t ldb, int n, const RefineCtrl *ctrl, double *eta, const int *skip) {
  if (skip && ld_volatile(skip)) return;
  const int c = blockIdx.x;
  double mr = 0.0, mx = 0.0, mb = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    mr = fmax(mr, fabs(R[(int64_t)c * ldr + i]));
    mx = fmax(mx, fabs(X[(int64_t)c * ldx + i]));
    mb = fmax(mb, fabs(B[(int64_t)c * ldb + i]));
  }
  __shared__ double red[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = mr;
    red[1][threadIdx.x >> 5] = mx;
    red[2][threadIdx.x >> 5] = mb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mr = fmax(mr, red[0][w]);
      mx = fmax(mx, red[1][w]);
      mb = fmax(mb, red[2][w]);
    }
    const double den = ctrl->normA * mx + mb;
    eta[c] = den > 0.0 ? mr / den : (mr > 0.0 ? INFINITY : 0.0);
  }
}

__global__ void refine_step_done_kernel(RefineCtrl *ctrl, const double *eta, int nrhs, double tol,
                                        const int *factor_info) {
  if (threadIdx.x != 0) return;
  if (ctrl->done) return;
  if (*factor_info != 0) {  // no usable factor: stop without touching X
    ctrl->done = 1;
    ctrl->berr = INFINITY;
    return;
  }
  double e = 0.0;
  for (int c = 0; c < nrhs; ++c) e = fmax(e, eta[c]);
  ctrl->iters += 1;
  ctrl->berr = e;
  if (e <= tol) ctrl->done = 1;
}

__global__ void refine_init_kernel(RefineCtrl *ctrl, const int *factor_info) {
  if (threadIdx.x == 0) {
    ctrl->done = *factor_info != 0 ? 1 : 0;
    ctrl->iters = 0;
    ctrl->berr = INFINITY;
    ctrl->normA = 0.0;
  }
}

__global__ void refine_out_kernel(const RefineCtrl *ctrl, int *dIters, double *dBerr) {
  if (threadIdx.x == 0) {
    if (dIters) *dIters = ctrl->iters;
    if (dBerr) *dBerr = ctrl->berr;
  }
}

struct RefineLayout {
  size_t ctrl, a32, fwork, r, r32, swork, eta, finfo, scale, total, fbytes, sbytes;
  int64_t lda32, ld32;
};

static RefineLayout refine_layout(int n, int nrhs, const chol_opts *opts) {
  RefineLayout L;
  L.lda32 = std::max<int64_t>(32, ((int64_t)n + 31) / 32 * 32);
  L.ld32 = L.lda32;
  size_t o = 0;
  L.ctrl = o; o += 256;
  L.finfo = o; o += 256;
  L.a32 = o; o += align_up((size_t)L.lda32 * n * 4, 256);
  L.fbytes = chol_factor_workspace_size(n, opts);
  L.fwork = o; o += align_up(L.fbytes, 256);
  L.r = o; o += align_up((size_t)n * std::max(nrhs, 1) * 8, 256);
  L.scale = o; o += align_up((size_t)std::max(n, 1) * 8, 256);
  L.r32 = o; o += align_up((size_t)L.ld32 * std::max(nrhs, 1) * 4, 256);
  L.sbytes = solve_workspace_bytes(n, nrhs);
  L.swork = o; o += align_up(L.sbytes, 256);
  L.eta = o; o += align_up((size_t)std::max(nrhs, 1) * 8, 256);
  L.total = o;
  return L;
}

}  // namespace chol

using namespace chol;

extern "C" size_t chol_solve_refine_workspace_size(int n, int nrhs, const chol_opts *opts) {
  if (n < 0 || nrhs < 0) return 0;
  if (n > 0 && chol_factor_workspace_size(n, opts) == 0) return 0;
  return refine_layout(n, nrhs, opts).total;
}

extern "C" chol_status chol_solve_refine(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb,
                                         double *dX, int ldx, int low_precision, double tol, int max_iter,
                                         const chol_opts *opts, void *dWork, size_t work_bytes, int *dInfo,
                                         int *dIters, double *dBerr, void *stream) {
  if (n < 0 || nrhs < 0 || !dInfo || !(tol >= 0.0) || max_iter < 1 || max_iter > 1000) return CHOL_ERR_INVALID_ARG;
  const int prec = low_precision == CHOL_F32 ? PREC_F32
                   : low_precision == CHOL_BF16 ? PREC_BF16
                   : low_precision == CHOL_BF16X3 ? PREC_BF16X3
                                                  : -1;
  if (prec < 0) return CHOL_ERR_UNSUPPORTED;
  if (lda < std::max(1, n) || ldb < std::max(1, n) || ldx < std::max(1, n)) return CHOL_ERR_INVALID_ARG;
  if (n > 0 && (!dA || (nrhs > 0 && (!dB || !dX)))) return CHOL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0 || nrhs == 0) {
    CHOL_CUDA_TRY(cudaMemsetAsync(dInfo, 0, sizeof(int), s));
    if (dIters) CHOL_CUDA_TRY(cudaMemsetAsync(dIters, 0, sizeof(int), s));
    if (dBerr) CHOL_CUDA_TRY(cudaMemsetAsync(dBerr, 0, sizeof(double), s));
    return CHOL_OK;
  }
  const RefineLayout L = refine_layout(n, nrhs, opts);
  if (L.fbytes == 0) return CHOL_ERR_INVALID_ARG;
  if (!dWork || work_bytes < L.total || ((uintptr_t)dWork & 255)) return CHOL_ERR_WORKSPACE;
  const DeviceInfo di = current_device_info();
  if (di.sms <= 0) return CHOL_ERR_CUDA;
  unsigned char *ws = static_cast<unsigned char *>(dWork);
  RefineCtrl *ctrl = reinterpret_cast<RefineCtrl *>(ws + L.ctrl);
  int *finfo = reinterpret_cast<int *>(ws + L.finfo);
  float *A32 = reinterpret_cast<float *>(ws + L.a32);
  double *R = reinterpret_cast<double *>(ws + L.r);
  float *R32 = reinterpret_cast<float *>(ws + L.r32);
  double *eta = reinterpret_cast<double *>(ws + L.eta);
  const int *skip = &ctrl->done;
  const int eblocks = di.sms * 8;

  // low-precision factor (of the diagonally scaled matrix for the BF16 forms)
  double *scale = prec == PREC_F32 ? nullptr : reinterpret_cast<double *>(ws + L.scale);
  if (scale) diag_scale_kernel<<<(n + 255) / 256, 256, 0, s>>>(dA, lda, n, scale);
  convert_lower_kernel<<<eblocks, 256, 0, s>>>(dA, lda, A32, L.lda32, n, scale);
  CHOL_CUDA_TRY(cudaGetLastError());
  chol_status st = factor_impl(prec, n, A32, (int)L.lda32, opts, ws + L.fwork, L.fbytes, finfo, stream);
  if (st != CHOL_OK) return st;
  CHOL_CUDA_TRY(cudaMemcpyAsync(dInfo, finfo, sizeof(int), cudaMemcpyDeviceToDevice, s));
  refine_init_kernel<<<1, 32, 0, s>>>(ctrl, finfo);
  // ||A||_inf
  rownorm_kernel<<<(n + RB - 1) / RB, 256, 0, s>>>(dA, lda, n, ctrl);
  CHOL_CUDA_TRY(cudaGetLastError());
  // x0 = 0, r0 = b
  CHOL_CUDA_TRY(cudaMemset2DAsync(dX, (size_t)ldx * 8, 0, (size_t)n * 8, nrhs, s));
  CHOL_CUDA_TRY(cudaMemcpy2DAsync(R, (size_t)n * 8, dB, (size_t)ldb * 8, (size_t)n * 8, nrhs,
                                  cudaMemcpyDeviceToDevice, s));
  const dim3 rgrid((n + RB - 1) / RB, (nrhs + RG - 1) / RG);
  for (int it = 0; it < max_iter; ++it) {
    to_f32_kernel<<<eblocks, 256, 0, s>>>(R, n, R32, L.ld32, n, nrhs, scale, skip);
    CHOL_CUDA_TRY(cudaGetLastError());
    st = solve_f32(n, nrhs, A32, (int)L.lda32, R32, (int)L.ld32, ws + L.swork, skip, s);
    if (st != CHOL_OK) return st;
    axpy_kernel<<<eblocks, 256, 0, s>>>(dX, ldx, R32, L.ld32, n, nrhs, scale, skip);
    const int cpt = cpt_for(std::min(nrhs, RG));
    if (cpt == 8) symm_residual_kernel<8><<<rgrid, 256, 0, s>>>(dA, lda, dX, ldx, dB, ldb, R, n, n, nrhs, skip);
    else if (cpt == 4) symm_residual_kernel<4><<<rgrid, 256, 0, s>>>(dA, lda, dX, ldx, dB, ldb, R, n, n, nrhs, skip);
    else if (cpt == 2) symm_residual_kernel<2><<<rgrid, 256, 0, s>>>(dA, lda, dX, ldx, dB, ldb, R, n, n, nrhs, skip);
    else symm_residual_kernel<1><<<rgrid, 256, 0, s>>>(dA, lda, dX, ldx, dB, ldb, R, n, n, nrhs, skip);
    berr_cols_kernel<<<nrhs, 256, 0, s>>>(R, n, dX, ldx, dB, ldb, n, ctrl, eta, skip);
    refine_step_done_kernel<<<1, 32, 0, s>>>(ctrl, eta, nrhs, tol, finfo);
    CHOL_CUDA_TRY(cudaGetLastError());
  }
  refine_out_kernel<<<1, 32, 0, s>>>(ctrl, dIters, dBerr);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}
