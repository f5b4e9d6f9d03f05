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
//   convert_lower   A (FP64, lower) -> A32 (FP32), with the absolute row sums of the
//                   symmetric A; norm_max turns them into ||A||_inf
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

// One 32 x 32 tile (I, J), I >= J, of the lower triangle per block (32 x 8 threads): A32 =
// float(A) (with `scale`, nullable: S A S with the powers of two of diag_scale_kernel,
// applied exactly before rounding: v s_i s_j by adding the scales' exponents to v's, with
// no FP64 multiplication (FP64 arithmetic is slow on this part); the FP64 product, exact as
// well, covers zeros, subnormals, infinities and results outside the normal range), and the
// absolute row sums of the symmetric A accumulated into rsum: |a_ij| counts for row i and,
// below the diagonal, for row j. The sums
// are FP32 (the norm only scales the backward error, and FP64 adds would run on the FP64
// pipe); entries above the diagonal of A32 are not written (nothing reads them).
__global__ void __launch_bounds__(256) convert_lower_kernel(const double *A, int64_t lda, float *A32, int64_t lda32,
                                                            int n, const double *scale, float *rsum) {
  const int I = blockIdx.x, J = blockIdx.y;
  if (J > I) return;
  __shared__ float rs[8][33], cs[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = I * 32 + tx;
  float rsum_i = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int jl = ty + 8 * u, j = J * 32 + jl;
    double v = 0.0;
    if (i < n && j < n && i >= j) {
      v = A[(int64_t)j * lda + i];
      double vs = v;
      if (scale) {
        const double si = scale[i], sj = scale[j];
        const int k = ((__double2hiint(si) >> 20) & 0x7ff) + ((__double2hiint(sj) >> 20) & 0x7ff) - 2046;
        const int hi = __double2hiint(v);
        const int E = (hi >> 20) & 0x7ff;
        vs = (E > 0 && E < 2047 && E + k > 0 && E + k < 2047) ? __hiloint2double(hi + k * (1 << 20), __double2loint(v))
                                                               : v * si * sj;
      }
      A32[(int64_t)j * lda32 + i] = (float)vs;
    }
    const float av = fabsf((float)v);
    rsum_i += av;
    // column j's entries below the diagonal count for row j (warp sum over the 32 rows)
    float c = i > j ? av : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (tx == 0) cs[jl] = c;
  }
  rs[ty][tx] = rsum_i;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += rs[k][threadIdx.x];
    if (I * 32 + threadIdx.x < n) atomicAdd(&rsum[I * 32 + threadIdx.x], t);
    if (J * 32 + threadIdx.x < n) atomicAdd(&rsum[J * 32 + threadIdx.x], cs[threadIdx.x]);
  }
}

// ||A||_inf = max_i rsum_i (one block)
__global__ void norm_max_kernel(const float *rsum, int n, RefineCtrl *ctrl) {
  __shared__ float w[32];
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, rsum[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? w[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      ctrl->normA = (double)m;
      // entries near FLT_MAX overflow the FP32 row sums: with an infinite (or NaN) norm every
      // eta would read 0 and the first step would pass for convergence, so no step is taken
      // and the backward error is reported as NaN (X stays zero)
      if (!isfinite(m)) {
        ctrl->done = 1;
        ctrl->berr = __longlong_as_double(0x7ff8000000000000ll);
      }
    }
  }
}

// Diagonal scaling of the low-precision forms: s_i = 2^-q for a_ii = m 2^e (m in [1, 2)),
// q = ceil(e / 2), so s_i^2 a_ii lies in [1/2, 2); 1 where a_ii <= 0 or is not finite. Powers
// of two, as LAPACK's xPOEQUB chooses its factors, scale every entry without a rounding
// error, and the scaled diagonal is within a factor two of Jacobi's unit one.
__global__ void diag_scale_kernel(const double *A, int64_t lda, int n, double *scale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double d = A[(int64_t)i * lda + i];
    double s = 1.0;
    if (d > 0.0 && isfinite(d)) s = ldexp(1.0, -((ilogb(d) + 1) >> 1));
    scale[i] = s;
  }
}

// Block (I, J) of the symmetric A from its lower triangle, as As[row in I][col in J]: (I, J)
// itself for J < I, (J, I)^T for J > I (read along its columns, contiguous), the symmetric
// diagonal block for J = I. sym_value gives element e (a = e mod 32, b = e / 32) of that read
// and sym_slot the As slot it goes to.
__device__ __forceinline__ double sym_value(const double *A, int64_t lda, int I, int J, int n, int e) {
  const int I0 = I * RB, J0 = J * RB, rows = min(RB, n - I0), jc = min(RB, n - J0);
  const int a = e & 31, b = e >> 5;
  if (J < I) return (a < rows && b < jc) ? __ldcg(A + (int64_t)(J0 + b) * lda + I0 + a) : 0.0;
  if (J > I) return (a < jc && b < rows) ? __ldcg(A + (int64_t)(I0 + b) * lda + J0 + a) : 0.0;
  if (a >= rows || b >= rows) return 0.0;
  return a >= b ? __ldcg(A + (int64_t)(I0 + b) * lda + I0 + a) : __ldcg(A + (int64_t)(I0 + a) * lda + I0 + b);
}
__device__ __forceinline__ int sym_slot(int I, int J, int e) {
  const int a = e & 31, b = e >> 5;
  return J > I ? b * RLD + a : a * RLD + b;
}

// R = B - A X (FP64). Block (I, g): rows I*32.., columns g*64..; the threads share the products
// as described in blockacc.cuh. The blocks of A and X for step J + 1 are loaded into registers
// while step J is multiplied, so the FP64 pipe does not wait for L2 between steps.
//
// The J range of a block row is cut into gridDim.z segments so that the grid has many more
// blocks than the SMs hold at once (a block row per block left a ~20 % imbalance between SMs
// holding three and four of them): segment s covers its share of J, starts from B when s = 0
// and from 0 otherwise, and writes its partial sums to R + s * pstride; sum_partials_kernel
// adds the segments in a fixed order (deterministic). With one segment R is written directly.
template <int CPT>
__global__ void __launch_bounds__(256, 4) symm_residual_kernel(const double *A, int64_t lda, const double *X,
                                                            int64_t ldx, const double *B, int64_t ldb, double *R,
                                                            int64_t ldr, int64_t pstride, int n, int nrhs,
                                                            const int *skip) {
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
  const int seg = blockIdx.z, nseg = gridDim.z;
  const int Jlo = (int)((int64_t)nrb * seg / nseg), Jhi = (int)((int64_t)nrb * (seg + 1) / nseg);
  R += (int64_t)seg * pstride;
  double acc[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) {
    const int c = sl.col(q);
    acc[q] = (seg == 0 && sl.kslice == 0 && rr < rows && c < cols) ? B[(int64_t)(c0 + c) * ldb + I0 + rr] : 0.0;
  }
  constexpr int NA = RB * RB / 256, NX = RB * RG / 256;
  double ra[NA], rx[NX];
  auto load = [&](int J) {
    const int J0 = J * RB, jc = min(RB, n - J0);
#pragma unroll
    for (int u = 0; u < NA; ++u) ra[u] = sym_value(A, lda, I, J, n, tid + 256 * u);
#pragma unroll
    for (int u = 0; u < NX; ++u) {
      const int e = tid + 256 * u, k = e & 31, c = e >> 5;
      rx[u] = (k < jc && c < cols) ? __ldcg(X + (int64_t)(c0 + c) * ldx + J0 + k) : 0.0;
    }
  };
  if (Jlo < Jhi) load(Jlo);
  for (int J = Jlo; J < Jhi; ++J) {
#pragma unroll
    for (int u = 0; u < NA; ++u) As[sym_slot(I, J, tid + 256 * u)] = ra[u];
#pragma unroll
    for (int u = 0; u < NX; ++u) {
      const int e = tid + 256 * u;
      Xs[(e & 31) * RG + (e >> 5)] = rx[u];
    }
    __syncthreads();
    if (J + 1 < Jhi) load(J + 1);
    acc_step<double, CPT>(acc, As, RLD, Xs, RG, rr, sl);
    __syncthreads();
  }
  acc_finish<double, CPT>(acc, Xs, RG, Red, rr, cols, sl);
  for (int e = tid; e < RB * cols; e += 256) {
    const int i = e & 31, c = e >> 5;
    if (i < rows) R[(int64_t)(c0 + c) * ldr + I0 + i] = Xs[i * RG + c];
  }
}

// R = sum over the segments of the partial residuals P + s * pstride (column-major, ld n)
__global__ void sum_partials_kernel(const double *P, int64_t pstride, int nseg, int n, int nrhs, double *R,
                                    int64_t ldr, const int *skip) {
  if (skip && ld_volatile(skip)) return;
  const int64_t total = (int64_t)n * nrhs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e - c * n;
    double t = 0.0;
    for (int sg = 0; sg < nseg; ++sg) t += P[sg * pstride + c * n + i];
    R[c * ldr + i] = t;
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
  size_t ctrl, a32, fwork, r, r32, swork, eta, finfo, scale, rsum, part, total, fbytes, sbytes;
  int64_t lda32, ld32;
  int nseg;  // J segments of the residual
};

static RefineLayout refine_layout(int n, int nrhs, const chol_opts *opts, int low_precision) {
  RefineLayout L;
  L.lda32 = std::max<int64_t>(32, ((int64_t)n + 31) / 32 * 32);
  L.ld32 = L.lda32;
  size_t o = 0;
  L.ctrl = o; o += 256;
  L.finfo = o; o += 256;
  L.a32 = o; o += align_up((size_t)L.lda32 * n * 4, 256);
  L.fbytes = chol_factor_lowp_workspace_size(low_precision, n, opts);
  L.fwork = o; o += align_up(L.fbytes, 256);
  L.r = o; o += align_up((size_t)n * std::max(nrhs, 1) * 8, 256);
  L.scale = o; o += align_up((size_t)std::max(n, 1) * 8, 256);
  L.rsum = o; o += align_up((size_t)std::max(n, 1) * 8, 256);
  {
    // about nine waves of residual blocks at three blocks per SM
    const int64_t rows = ((int64_t)n + RB - 1) / RB * (((int64_t)std::max(nrhs, 1) + RG - 1) / RG);
    const DeviceInfo di = current_device_info();
    const int64_t want = (int64_t)std::max(di.sms, 1) * 3 * 9;
    L.nseg = (int)std::max<int64_t>(1, std::min<int64_t>({32, (want + rows - 1) / rows, ((int64_t)n + RB - 1) / RB}));
  }
  L.part = o;
  if (L.nseg > 1) o += align_up((size_t)L.nseg * n * std::max(nrhs, 1) * 8, 256);
  L.r32 = o; o += align_up((size_t)L.ld32 * std::max(nrhs, 1) * 4, 256);
  L.sbytes = solve_workspace_bytes(n, nrhs);
  L.swork = o; o += align_up(L.sbytes, 256);
  L.eta = o; o += align_up((size_t)std::max(nrhs, 1) * 8, 256);
  L.total = o;
  return L;
}

}  // namespace chol

using namespace chol;

extern "C" size_t chol_solve_refine_prec_workspace_size(int low_precision, int n, int nrhs, const chol_opts *opts) {
  if (n < 0 || nrhs < 0) return 0;
  if (n > 0 && chol_factor_lowp_workspace_size(low_precision, n, opts) == 0) return 0;
  return refine_layout(n, nrhs, opts, low_precision).total;
}

extern "C" size_t chol_solve_refine_workspace_size(int n, int nrhs, const chol_opts *opts) {
  // enough for every low-precision form
  size_t best = 0;
  for (int p : {CHOL_F32, CHOL_BF16, CHOL_BF16X3}) {
    const size_t b = chol_solve_refine_prec_workspace_size(p, n, nrhs, opts);
    if (b == 0) return 0;
    best = std::max(best, b);
  }
  return best;
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
  const RefineLayout L = refine_layout(n, nrhs, opts, low_precision);
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
  float *rsum = reinterpret_cast<float *>(ws + L.rsum);
  CHOL_CUDA_TRY(cudaMemsetAsync(rsum, 0, (size_t)n * 4, s));
  {
    const int nt = (n + 31) / 32;
    convert_lower_kernel<<<dim3(nt, nt), 256, 0, s>>>(dA, lda, A32, L.lda32, n, scale, rsum);
    CHOL_CUDA_TRY(cudaGetLastError());
  }
  chol_status st = factor_impl(prec, n, A32, (int)L.lda32, opts, ws + L.fwork, L.fbytes, finfo, stream);
  if (st != CHOL_OK) return st;
  CHOL_CUDA_TRY(cudaMemcpyAsync(dInfo, finfo, sizeof(int), cudaMemcpyDeviceToDevice, s));
  refine_init_kernel<<<1, 32, 0, s>>>(ctrl, finfo);
  // ||A||_inf from the row sums of the conversion pass
  norm_max_kernel<<<1, 1024, 0, s>>>(rsum, n, ctrl);
  CHOL_CUDA_TRY(cudaGetLastError());
  // x0 = 0, r0 = b
  CHOL_CUDA_TRY(cudaMemset2DAsync(dX, (size_t)ldx * 8, 0, (size_t)n * 8, nrhs, s));
  CHOL_CUDA_TRY(cudaMemcpy2DAsync(R, (size_t)n * 8, dB, (size_t)ldb * 8, (size_t)n * 8, nrhs,
                                  cudaMemcpyDeviceToDevice, s));
  const dim3 rgrid((n + RB - 1) / RB, (nrhs + RG - 1) / RG, L.nseg);
  double *part = reinterpret_cast<double *>(ws + L.part);
  // with segments the residual kernel writes partials (ld n), summed into R afterwards
  double *Rout = L.nseg > 1 ? part : R;
  const int64_t pstride = (int64_t)n * nrhs;
  for (int it = 0; it < max_iter; ++it) {
    to_f32_kernel<<<eblocks, 256, 0, s>>>(R, n, R32, L.ld32, n, nrhs, scale, skip);
    CHOL_CUDA_TRY(cudaGetLastError());
    st = solve_f32(n, nrhs, A32, (int)L.lda32, R32, (int)L.ld32, ws + L.swork, skip, s);
    if (st != CHOL_OK) return st;
    axpy_kernel<<<eblocks, 256, 0, s>>>(dX, ldx, R32, L.ld32, n, nrhs, scale, skip);
    const int cpt = cpt_for(std::min(nrhs, RG));
    if (cpt == 8)
      symm_residual_kernel<8><<<rgrid, 256, 0, s>>>(dA, lda, dX, ldx, dB, ldb, Rout, n, pstride, n, nrhs, skip);
    else if (cpt == 4)
      symm_residual_kernel<4><<<rgrid, 256, 0, s>>>(dA, lda, dX, ldx, dB, ldb, Rout, n, pstride, n, nrhs, skip);
    else if (cpt == 2)
      symm_residual_kernel<2><<<rgrid, 256, 0, s>>>(dA, lda, dX, ldx, dB, ldb, Rout, n, pstride, n, nrhs, skip);
    else
      symm_residual_kernel<1><<<rgrid, 256, 0, s>>>(dA, lda, dX, ldx, dB, ldb, Rout, n, pstride, n, nrhs, skip);
    if (L.nseg > 1) sum_partials_kernel<<<eblocks, 256, 0, s>>>(part, pstride, L.nseg, n, nrhs, R, n, skip);
    berr_cols_kernel<<<nrhs, 256, 0, s>>>(R, n, dX, ldx, dB, ldb, n, ctrl, eta, skip);
    refine_step_done_kernel<<<1, 32, 0, s>>>(ctrl, eta, nrhs, tol, finfo);
    CHOL_CUDA_TRY(cudaGetLastError());
  }
  refine_out_kernel<<<1, 32, 0, s>>>(ctrl, dIters, dBerr);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}
