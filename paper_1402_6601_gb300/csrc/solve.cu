// Forward and back substitution with the Cholesky factor, L Y = B then L^T X = Y.
//
// The right-hand sides are cut into 32-row blocks r and groups g of up to 64 columns. One
// thread block handles one item (r, g) at a time: it accumulates B_r - sum_m L_rm Y_m over
// the blocks m already solved (forward; L_mr^T X_m over m > r backward), waiting on each
// m's ready flag, then solves the 32 x 32 diagonal block and publishes Y_r. Items are
// claimed from an atomic counter in solve order, so every item waits only on items that
// were claimed earlier and are held by running blocks: the sweep always progresses, with
// or without co-residency. Waits are bounded (timeout -> CHOL_INFO_TIMEOUT in *dInfo).
//
// The kernel is instantiated for FP64 (chol_solve) and FP32 (the low-precision solves of
// the mixed-precision refinement). In FP64 both sweeps are bound by the FP64 pipe (n^2 nrhs
// fused multiply-adds against n^2/2 * 8 bytes of L).
#include <algorithm>
#include <mutex>
#include "common.cuh"
#include "blockacc.cuh"
#include "internal.cuh"

namespace chol {

constexpr int SB = 32;   // rows per block
constexpr int SG = 64;   // right-hand sides per group
constexpr int SNT = 256;
constexpr int SLD = SB + 1;
constexpr int SOLVE_EXCL_SMEM = 120 * 1024;  // unused bytes that keep the SM to one block

struct SolveCtrl {
  unsigned int next_item;
  int abort;
  int info;
  int pad[61];
};

struct SolveArgs {
  const void *L;  // T, by the kernel instantiation
  int64_t lda;
  void *B;
  int64_t ldb;
  int n, nrhs, nrb, ngroups;
  int64_t nitems;
  int trans;  // 0: L Y = B (forward), 1: L^T X = B (backward)
  int64_t timeout_ns;
  SolveCtrl *ctrl;
  const int *prev_abort;  // abort flag of the sweep that produced B (nullable)
  const int *skip;        // when set (nonzero) on entry, the launch does nothing (nullable)
  int *flags;
};

// b / d from r = RN(1/d) with one Markstein correction step (see the tile bodies): the
// correctly rounded quotient in three dependent operations.
template <class T>
__device__ __forceinline__ T squot(T b, T d, T r) {
  const T x = b * r;
  const T e = fma(-x, d, b);
  return fma(e, r, x);
}

template <class T, int CPT>
__global__ void __launch_bounds__(SNT, 1) solve_kernel(const __grid_constant__ SolveArgs a) {
  __shared__ T Ls[SB * SLD];  // off-diagonal block of the current step
  __shared__ T Ld[SB * SLD];  // diagonal block of the item (prefetched)
  __shared__ T Ys[SB * SG];
  __shared__ T Red[SB * SG];  // k-slice partial sums
  __shared__ T Rs[SB];        // reciprocals of the diagonal
  __shared__ long long s_item;
  __shared__ int s_abort;
  const T *L = static_cast<const T *>(a.L);
  T *B = static_cast<T *>(a.B);
  if (a.skip && ld_volatile(a.skip)) return;
  const int tid = threadIdx.x;
  const int rr = tid & 31, warp = tid >> 5;
  while (true) {
    if (tid == 0) {
      s_abort = ld_volatile(&a.ctrl->abort) || (a.prev_abort && ld_volatile(a.prev_abort));
      s_item = s_abort ? -1 : (long long)atomicAdd(&a.ctrl->next_item, 1u);
    }
    __syncthreads();
    const long long item = s_item;
    if (item < 0 || item >= a.nitems) break;
    const int g = (int)(item % a.ngroups);
    const int ord = (int)(item / a.ngroups);
    const int r = a.trans ? a.nrb - 1 - ord : ord;
    const int r0 = r * SB, rows = min(SB, a.n - r0);
    const int c0 = g * SG, cols = min(SG, a.nrhs - c0);
    const Slices<CPT> sl(cols, warp);
    // the diagonal block and its reciprocals do not depend on other items: load them now,
    // off the chain of waits. Rows past the end of the matrix get an identity block, so
    // the substitution runs over a fixed 32 rows with register-resident data.
    for (int e = tid; e < SB * SB; e += SNT) {
      const int i = e & 31, j = e >> 5;
      Ld[i * SLD + j] = (i < rows && j < rows && i >= j) ? __ldcg(L + (int64_t)(r0 + j) * a.lda + r0 + i)
                                                          : (i == j ? T(1) : T(0));
    }
    if (tid < SB) Rs[tid] = tid < rows ? T(1) / __ldcg(L + (int64_t)(r0 + tid) * a.lda + r0 + tid) : T(1);
    T acc[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int c = sl.col(q);
      acc[q] = (sl.kslice == 0 && rr < rows && c < cols) ? __ldcg(B + (int64_t)(c0 + c) * a.ldb + r0 + rr) : T(0);
    }
    // blocks are consumed in the order the sweep produces them (forward: 0, 1, ...;
    // backward: nrb-1, nrb-2, ...), so an item only waits on the newest block it needs
    const int nsteps = a.trans ? a.nrb - 1 - r : r;
    for (int step = 0; step < nsteps; ++step) {
      const int m = a.trans ? a.nrb - 1 - step : step;
      const int m0 = m * SB, mrows = min(SB, a.n - m0);
      // L block into Ls as Ls[row of the r block][k] (forward: L_rm; backward: L_mr^T)
      for (int e = tid; e < SB * SB; e += SNT) {
        const int i = e & 31, j = e >> 5;
        if (!a.trans) {  // element (r0+i, m0+j)
          Ls[i * SLD + j] = (i < rows && j < mrows) ? __ldcg(L + (int64_t)(m0 + j) * a.lda + r0 + i) : T(0);
        } else {         // element (m0+i, r0+j) stored at [j][i]
          Ls[j * SLD + i] = (i < mrows && j < rows) ? __ldcg(L + (int64_t)(r0 + j) * a.lda + m0 + i) : T(0);
        }
      }
      // wait until block m of this group is solved
      if (tid == 0) {
        const uint64_t t0 = globaltimer_ns();
        int64_t spins = 0;
        unsigned slp = 32;
        while (ld_volatile(&a.flags[(int64_t)m * a.ngroups + g]) == 0) {
          if (ld_volatile(&a.ctrl->abort)) { s_abort = 1; break; }
          if (globaltimer_ns() - t0 > (uint64_t)a.timeout_ns || ++spins > (a.timeout_ns >> 7) + 100000) {
            atomicCAS(&a.ctrl->info, 0, CHOL_INFO_TIMEOUT);
            atomicExch(&a.ctrl->abort, 1);
            s_abort = 1;
            break;
          }
          __nanosleep(slp);
          slp = slp < 128 ? slp * 2 : 128;
        }
        __threadfence();
      }
      __syncthreads();
      if (s_abort) break;
      for (int e = tid; e < SB * SG; e += SNT) {
        const int k = e & 31, c = e >> 5;
        Ys[k * SG + c] = (k < mrows && c < cols) ? __ldcg(B + (int64_t)(c0 + c) * a.ldb + m0 + k) : T(0);
      }
      __syncthreads();
      acc_step<T, CPT>(acc, Ls, SLD, Ys, SG, rr, sl);
      __syncthreads();
    }
    if (s_abort) break;
    acc_finish<T, CPT>(acc, Ys, SG, Red, rr, cols, sl);
    // diagonal block: one thread per right-hand side runs the substitution, so every FP64
    // instruction of the block does useful work (the FP64 pipe, not latency, bounds it)
    if (tid < cols) {
      const int c = tid;
      T x[SB];
#pragma unroll
      for (int i = 0; i < SB; ++i) x[i] = Ys[i * SG + c];
      // right-looking: once x_k is known every later row is updated at once, so each x_k
      // is one quotient and one multiply-add after x_{k-1}
      if (!a.trans) {
#pragma unroll
        for (int k = 0; k < SB; ++k) {
          x[k] = squot(x[k], Ld[k * SLD + k], Rs[k]);
#pragma unroll
          for (int i = k + 1; i < SB; ++i) x[i] = fma(-Ld[i * SLD + k], x[k], x[i]);
        }
      } else {
#pragma unroll
        for (int k = SB - 1; k >= 0; --k) {
          x[k] = squot(x[k], Ld[k * SLD + k], Rs[k]);
#pragma unroll
          for (int i = 0; i < k; ++i) x[i] = fma(-Ld[k * SLD + i], x[k], x[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < SB; ++i)
        if (i < rows) __stcg(B + (int64_t)(c0 + c) * a.ldb + r0 + i, x[i]);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) *(volatile int *)&a.flags[(int64_t)r * a.ngroups + g] = 1;
  }
}

__global__ void solve_info_kernel(const SolveCtrl *c0, const SolveCtrl *c1, int *dInfo) {
  if (threadIdx.x == 0) *dInfo = c0->info ? c0->info : (c1 ? c1->info : 0);
}

// workspace: two control blocks (one per sweep) and two flag arrays
static size_t flags_bytes(int n, int nrhs) {
  const int64_t nrb = (n + SB - 1) / SB;
  const int64_t ng = (nrhs + SG - 1) / SG;
  return align_up((size_t)std::max<int64_t>(1, nrb * ng) * 4, 256);
}
static size_t solve_ws(int n, int nrhs) { return 512 + 2 * flags_bytes(n, nrhs); }

size_t solve_workspace_bytes(int n, int nrhs) { return solve_ws(n, nrhs); }

template <class T, int CPT>
static cudaError_t launch_solve(const SolveArgs &a, int grid, cudaStream_t s) {
  // one block per SM: the dynamic shared memory request (more than half an SM's) makes a
  // second block impossible
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(solve_kernel<T, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_EXCL_SMEM);
  });
  solve_kernel<T, CPT><<<grid, SNT, SOLVE_EXCL_SMEM, s>>>(a);
  return cudaGetLastError();
}

template <class T>
static chol_status launch_sweep(int trans, int slot, int n, int nrhs, const T *dL, int lda, T *dB, int ldb,
                                void *dWork, const int *skip, cudaStream_t s) {
  SolveArgs a;
  a.L = dL; a.lda = lda; a.B = dB; a.ldb = ldb; a.n = n; a.nrhs = nrhs;
  a.nrb = (n + SB - 1) / SB;
  a.ngroups = (nrhs + SG - 1) / SG;
  a.nitems = (int64_t)a.nrb * a.ngroups;
  a.trans = trans;
  a.timeout_ns = 10000000000ll;
  a.skip = skip;
  unsigned char *ws = static_cast<unsigned char *>(dWork);
  a.ctrl = reinterpret_cast<SolveCtrl *>(ws + 256 * slot);
  a.prev_abort = slot == 1 ? &reinterpret_cast<SolveCtrl *>(ws)->abort : nullptr;
  a.flags = reinterpret_cast<int *>(ws + 512 + flags_bytes(n, nrhs) * slot);
  CHOL_CUDA_TRY(cudaMemsetAsync(a.ctrl, 0, 256, s));
  CHOL_CUDA_TRY(cudaMemsetAsync(a.flags, 0, flags_bytes(n, nrhs), s));
  // One block per SM: FP64 work of a second block on the same SM would starve the
  // dependent chain of the diagonal solves (a dependent FP64 operation waits behind every
  // queued FP64 instruction of the SM). The dynamic shared memory request (more than half
  // of an SM's) makes a second block impossible.
  const DeviceInfo di = current_device_info();
  const int64_t grid = std::min<int64_t>(a.nitems, (int64_t)std::max(1, di.sms));
  const int cpt = cpt_for(std::min(nrhs, SG));
  cudaError_t e;
  if (cpt == 8) e = launch_solve<T, 8>(a, (int)grid, s);
  else if (cpt == 4) e = launch_solve<T, 4>(a, (int)grid, s);
  else if (cpt == 2) e = launch_solve<T, 2>(a, (int)grid, s);
  else e = launch_solve<T, 1>(a, (int)grid, s);
  CHOL_CUDA_TRY(e);
  return CHOL_OK;
}

static chol_status write_info(void *dWork, int slots, int *dInfo, cudaStream_t s) {
  if (!dInfo) return CHOL_OK;
  unsigned char *ws = static_cast<unsigned char *>(dWork);
  const SolveCtrl *c0 = reinterpret_cast<const SolveCtrl *>(ws);
  const SolveCtrl *c1 = slots > 1 ? reinterpret_cast<const SolveCtrl *>(ws + 256) : nullptr;
  solve_info_kernel<<<1, 32, 0, s>>>(c0, c1, dInfo);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

static chol_status check_args(int n, int nrhs, const void *dL, int lda, void *dB, int ldb, void *dWork,
                              size_t work_bytes) {
  if (n < 0 || nrhs < 0) return CHOL_ERR_INVALID_ARG;
  if (lda < std::max(1, n) || ldb < std::max(1, n)) return CHOL_ERR_INVALID_ARG;
  if (n > 0 && nrhs > 0 && (!dL || !dB)) return CHOL_ERR_INVALID_ARG;
  if (n > 0 && nrhs > 0 && (!dWork || work_bytes < solve_ws(n, nrhs) || ((uintptr_t)dWork & 255)))
    return CHOL_ERR_WORKSPACE;
  return CHOL_OK;
}

// FP32 forward + back substitution in place on dB (n x nrhs), skipped when *skip != 0.
chol_status solve_f32(int n, int nrhs, const float *dL, int lda, float *dB, int ldb, void *dWork,
                      const int *skip, cudaStream_t s) {
  if (n == 0 || nrhs == 0) return CHOL_OK;
  chol_status r = launch_sweep<float>(0, 0, n, nrhs, dL, lda, dB, ldb, dWork, skip, s);
  if (r != CHOL_OK) return r;
  return launch_sweep<float>(1, 1, n, nrhs, dL, lda, dB, ldb, dWork, skip, s);
}

}  // namespace chol

using namespace chol;

extern "C" size_t chol_solve_workspace_size(int n, int nrhs) {
  if (n < 0 || nrhs < 0) return 0;
  return solve_ws(n, nrhs);
}

extern "C" chol_status chol_trsm_sweep(int uplo_t, int n, int nrhs, const double *dL, int lda,
                                       double *dB, int ldb, void *dWork, size_t work_bytes,
                                       int *dInfo, void *stream) {
  const chol_status st = check_args(n, nrhs, dL, lda, dB, ldb, dWork, work_bytes);
  if (st != CHOL_OK) return st;
  if (uplo_t != 0 && uplo_t != 1) return CHOL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0 || nrhs == 0) {
    if (dInfo) CHOL_CUDA_TRY(cudaMemsetAsync(dInfo, 0, sizeof(int), s));
    return CHOL_OK;
  }
  const chol_status r = launch_sweep<double>(uplo_t, 0, n, nrhs, dL, lda, dB, ldb, dWork, nullptr, s);
  if (r != CHOL_OK) return r;
  return write_info(dWork, 1, dInfo, s);
}

extern "C" chol_status chol_solve(int n, int nrhs, const double *dL, int lda, double *dB, int ldb,
                                  void *dWork, size_t work_bytes, int *dInfo, void *stream) {
  const chol_status st = check_args(n, nrhs, dL, lda, dB, ldb, dWork, work_bytes);
  if (st != CHOL_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0 || nrhs == 0) {
    if (dInfo) CHOL_CUDA_TRY(cudaMemsetAsync(dInfo, 0, sizeof(int), s));
    return CHOL_OK;
  }
  chol_status r = launch_sweep<double>(0, 0, n, nrhs, dL, lda, dB, ldb, dWork, nullptr, s);
  if (r != CHOL_OK) return r;
  // the backward sweep skips its work if the forward one aborted
  r = launch_sweep<double>(1, 1, n, nrhs, dL, lda, dB, ldb, dWork, nullptr, s);
  if (r != CHOL_OK) return r;
  return write_info(dWork, 2, dInfo, s);
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of chol_solve. Its workspace is a fixed array of this library in
// device global memory, so the caller needs no device allocation at all.

namespace chol {

constexpr size_t SOLVE_NOALLOC_BYTES = 256 * 1024;
static __device__ __align__(256) unsigned char g_solve_scratch[SOLVE_NOALLOC_BYTES];

// Device address of g_solve_scratch on device `dev` (which must be current). In host code
// the symbol's name is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress and cached.
static void *noalloc_scratch(int dev, cudaError_t *err) {
  static std::mutex mu;
  static void *ptrs[128] = {};
  if (dev < 0 || dev >= 128) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!ptrs[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);
    if (e != cudaSuccess) {
      *err = e;
      return nullptr;
    }
    ptrs[dev] = p;
  }
  *err = cudaSuccess;
  return ptrs[dev];
}

}  // namespace chol

extern "C" chol_status chol_solve_noalloc(int n, int nrhs, const double *dL, int lda, double *dB,
                                          int ldb, int *dInfo, void *stream) {
  if (n < 0 || nrhs < 0) return CHOL_ERR_INVALID_ARG;
  if (solve_ws(n, nrhs) > SOLVE_NOALLOC_BYTES) return CHOL_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CHOL_ERR_CUDA;
  cudaError_t err = cudaSuccess;
  void *scratch = noalloc_scratch(dev, &err);
  if (!scratch) return CHOL_ERR_CUDA;
  // the sweeps clear the control blocks and flags they use before every launch
  return chol_solve(n, nrhs, dL, lda, dB, ldb, scratch, SOLVE_NOALLOC_BYTES, dInfo, stream);
}
