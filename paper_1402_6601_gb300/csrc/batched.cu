// Batched factor + solve of many independent small SPD matrices in one persistent launch (not
// in the paper: its factorization applied to a batch of uneven sizes).
//
// The batch is ordered on the device by decreasing order n (a counting sort in one block, so
// no host round trip is needed and the whole sequence can be captured into a CUDA graph);
// each worker block then claims the next matrix from an atomic counter (largest first, the
// longest-processing-time rule that keeps the tail short) and factors it alone with the
// blocked POTRF tile body of the factorization (32-column panels, DFMA or FFMA updates),
// then runs forward and back substitution on its right-hand side. Matrices are independent,
// so there is no dependency wait: the only shared state is the counter.
#include <algorithm>
#include <mutex>
#include "common.cuh"
#include "internal.cuh"
#include "tiles_f32.cuh"
#include "tiles_f64.cuh"

namespace chol {

constexpr int BATCH_MAX_N = 4096;

struct BatchArgs {
  int batch;
  const int *N;
  void *const *A;
  const int *lda;
  void *const *B;  // nullable: factor only; a null entry skips that matrix's solve
  int *info;
  const int *order;
  unsigned int *counter;
  int solve_only;  // 1: A already holds the factors; only the substitutions run
  int wide_min_n;  // FP64 members of at least this order use 64-column panels
};

// order = indices sorted by decreasing N (ties in any order), or the identity; counter = 0
__global__ void __launch_bounds__(1024) batch_order_kernel(int batch, const int *N, int *order, int lpt,
                                                           unsigned int *counter) {
  __shared__ int hist[BATCH_MAX_N + 2];
  if (threadIdx.x == 0) *counter = 0u;
  if (!lpt) {
    for (int i = threadIdx.x; i < batch; i += blockDim.x) order[i] = i;
    return;
  }
  for (int b = threadIdx.x; b < BATCH_MAX_N + 2; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < batch; i += blockDim.x) {
    const int n = min(max(N[i], 0), BATCH_MAX_N);
    atomicAdd(&hist[BATCH_MAX_N - n], 1);  // bin 0 = largest n
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive prefix sum over the bins
    int run = 0;
    for (int b = 0; b < BATCH_MAX_N + 1; ++b) {
      const int c = hist[b];
      hist[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < batch; i += blockDim.x) {
    const int n = min(max(N[i], 0), BATCH_MAX_N);
    order[atomicAdd(&hist[BATCH_MAX_N - n], 1)] = i;
  }
}

// b / d from r = RN(1/d) with one Markstein correction: the correctly rounded quotient (the
// same value as b / d) in three dependent operations after r, which is taken for all 32
// diagonal entries of a block at once, off the substitution's chain.
template <class T>
__device__ __forceinline__ T bquot(T b, T d, T r) {
  const T x = b * r;
  const T e = fma(-x, d, b);
  return fma(e, r, x);
}

// Forward and back substitution L L^T x = b for one matrix by the whole block; b in place.
// 32-row blocks: warp 0 solves the diagonal block (lanes = rows, x_k broadcast by shuffle),
// then all threads update the remaining rows with that block's columns. The L values a lane
// or a thread needs for a block are loaded into registers before its chain of dependent
// operations starts, so the chain waits for memory once per block, not once per step (L was
// just written through L2 by the factor).
template <class T>
__device__ void block_solve_vec(const T *L, int64_t lda, int n, T *b, T *xs) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < n; i += blockDim.x) xs[i] = b[i];
  __syncthreads();
  for (int p = 0; p < n; p += 32) {  // L y = b
    const int pb = min(32, n - p);
    if (tid < 32) {
      T lr[32];  // row p + lane of the diagonal block
#pragma unroll
      for (int k = 0; k < 32; ++k) lr[k] = (lane < pb && k < pb) ? L[(int64_t)(p + k) * lda + p + lane] : T(0);
      T y = lane < pb ? xs[p + lane] : T(0);
      const T dl = lane < pb ? L[(int64_t)(p + lane) * lda + p + lane] : T(1);
      const T rl = T(1) / dl;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if (k < pb) {
          const T yk = bquot(__shfl_sync(0xffffffffu, y, k), __shfl_sync(0xffffffffu, dl, k),
                             __shfl_sync(0xffffffffu, rl, k));
          if (lane == k) y = yk;
          else if (lane > k && lane < pb) y = fma(-lr[k], yk, y);
        }
      }
      if (lane < pb) xs[p + lane] = y;
    }
    __syncthreads();
    for (int i = p + pb + tid; i < n; i += blockDim.x) {
      T lv[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) lv[k] = k < pb ? L[(int64_t)(p + k) * lda + i] : T(0);
      T t = xs[i];
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k < pb) t = fma(-lv[k], xs[p + k], t);
      xs[i] = t;
    }
    __syncthreads();
  }
  for (int p0 = ((n - 1) / 32) * 32; p0 >= 0; p0 -= 32) {  // L^T x = y
    const int pb = min(32, n - p0);
    if (tid < 32) {
      T lc[32];  // column p0 + lane of the diagonal block (contiguous)
#pragma unroll
      for (int k = 0; k < 32; ++k) lc[k] = (lane < pb && k < pb) ? L[(int64_t)(p0 + lane) * lda + p0 + k] : T(0);
      T x = lane < pb ? xs[p0 + lane] : T(0);
      const T dl = lane < pb ? L[(int64_t)(p0 + lane) * lda + p0 + lane] : T(1);
      const T rl = T(1) / dl;
#pragma unroll
      for (int k = 31; k >= 0; --k) {
        if (k < pb) {
          const T xk = bquot(__shfl_sync(0xffffffffu, x, k), __shfl_sync(0xffffffffu, dl, k),
                             __shfl_sync(0xffffffffu, rl, k));
          if (lane == k) x = xk;
          else if (lane < k) x = fma(-lc[k], xk, x);
        }
      }
      if (lane < pb) xs[p0 + lane] = x;
    }
    __syncthreads();
    for (int i = tid; i < p0; i += blockDim.x) {
      T lv[32];  // row p0.. of column i (contiguous)
#pragma unroll
      for (int k = 0; k < 32; ++k) lv[k] = k < pb ? L[(int64_t)i * lda + p0 + k] : T(0);
      T t = xs[i];
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k < pb) t = fma(-lv[k], xs[p0 + k], t);
      xs[i] = t;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += blockDim.x) b[i] = xs[i];
  __syncthreads();
}

template <class T>
struct BatchTiles;
template <>
struct BatchTiles<double> {
  static constexpr int SMEM = TILE_SMEM_BYTES;
  __device__ static int potrf(double *G, int64_t ld, int n, double *s, int pw) { return potrf_tile(G, ld, n, s, pw); }
};
template <>
struct BatchTiles<float> {
  static constexpr int SMEM = f32::TILE_SMEM_BYTES;
  __device__ static int potrf(float *G, int64_t ld, int n, float *s, int) { return f32::potrf_tile(G, ld, n, s); }
};

template <class T, int MINB>
__global__ void __launch_bounds__(NT, MINB) batched_kernel(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smem = reinterpret_cast<T *>(smem_raw);
  __shared__ int s_m;
  while (true) {
    if (threadIdx.x == 0) {
      const unsigned int k = atomicAdd(a.counter, 1u);
      s_m = k < (unsigned)a.batch ? a.order[k] : -1;
    }
    __syncthreads();
    const int m = s_m;
    if (m < 0) break;
    const int n = a.N[m];
    T *A = static_cast<T *>(a.A[m]);
    const int lda = a.lda[m];
    if (n > BATCH_MAX_N || lda < max(n, 1) || (n > 0 && !A)) {  // uniform: every thread reads the same
      if (threadIdx.x == 0) a.info[m] = CHOL_INFO_BAD_ARG;
      __syncthreads();
      continue;
    }
    const int f = (n > 0 && !a.solve_only) ? BatchTiles<T>::potrf(A, lda, n, smem, n >= a.wide_min_n ? 64 : 32) : 0;
    if (threadIdx.x == 0) a.info[m] = f;
    if (!f && n > 0 && a.B && a.B[m]) block_solve_vec<T>(A, lda, n, static_cast<T *>(a.B[m]), smem);
    __syncthreads();
  }
}

// dst[m] = src[m] (n x n, the lower triangle is enough for the factor)
template <class T>
__global__ void batch_copy_kernel(int batch, const int *N, void *const *src, void *const *dst, const int *lda) {
  for (int m = blockIdx.x; m < batch; m += gridDim.x) {
    const int n = min(N[m], BATCH_MAX_N);
    const int ld = lda[m];
    const T *S = static_cast<const T *>(src[m]);
    T *D = static_cast<T *>(dst[m]);
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
      const int64_t j = e / n, i = e - j * n;
      if (i >= j) D[j * ld + i] = S[j * ld + i];
    }
  }
}

static size_t batch_ws(int batch) { return 256 + align_up((size_t)std::max(1, batch) * 4, 256); }

template <class T, int MINB>
static cudaError_t launch_batched(const BatchArgs &a, int grid, cudaStream_t s) {
  constexpr int smem = std::max(BatchTiles<T>::SMEM, BATCH_MAX_N * (int)sizeof(T));
  const cudaError_t e = set_smem_attr((const void *)batched_kernel<T, MINB>, smem);
  if (e != cudaSuccess) return e;
  batched_kernel<T, MINB><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <class T>
static int batch_blocks_per_sm(int wps) {
  int occ = 0;
  constexpr int smem = std::max(BatchTiles<T>::SMEM, BATCH_MAX_N * (int)sizeof(T));
  if (wps >= 2) {
    if (set_smem_attr((const void *)batched_kernel<T, 2>, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel<T, 2>, NT, smem) != cudaSuccess) occ = 1;
  } else {
    occ = 1;
  }
  return std::max(1, std::min(occ, wps));
}

}  // namespace chol

using namespace chol;

extern "C" void chol_batch_opts_default(chol_batch_opts *o) {
  if (!o) return;
  o->workers_per_sm = 1;
  o->lpt_order = 1;
  o->wide_panel_min_n = 0;
}

extern "C" size_t chol_batched_workspace_size(int batch) {
  if (batch < 0) return 0;
  return batch_ws(batch);
}

static chol_status batched_impl(int precision, int batch, const int *dN, void *const *dA, const int *dLda,
                                void *const *dB, int *dInfo, const chol_batch_opts *bopts, void *dWork,
                                size_t work_bytes, void *stream, int solve_only) {
  if (batch < 0 || (precision != CHOL_F64 && precision != CHOL_F32)) return CHOL_ERR_INVALID_ARG;
  if (batch == 0) return CHOL_OK;
  if (!dN || !dA || !dLda || !dInfo) return CHOL_ERR_INVALID_ARG;
  if (!dWork || work_bytes < batch_ws(batch) || ((uintptr_t)dWork & 255)) return CHOL_ERR_WORKSPACE;
  chol_batch_opts o;
  chol_batch_opts_default(&o);
  if (bopts) o = *bopts;
  if (o.workers_per_sm < 1 || o.workers_per_sm > 2) return CHOL_ERR_INVALID_ARG;
  const DeviceInfo di = current_device_info();
  if (di.sms <= 0) return CHOL_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *ws = static_cast<unsigned char *>(dWork);
  BatchArgs a;
  a.batch = batch;
  a.N = dN;
  a.A = dA;
  a.lda = dLda;
  a.B = dB;
  a.info = dInfo;
  a.counter = reinterpret_cast<unsigned int *>(ws);
  a.order = reinterpret_cast<int *>(ws + 256);
  a.solve_only = solve_only;
  a.wide_min_n = o.wide_panel_min_n < 0 ? 0 : o.wide_panel_min_n;
  batch_order_kernel<<<1, 1024, 0, s>>>(batch, dN, const_cast<int *>(a.order), o.lpt_order, a.counter);
  CHOL_CUDA_TRY(cudaGetLastError());
  cudaError_t e;
  if (precision == CHOL_F64) {
    const int per = batch_blocks_per_sm<double>(o.workers_per_sm);
    const int grid = std::min(batch, di.sms * per);
    e = per >= 2 ? launch_batched<double, 2>(a, grid, s) : launch_batched<double, 1>(a, grid, s);
  } else {
    const int per = batch_blocks_per_sm<float>(o.workers_per_sm);
    const int grid = std::min(batch, di.sms * per);
    e = per >= 2 ? launch_batched<float, 2>(a, grid, s) : launch_batched<float, 1>(a, grid, s);
  }
  CHOL_CUDA_TRY(e);
  return CHOL_OK;
}

extern "C" chol_status chol_posv_batched(int precision, int batch, const int *dN, void *const *dA, const int *dLda,
                                         void *const *dB, int *dInfo, const chol_batch_opts *bopts, void *dWork,
                                         size_t work_bytes, void *stream) {
  return batched_impl(precision, batch, dN, dA, dLda, dB, dInfo, bopts, dWork, work_bytes, stream, 0);
}

extern "C" chol_status chol_factor_batched(int precision, int batch, const int *dN, void *const *dA,
                                           const int *dLda, int *dInfo, const chol_batch_opts *bopts, void *dWork,
                                           size_t work_bytes, void *stream) {
  return batched_impl(precision, batch, dN, dA, dLda, nullptr, dInfo, bopts, dWork, work_bytes, stream, 0);
}

extern "C" chol_status chol_solve_batched(int precision, int batch, const int *dN, void *const *dL,
                                          const int *dLda, void *const *dB, int *dInfo,
                                          const chol_batch_opts *bopts, void *dWork, size_t work_bytes,
                                          void *stream) {
  if (batch > 0 && !dB) return CHOL_ERR_INVALID_ARG;
  return batched_impl(precision, batch, dN, dL, dLda, dB, dInfo, bopts, dWork, work_bytes, stream, 1);
}

extern "C" chol_status chol_batched_autotune(int precision, int batch, const int *dN, void *const *dAsrc,
                                             void *const *dAscratch, const int *dLda, int *dInfo, void *dWork,
                                             size_t work_bytes, chol_batch_opts *best, float *best_ms,
                                             void *stream) {
  if (!best || batch < 1 || !dAsrc || !dAscratch) return CHOL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const DeviceInfo di = current_device_info();
  if (di.sms <= 0) return CHOL_ERR_CUDA;
  cudaEvent_t e0, e1;
  CHOL_CUDA_TRY(cudaEventCreate(&e0));
  CHOL_CUDA_TRY(cudaEventCreate(&e1));
  float best_t = 1e30f;
  chol_batch_opts cand, win;
  chol_batch_opts_default(&win);
  chol_status st = CHOL_OK;
  // FP64: the order from which members use 64-column panels (none, 384, 256, 128, all)
  const int wide_cands[5] = {BATCH_MAX_N + 1, 384, 256, 128, 0};
  const int nwide = precision == CHOL_F64 ? 5 : 1;
  for (int wps = 1; wps <= 2 && st == CHOL_OK; ++wps) {
    for (int lpt = 0; lpt <= 1 && st == CHOL_OK; ++lpt) {
      for (int wi = 0; wi < nwide && st == CHOL_OK; ++wi) {
        cand.workers_per_sm = wps;
        cand.lpt_order = lpt;
        cand.wide_panel_min_n = precision == CHOL_F64 ? wide_cands[wi] : 0;
        float t = 0.f;
        for (int rep = 0; rep < 2 && st == CHOL_OK; ++rep) {
          if (precision == CHOL_F64)
            batch_copy_kernel<double><<<di.sms * 4, 256, 0, s>>>(batch, dN, dAsrc, dAscratch, dLda);
          else
            batch_copy_kernel<float><<<di.sms * 4, 256, 0, s>>>(batch, dN, dAsrc, dAscratch, dLda);
          if (cudaGetLastError() != cudaSuccess) { st = CHOL_ERR_CUDA; break; }
          if (cudaEventRecord(e0, s) != cudaSuccess) { st = CHOL_ERR_CUDA; break; }
          st = chol_posv_batched(precision, batch, dN, dAscratch, dLda, nullptr, dInfo, &cand, dWork, work_bytes,
                                 stream);
          if (st != CHOL_OK) break;
          if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { st = CHOL_ERR_CUDA; break; }
          cudaEventElapsedTime(&t, e0, e1);  // the second repetition is kept
        }
        if (st == CHOL_OK && t < best_t) {
          best_t = t;
          win = cand;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CHOL_OK) return st;
  *best = win;
  if (best_ms) *best_ms = best_t;
  return CHOL_OK;
}
