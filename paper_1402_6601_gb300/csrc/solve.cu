// Forward and back substitution with the Cholesky factor, L Y = B then L^T X = Y.
//
// The right-hand sides are cut into 32-row blocks r and groups g of up to 32 columns. One
// thread block handles one item (r, g) at a time: it accumulates B_r - sum_m L_rm Y_m over
// the blocks m already solved (forward; L_mr^T X_m over m > r backward), then solves its
// 32 x 32 diagonal block and publishes Y_r with a ready flag. Items are claimed from an
// atomic counter in solve order, so every item waits only on items that were claimed earlier
// and are held by running blocks: the sweep always progresses, with or without co-residency.
//
// Inside an item the eight warps split the blocks m (warp w takes m = w, w + 8, ... in the
// order the sweep produces them) and work independently: a warp loads its L block, obtains
// Y_m, stages it in its own shared-memory rows and accumulates into registers (lane = row of
// the item, one register per right-hand side). The block synchronises once per item, to add
// the eight partial sums.
//
// A solved block publishes a ready flag after a release fence; a warp checks the flags of its
// next 32 blocks with one load per lane (blocks solved long ago cost no polling round trip)
// and polls only a block that is not ready yet. Waits are bounded (timeout ->
// CHOL_INFO_TIMEOUT in *dInfo). In FP32 (the refinement's sweeps) the 32 x 32 diagonal block
// is inverted while the item accumulates, so the chain only carries its product with the
// block; FP64 keeps the substitution (exact on integer data).
//
// The kernel is instantiated for FP64 (chol_solve) and FP32 (the low-precision solves of
// the mixed-precision refinement). In FP64 both sweeps are bound by the FP64 pipe (n^2 nrhs
// fused multiply-adds against n^2/2 * 8 bytes of L).
#include <algorithm>
#include <mutex>
#include "common.cuh"
#include "internal.cuh"

namespace chol {

constexpr int SB = 32;   // rows per block
constexpr int SG = 32;   // right-hand sides per group (one accumulator register per lane each)
constexpr int SNT = 256;
constexpr int SNW = SNT / 32;
constexpr int SLD = SB + 1;
constexpr int SOLVE_EXCL_SMEM = 120 * 1024;  // at least this much, so an SM holds one block

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

// shared memory of solve_kernel<T, NC>, in elements of T
template <class T, int NC>
struct SolveSmem {
  static constexpr int V = 16 / (int)sizeof(T) < NC ? 16 / (int)sizeof(T) : NC;  // vector width
  static constexpr int YLD = NC + 16 / (int)sizeof(T);  // row stride: 16-byte rows, no conflicts
  static constexpr size_t YW = (size_t)SNW * SB * YLD;  // per-warp Y_m rows, later partial sums
  static constexpr size_t LT = (size_t)SNW * SB * SLD;  // per-warp transposed L block (backward)
  static constexpr size_t YS = (size_t)SB * YLD;        // the item's block before the diagonal solve
  static constexpr size_t LD = (size_t)SB * SLD + SB;   // diagonal block and its reciprocals
  static constexpr size_t DI = (size_t)SB * SLD;        // inverse of the diagonal block (FP32)
  static constexpr size_t NEED = (YW + LT + YS + LD + DI) * sizeof(T);
  static constexpr size_t BYTES = NEED > (size_t)SOLVE_EXCL_SMEM ? NEED : (size_t)SOLVE_EXCL_SMEM;
};

template <class T, int V>
struct VecOf;
template <> struct VecOf<float, 4> { using type = float4; };
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<double, 2> { using type = double2; };
template <> struct VecOf<double, 1> { using type = double; };

template <class T, int V>
__device__ __forceinline__ void vload(const T *p, T (&v)[V]) {
  using VT = typename VecOf<T, V>::type;
  const VT x = *reinterpret_cast<const VT *>(p);
  const T *e = reinterpret_cast<const T *>(&x);
#pragma unroll
  for (int u = 0; u < V; ++u) v[u] = e[u];
}

template <class T, int NC>
__global__ void __launch_bounds__(SNT, 1) solve_kernel(const __grid_constant__ SolveArgs a) {
  using S = SolveSmem<T, NC>;
  constexpr int V = S::V, YLD = S::YLD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Yw = reinterpret_cast<T *>(smem_raw);
  T *Lt = Yw + S::YW;
  T *Ys = Lt + S::LT;
  T *Ld = Ys + S::YS;
  T *Rs = Ld + SB * SLD;
  T *Di = Rs + SB;
  constexpr bool INV = sizeof(T) == 4;  // FP32: multiply by the inverted diagonal block
  __shared__ long long s_item;
  __shared__ int s_abort;
  const T *L = static_cast<const T *>(a.L);
  T *B = static_cast<T *>(a.B);
  if (a.skip && ld_volatile(a.skip)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T *yw = Yw + (size_t)warp * SB * YLD;
  T *lt = Lt + (size_t)warp * SB * SLD;
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
    // the diagonal block and its reciprocals do not depend on other items: load them now,
    // off the chain of waits. Rows past the end of the matrix get an identity block, so the
    // substitution runs over a fixed 32 rows with register-resident data.
    for (int e = tid; e < SB * SB; e += SNT) {
      const int i = e & 31, j = e >> 5;
      Ld[i * SLD + j] = (i < rows && j < rows && i >= j) ? __ldcg(L + (int64_t)(r0 + j) * a.lda + r0 + i)
                                                          : (i == j ? T(1) : T(0));
    }
    if (tid < SB) Rs[tid] = tid < rows ? T(1) / __ldcg(L + (int64_t)(r0 + tid) * a.lda + r0 + tid) : T(1);
    if (INV) {
      // D^-1 by columns: lane j of warp 0 solves D y = e_j (right-looking, register resident;
      // y stays zero above row j, so no lane needs a predicate), while the other warps start
      // accumulating. Identity padding past the end of the matrix gives an identity inverse.
      __syncthreads();
      if (warp == 0) {
        T y[SB];
#pragma unroll
        for (int i = 0; i < SB; ++i) y[i] = i == lane ? T(1) : T(0);
#pragma unroll
        for (int k = 0; k < SB; ++k) {
          y[k] = squot(y[k], Ld[k * SLD + k], Rs[k]);
#pragma unroll
          for (int i = k + 1; i < SB; ++i) y[i] = fma(-Ld[i * SLD + k], y[k], y[i]);
        }
#pragma unroll
        for (int i = 0; i < SB; ++i) Di[i * SLD + lane] = y[i];
      }
    }
    // this thread's entries of B_r for the final sum, loaded now (off the chain)
    constexpr int BPT = (SB * NC + SNT - 1) / SNT;
    T bv[BPT];
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      const int e = tid + u * SNT, i = e & (SB - 1), q = e >> 5;
      bv[u] = (e < SB * NC && i < rows && q < cols) ? __ldcg(B + (int64_t)(c0 + q) * a.ldb + r0 + i) : T(0);
    }
    // warp-parallel accumulation over the solved blocks
    T acc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = T(0);
    const int nsteps = a.trans ? a.nrb - 1 - r : r;
    int wab = 0;
    // readiness of the warp's next 32 blocks: bit j <-> step mbase + SNW j, one flag load per
    // lane and a ballot, so blocks solved long ago cost no polling round trip
    unsigned ready = 0u;
    int mbase = warp;
    for (int step = warp; step < nsteps; step += SNW) {
      const int m = a.trans ? a.nrb - 1 - step : step;
      const int m0 = m * SB, mrows = min(SB, a.n - m0);
      // L block, issued before any wait (it does not depend on other items). Forward: lane =
      // row of the item, lr[k] = L_rm(lane, k). Backward: lane = row k of block m,
      // lr[i] = L_mr(lane, i), staged transposed below.
      T lr[SB];
      if (!a.trans) {
#pragma unroll
        for (int k = 0; k < SB; ++k)
          lr[k] = (lane < rows && k < mrows) ? __ldcg(L + (int64_t)(m0 + k) * a.lda + r0 + lane) : T(0);
      } else {
#pragma unroll
        for (int i = 0; i < SB; ++i)
          lr[i] = (lane < mrows && i < rows) ? __ldcg(L + (int64_t)(r0 + i) * a.lda + m0 + lane) : T(0);
      }
      T yv[NC];
      int jb = (step - mbase) / SNW;
      if (jb >= 32 || !((ready >> jb) & 1u)) {
        const int sl = step + SNW * lane;
        int f = 1;
        if (sl < nsteps) {
          const int ml = a.trans ? a.nrb - 1 - sl : sl;
          f = ld_volatile(&a.flags[(int64_t)ml * a.ngroups + g]) != 0;
        }
        ready = __ballot_sync(0xffffffffu, f);
        mbase = step;
        jb = 0;
        if (!(ready & 1u)) {
          // wait until block m of this group is solved (one lane, bounded)
          if (lane == 0) {
            const uint64_t t0 = globaltimer_ns();
            int64_t spins = 0;
            unsigned slp = 32;
            while (ld_volatile(&a.flags[(int64_t)m * a.ngroups + g]) == 0) {
              if (ld_volatile(&a.ctrl->abort)) { wab = 1; break; }
              if (globaltimer_ns() - t0 > (uint64_t)a.timeout_ns || ++spins > (a.timeout_ns >> 7) + 100000) {
                atomicCAS(&a.ctrl->info, 0, CHOL_INFO_TIMEOUT);
                atomicExch(&a.ctrl->abort, 1);
                wab = 1;
                break;
              }
              __nanosleep(slp);
              slp = slp < 128 ? slp * 2 : 128;
            }
          }
          wab = __shfl_sync(0xffffffffu, wab, 0);
          if (wab) break;
          ready = 1u;  // only this block is known to be solved
        }
        // every flag this warp observed is ordered before the loads of the blocks' data
        __threadfence();
        __syncwarp();
      }
      // Y block m (lane k stages row k), loaded once the block is known to be solved
#pragma unroll
      for (int q = 0; q < NC; ++q)
        yv[q] = (lane < mrows && q < cols) ? __ldcg(B + (int64_t)(c0 + q) * a.ldb + m0 + lane) : T(0);
#pragma unroll
      for (int q = 0; q < NC; ++q) yw[lane * YLD + q] = yv[q];
      if (a.trans) {
#pragma unroll
        for (int i = 0; i < SB; ++i) lt[lane * SLD + i] = lr[i];
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < SB; ++k) {
        const T l = a.trans ? lt[k * SLD + lane] : lr[k];
#pragma unroll
        for (int q = 0; q < NC; q += V) {
          T y[V];
          vload<T, V>(yw + k * YLD + q, y);
#pragma unroll
          for (int u = 0; u < V; ++u) acc[q + u] = fma(l, y[u], acc[q + u]);
        }
      }
      __syncwarp();
    }
    if (wab && lane == 0) s_abort = 1;
    // the eight partial sums: into the warps' rows, then B_r minus their sum into Ys
#pragma unroll
    for (int q = 0; q < NC; ++q) yw[lane * YLD + q] = acc[q];
    __syncthreads();
    if (s_abort) break;
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      const int e = tid + u * SNT, i = e & (SB - 1), q = e >> 5;
      if (e < SB * NC) {
        T sum = T(0);
#pragma unroll
        for (int w = 0; w < SNW; ++w) sum += Yw[(size_t)w * SB * YLD + i * YLD + q];
        Ys[i * YLD + q] = bv[u] - sum;
      }
    }
    __syncthreads();
    T *Xo = Ys;  // the solved block, row-major with stride YLD
    if (INV) {
      // forward x = D^-1 (b - sum), backward x = D^-T (b - sum): independent 32-term
      // products (D^-1 is zero above the diagonal)
      Xo = Yw;     // free once the partial sums are added
#pragma unroll
      for (int u = 0; u < (SB * NC + SNT - 1) / SNT; ++u) {
        const int e = tid + u * SNT, i = e & (SB - 1), q = e >> 5;
        if (e < SB * NC) {
          T t = T(0);
#pragma unroll
          for (int k = 0; k < SB; ++k) t = fma(a.trans ? Di[k * SLD + i] : Di[i * SLD + k], Ys[k * YLD + q], t);
          Xo[i * YLD + q] = t;
        }
      }
    } else if (tid < cols) {
      // diagonal block: one thread per right-hand side runs the substitution
      const int c = tid;
      T x[SB];
#pragma unroll
      for (int i = 0; i < SB; ++i) x[i] = Ys[i * YLD + c];
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
      for (int i = 0; i < SB; ++i) Ys[i * YLD + c] = x[i];
    }
    __syncthreads();
    // write the solved block column by column (one warp per column: 32 consecutive rows)
    for (int c = warp; c < cols; c += SNW)
      if (lane < rows) __stcg(B + (int64_t)(c0 + c) * a.ldb + r0 + lane, Xo[lane * YLD + c]);
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

template <class T, int NC>
static cudaError_t launch_solve(const SolveArgs &a, int grid, cudaStream_t s) {
  // one block per SM: the dynamic shared memory request (more than half an SM's) makes a
  // second block impossible
  constexpr size_t bytes = SolveSmem<T, NC>::BYTES;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(solve_kernel<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  });
  solve_kernel<T, NC><<<grid, SNT, bytes, s>>>(a);
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
  // accumulator registers per lane: the smallest power of two that holds a group
  const int w = std::min(nrhs, SG);
  cudaError_t e;
  if (w <= 1) e = launch_solve<T, 1>(a, (int)grid, s);
  else if (w <= 2) e = launch_solve<T, 2>(a, (int)grid, s);
  else if (w <= 4) e = launch_solve<T, 4>(a, (int)grid, s);
  else if (w <= 8) e = launch_solve<T, 8>(a, (int)grid, s);
  else if (w <= 16) e = launch_solve<T, 16>(a, (int)grid, s);
  else e = launch_solve<T, 32>(a, (int)grid, s);
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
