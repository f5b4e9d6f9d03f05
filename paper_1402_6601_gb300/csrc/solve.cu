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
  int trans;  // 0: L Y = B (forward), 1: L^T X = B (backward), 2: U X = B (backward, U upper,
              //    the LU solve's back substitution)
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

// shared memory of solve_kernel<T, NC, SBK>, in elements of T (SBK rows per item; L and Y
// blocks are consumed in 32-row chunks)
template <class T, int NC, int SBK>
struct SolveSmem {
  static constexpr int V = 16 / (int)sizeof(T) < NC ? 16 / (int)sizeof(T) : NC;  // vector width
  static constexpr int YLD = NC + 16 / (int)sizeof(T);  // row stride: 16-byte rows, no conflicts
  static constexpr int DLD = SBK + 1;                   // stride of the diagonal block
  static constexpr int MLD = SBK + 4;                   // stride of its inverse: 16-byte columns
  static constexpr size_t YW = (size_t)SNW * SBK * YLD; // per-warp Y chunk, later partial sums
                                                        // (column-major, SBK x NC)
  static constexpr size_t LT = (size_t)SNW * SB * DLD;  // per-warp transposed L chunk (backward)
  static constexpr size_t YS = (size_t)SBK * YLD;       // the item's block before the diagonal solve
  static constexpr size_t LD = (size_t)SBK * DLD + SBK; // diagonal block and its reciprocals
  static constexpr size_t DI = (size_t)SBK * MLD;       // inverse of the diagonal block (FP32)
  // FP32: the newest solved block's L block G and W = D^-1 G (D^-T G backward), k-major
  static constexpr bool NW = sizeof(T) == 4;
  static constexpr size_t GS = NW ? (size_t)SBK * DLD : 0;
  static constexpr size_t WM = NW ? (size_t)SBK * MLD : 0;
  static constexpr size_t NEED = (YW + LT + YS + LD + DI + GS + WM) * sizeof(T);
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

// SBK rows per item: 32 (lane = row) or, in FP32, 64 (lane = rows lane and lane + 32), which
// halves the number of links in the chain of block rows. MODE (a.trans): 0 forward with the
// lower L, 1 backward with L^T, 2 backward with an upper U whose blocks are read like L's in
// the forward sweep (row block r, column block m > r: U(r0 + i, m0 + k) at (m0 + k) lda + r0 + i).
template <class T, int NC, int SBK, int MODE>
__global__ void __launch_bounds__(SNT, 1) solve_kernel(const __grid_constant__ SolveArgs a) {
  using S = SolveSmem<T, NC, SBK>;
  constexpr int V = S::V, YLD = S::YLD, DLD = S::DLD, MLD = S::MLD;
  constexpr int RPL = SBK / 32;         // rows per lane
  constexpr bool INV = sizeof(T) == 4;  // FP32: multiply by the inverted diagonal block
  constexpr bool TRANS = MODE == 1;     // blocks of L read transposed
  constexpr bool REV = MODE != 0;       // blocks solved from the last one up
  // FP64 with many right-hand sides: warps split the columns instead of the solved blocks
  constexpr bool QS = !INV && NC >= 2 * SNW && SBK == 32;
  static_assert(SBK == 32 || (SBK == 64 && INV), "64-row items are for the FP32 sweeps");
  static_assert(MODE != 2 || !INV, "the upper sweep is FP64");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Yw = reinterpret_cast<T *>(smem_raw);
  T *Lt = Yw + S::YW;
  T *Ys = Lt + S::LT;
  T *Ld = Ys + S::YS;
  T *Rs = Ld + SBK * DLD;
  T *Mi = Rs + SBK;  // 16-byte aligned: YW, LT, YS and LD are multiples of four elements
  T *Gs = Mi + S::DI;
  T *Wm = Gs + S::GS;  // 16-byte aligned: DI and GS are multiples of four elements
  __shared__ long long s_item;
  __shared__ int s_abort;
  __shared__ T s_xk[2][32];  // x_k of every column, by step parity (diagonal solve)
  const T *L = static_cast<const T *>(a.L);
  T *B = static_cast<T *>(a.B);
  if (a.skip && ld_volatile(a.skip)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T *yw = Yw + (size_t)warp * SBK * YLD;
  T *lt = Lt + (size_t)warp * SB * DLD;
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
    const int r = REV ? a.nrb - 1 - ord : ord;
    const int r0 = r * SBK, rows = min(SBK, a.n - r0);
    const int c0 = g * SG, cols = min(SG, a.nrhs - c0);
    // the diagonal block and its reciprocals do not depend on other items: load them now,
    // off the chain of waits. Rows past the end of the matrix get an identity block, so the
    // substitution runs over a fixed SBK rows with register-resident data.
    // (MODE 2 stores U^T, so that the backward substitution reads it as it reads L)
    for (int e = tid; e < SBK * SBK; e += SNT) {
      const int i = e % SBK, j = e / SBK;
      const int64_t at = MODE == 2 ? (int64_t)(r0 + i) * a.lda + r0 + j : (int64_t)(r0 + j) * a.lda + r0 + i;
      Ld[i * DLD + j] = (i < rows && j < rows && i >= j) ? __ldcg(L + at) : (i == j ? T(1) : T(0));
    }
    if (tid < SBK) Rs[tid] = tid < rows ? T(1) / __ldcg(L + (int64_t)(r0 + tid) * a.lda + r0 + tid) : T(1);
    // FP32: the solved block next to this one (r - 1 forward, r + 1 backward) is the last to
    // arrive; its contribution is applied after the diagonal product as W y with W = D^-1 G
    // (D^-T G backward), G(j, k) = L(r0 + j, mN0 + k) forward, L(mN0 + k, r0 + j) backward,
    // so the chain of block rows holds one SBK x SBK product per link instead of the newest
    // block's partial products, the sum over the warps and the diagonal product
    const int nsteps_all = REV ? a.nrb - 1 - r : r;
    const bool newest = INV && nsteps_all > 0;
    const int mN = REV ? r + 1 : r - 1;
    const int mN0 = mN * SBK, mrows = newest ? min(SBK, a.n - mN0) : 0;
    if constexpr (INV) {
      if (newest) {
        for (int e = tid; e < SBK * SBK; e += SNT) {
          const int j = TRANS ? e / SBK : e % SBK, k = TRANS ? e % SBK : e / SBK;
          const int64_t at = TRANS ? (int64_t)(r0 + j) * a.lda + mN0 + k : (int64_t)(mN0 + k) * a.lda + r0 + j;
          Gs[j * DLD + k] = (j < rows && k < mrows) ? __ldcg(L + at) : T(0);
        }
      }
    }
    if constexpr (INV) {
      // D^-1 by columns: thread j of the first SBK threads solves D y = e_j (right-looking;
      // y stays zero above row j) while the other warps start accumulating. It is stored as
      // the matrix the product below reads k-major, Mi[k * MLD + i]: D^-1(i, k) forward,
      // D^-1(k, i) = D^-T(i, k) backward. Identity padding gives an identity inverse.
      __syncthreads();
      if (tid < SBK) {
        const int j = tid;
        T *col = TRANS ? Mi + j : Mi + j * MLD;  // entry i of column j at col[i * cs]
        const int cs = TRANS ? MLD : 1;
        for (int i = 0; i < SBK; ++i) col[i * cs] = i == j ? T(1) : T(0);
        for (int k = j; k < SBK; ++k) {
          const T yk = squot(col[k * cs], Ld[k * DLD + k], Rs[k]);
          col[k * cs] = yk;
#pragma unroll 4
          for (int i = k + 1; i < SBK; ++i) col[i * cs] = fma(-Ld[i * DLD + k], yk, col[i * cs]);
        }
        if (newest) {
          // the same threads, once the whole inverse is in place: row i = tid of W, stored
          // k-major like Mi, W(i, k) = sum_j Dop(i, j) G(j, k) with Dop(i, j) = Mi[j MLD + i]
          asm volatile("bar.sync 1, %0;" ::"r"(SBK));
          const int i = tid;
          T mrow[SBK];
#pragma unroll
          for (int jj = 0; jj < SBK; ++jj) mrow[jj] = Mi[jj * MLD + i];
          for (int k = 0; k < SBK; ++k) {
            T w = T(0);
#pragma unroll
            for (int jj = 0; jj < SBK; ++jj) w = fma(mrow[jj], Gs[jj * DLD + k], w);
            Wm[k * MLD + i] = w;
          }
        }
      }
    }
    if constexpr (QS) {
      // many right-hand sides (FP64): warp w owns the columns QC w .. QC w + QC - 1 of the group
      // over every solved block, in solve order, so the newest block's work is spread over all
      // eight warps instead of falling to one, and each warp's sums are final (no reduction)
      constexpr int QC = NC / SNW;
      const int qw = warp * QC;
      T bq[QC], accq[QC];
#pragma unroll
      for (int u = 0; u < QC; ++u) {
        bq[u] = (lane < rows && qw + u < cols) ? __ldcg(B + (int64_t)(c0 + qw + u) * a.ldb + r0 + lane) : T(0);
        accq[u] = T(0);
      }
      const int nsteps = REV ? a.nrb - 1 - r : r;
      int wab = 0;
      unsigned ready = 0u;  // bit j <-> step mbase + j
      int mbase = 0;
      for (int step = 0; step < nsteps; ++step) {
        const int m = REV ? a.nrb - 1 - step : step;
        const int k0 = m * SB, krows = min(SB, a.n - k0);
        // L block, issued before any wait: forward lane = row of the item, lr[k] = L(r0 +
        // lane, k0 + k); backward lane = row k0 + lane, lb[i] = L(k0 + lane, r0 + i)
        T lr[TRANS ? 1 : SB];
        T lb[TRANS ? SB : 1];
        if (!TRANS) {
#pragma unroll
          for (int k = 0; k < SB; ++k)
            lr[k] = (lane < rows && k < krows) ? __ldcg(L + (int64_t)(k0 + k) * a.lda + r0 + lane) : T(0);
        } else {
#pragma unroll
          for (int i = 0; i < SB; ++i)
            lb[i] = (lane < krows && i < rows) ? __ldcg(L + (int64_t)(r0 + i) * a.lda + k0 + lane) : T(0);
        }
        const int jb = step - mbase;
        if (jb >= 32 || !((ready >> jb) & 1u)) {
          const int sl = step + lane;
          int f = 1;
          if (sl < nsteps) {
            const int ml = REV ? a.nrb - 1 - sl : sl;
            f = ld_volatile(&a.flags[(int64_t)ml * a.ngroups + g]) != 0;
          }
          ready = __ballot_sync(0xffffffffu, f);
          mbase = step;
          if (!(ready & 1u)) {
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
            ready = 1u;
          }
          __threadfence();
          __syncwarp();
        }
        // this warp's columns of the solved block (lane k stages row k0 + k)
#pragma unroll
        for (int u = 0; u < QC; ++u)
          yw[lane * YLD + u] = (lane < krows && qw + u < cols) ? __ldcg(B + (int64_t)(c0 + qw + u) * a.ldb + k0 + lane)
                                                              : T(0);
        if (TRANS) {
#pragma unroll
          for (int i = 0; i < SB; ++i) lt[lane * DLD + i] = lb[i];
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < SB; ++k) {
          const T l = TRANS ? lt[k * DLD + lane] : lr[TRANS ? 0 : k];
#pragma unroll
          for (int u = 0; u < QC; ++u) accq[u] = fma(l, yw[k * YLD + u], accq[u]);
        }
        __syncwarp();
      }
      if (wab && lane == 0) s_abort = 1;
#pragma unroll
      for (int u = 0; u < QC; ++u)
        if (qw + u < NC) Ys[lane * YLD + qw + u] = bq[u] - accq[u];
      __syncthreads();
      if (s_abort) break;
    } else {
      // this thread's entries of B_r for the final sum, loaded now (off the chain)
      constexpr int BPT = (SBK * NC + SNT - 1) / SNT;
      T bv[BPT];
  #pragma unroll
      for (int u = 0; u < BPT; ++u) {
        const int e = tid + u * SNT, i = e % SBK, q = e / SBK;
        bv[u] = (e < SBK * NC && i < rows && q < cols) ? __ldcg(B + (int64_t)(c0 + q) * a.ldb + r0 + i) : T(0);
      }
      // warp-parallel accumulation over the solved blocks
      T acc[RPL][NC];
  #pragma unroll
      for (int rr = 0; rr < RPL; ++rr)
  #pragma unroll
        for (int q = 0; q < NC; ++q) acc[rr][q] = T(0);
      // (FP32: all solved blocks but the newest, which follows the diagonal product)
      const int nsteps = newest ? nsteps_all - 1 : nsteps_all;
      // the solved blocks are consumed in 32-row chunks, one chunk per warp step: chunk kc of
      // block m is step m * RPL + kc, so the chunks of the newest block go to different warps.
      // FP64 forward-read sweeps with one or two columns cut every chunk into QTR quarters of
      // its 32 k values, dealt to consecutive warps (different SM sub-partitions): a warp-wide
      // FP64 instruction costs its sub-partition ~64 cycles, so the newest block's 32 dependent
      // FMAs on one warp were ~2000 cycles of every link of the chain, and are ~500 split
      constexpr int QTR = (!INV && !TRANS && NC <= 2 && SBK == 32) ? 4 : 1;
      constexpr int KQ = SB / QTR;
      const int nchunks = nsteps * RPL;
      const int nunits = nchunks * QTR;
      int wab = 0;
      // readiness of the warp's next 32 units: bit j <-> unit mbase + SNW j, one flag load per
      // lane and a ballot, so blocks solved long ago cost no polling round trip
      unsigned ready = 0u;
      int mbase = warp;
      for (int unit = warp; unit < nunits; unit += SNW) {
        const int step = unit / QTR, kq0 = (unit % QTR) * KQ;
        const int mi = step / RPL, kc = step % RPL;
        const int m = REV ? a.nrb - 1 - mi : mi;
        const int k0 = m * SBK + SB * kc, krows = min(SB, a.n - k0);  // this 32-row chunk of block m
        // L chunk, issued before any wait (it does not depend on other items). Forward: lane =
        // row of the item, lr[rr][k] = L(r0 + lane + 32 rr, k0 + k). Backward: lane = row k0 +
        // lane, lb[i] = L(k0 + lane, r0 + i), staged transposed below.
        T lr[TRANS ? 1 : RPL][KQ];
        T lb[TRANS ? SBK : 1];
        if (!TRANS) {
  #pragma unroll
          for (int rr = 0; rr < RPL; ++rr)
  #pragma unroll
            for (int kk = 0; kk < KQ; ++kk)
              lr[rr][kk] = (lane + SB * rr < rows && kq0 + kk < krows)
                               ? __ldcg(L + (int64_t)(k0 + kq0 + kk) * a.lda + r0 + lane + SB * rr) : T(0);
        } else {
  #pragma unroll
          for (int i = 0; i < SBK; ++i)
            lb[i] = (lane < krows && i < rows) ? __ldcg(L + (int64_t)(r0 + i) * a.lda + k0 + lane) : T(0);
        }
        int jb = (unit - mbase) / SNW;
        if (jb >= 32 || !((ready >> jb) & 1u)) {
          const int sl = unit + SNW * lane;
          int f = 1;
          if (sl < nunits) {
            const int ml = REV ? a.nrb - 1 - sl / QTR / RPL : sl / QTR / RPL;
            f = ld_volatile(&a.flags[(int64_t)ml * a.ngroups + g]) != 0;
          }
          ready = __ballot_sync(0xffffffffu, f);
          mbase = unit;
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
        // Y chunk (lane k stages row k0 + k), loaded once the block is known to be solved
        T yv[NC];
  #pragma unroll
        for (int q = 0; q < NC; ++q)
          yv[q] = (lane < krows && q < cols) ? __ldcg(B + (int64_t)(c0 + q) * a.ldb + k0 + lane) : T(0);
  #pragma unroll
        for (int q = 0; q < NC; ++q) yw[lane * YLD + q] = yv[q];
        if (TRANS) {
  #pragma unroll
          for (int i = 0; i < SBK; ++i) lt[lane * DLD + i] = lb[i];
        }
        __syncwarp();
  #pragma unroll
        for (int kk = 0; kk < KQ; ++kk) {
          const int k = kq0 + kk;
          T l[RPL];
  #pragma unroll
          for (int rr = 0; rr < RPL; ++rr) l[rr] = TRANS ? lt[k * DLD + lane + SB * rr] : lr[TRANS ? 0 : rr][kk];
  #pragma unroll
          for (int q = 0; q < NC; q += V) {
            T y[V];
            vload<T, V>(yw + k * YLD + q, y);
  #pragma unroll
            for (int rr = 0; rr < RPL; ++rr)
  #pragma unroll
              for (int u = 0; u < V; ++u) acc[rr][q + u] = fma(l[rr], y[u], acc[rr][q + u]);
          }
        }
        __syncwarp();
      }
      if (wab && lane == 0) s_abort = 1;
      // the eight partial sums, column-major per warp (consecutive lanes, consecutive words),
      // then B_r minus their sum into Ys
  #pragma unroll
      for (int rr = 0; rr < RPL; ++rr)
  #pragma unroll
        for (int q = 0; q < NC; ++q) yw[q * SBK + lane + SB * rr] = acc[rr][q];
      __syncthreads();
      if (s_abort) break;
  #pragma unroll
      for (int u = 0; u < BPT; ++u) {
        const int e = tid + u * SNT, i = e % SBK, q = e / SBK;
        if (e < SBK * NC) {
          T sum = T(0);
  #pragma unroll
          for (int w = 0; w < SNW; ++w) sum += Yw[(size_t)w * SBK * YLD + q * SBK + i];
          Ys[i * YLD + q] = bv[u] - sum;
        }
      }
      __syncthreads();
    }
    T *Xo = Ys;  // the solved block, row-major with stride YLD
    if constexpr (INV) {
      // forward x = D^-1 (b - sum), backward x = D^-T (b - sum): independent SBK-term
      // products (D^-1 is zero above the diagonal)
      Xo = Yw;  // free once the partial sums are added
      // thread: column q, RPT consecutive rows; per k one broadcast of Y(k, q) and RPT/4
      // vector loads of Mi's column k (same k order as a plain dot product)
      constexpr int RPT = SBK * NC / SNT >= 4 ? SBK * NC / SNT : 4;
      static_assert(SBK % RPT == 0 && RPT % 4 == 0, "rows per thread");
      if (tid < SBK * NC / RPT) {
        const int q = tid % NC, i0 = (tid / NC) * RPT;
        T t[RPT];
#pragma unroll
        for (int u = 0; u < RPT; ++u) t[u] = T(0);
#pragma unroll 8
        for (int k = 0; k < SBK; ++k) {
          const T y = Ys[k * YLD + q];
#pragma unroll
          for (int u = 0; u < RPT; u += 4) {
            T m[4];
            vload<T, 4>(Mi + k * MLD + i0 + u, m);
#pragma unroll
            for (int v = 0; v < 4; ++v) t[u + v] = fma(m[v], y, t[u + v]);
          }
        }
#pragma unroll
        for (int u = 0; u < RPT; ++u) Xo[(i0 + u) * YLD + q] = t[u];
      }
      if (newest) {
        // wait for the newest block (one thread, bounded), stage it in Ys (free now) and
        // subtract W y from the diagonal product
        __syncthreads();
        if (tid == 0) {
          const uint64_t t0 = globaltimer_ns();
          int64_t spins = 0;
          while (ld_volatile(&a.flags[(int64_t)mN * a.ngroups + g]) == 0) {
            if (ld_volatile(&a.ctrl->abort)) { s_abort = 1; break; }
            if (globaltimer_ns() - t0 > (uint64_t)a.timeout_ns || ++spins > (a.timeout_ns >> 7) + 100000) {
              atomicCAS(&a.ctrl->info, 0, CHOL_INFO_TIMEOUT);
              atomicExch(&a.ctrl->abort, 1);
              s_abort = 1;
              break;
            }
            __nanosleep(32);
          }
          // the flag is ordered before the block's data
          __threadfence();
        }
        __syncthreads();
        if (s_abort) break;
        for (int e = tid; e < SBK * NC; e += SNT) {
          const int k = e % SBK, q = e / SBK;
          Ys[k * YLD + q] = (k < mrows && q < cols) ? __ldcg(B + (int64_t)(c0 + q) * a.ldb + mN0 + k) : T(0);
        }
        __syncthreads();
        if (tid < SBK * NC / RPT) {
          const int q = tid % NC, i0 = (tid / NC) * RPT;
          T t[RPT];
#pragma unroll
          for (int u = 0; u < RPT; ++u) t[u] = Xo[(i0 + u) * YLD + q];
#pragma unroll 8
          for (int k = 0; k < SBK; ++k) {
            const T y = Ys[k * YLD + q];
#pragma unroll
            for (int u = 0; u < RPT; u += 4) {
              T m[4];
              vload<T, 4>(Wm + k * MLD + i0 + u, m);
#pragma unroll
              for (int v = 0; v < 4; ++v) t[u + v] = fma(-m[v], y, t[u + v]);
            }
          }
#pragma unroll
          for (int u = 0; u < RPT; ++u) Xo[(i0 + u) * YLD + q] = t[u];
        }
      }
    } else if (cols <= SNW / 2) {
      // diagonal block, at most 4 right-hand sides: one warp per right-hand side (one per SM
      // sub-partition), lane = row; x_k on lane k, then one warp-wide FMA for the rows below
      const int c = warp;
      if (c < cols) {
        T x = Ys[lane * YLD + c];
        const T rinv = Rs[lane];
        if (!REV) {
#pragma unroll
          for (int k = 0; k < SBK; ++k) {
            if (lane == k) x = squot(x, Ld[k * DLD + k], rinv);
            const T xk = __shfl_sync(0xffffffffu, x, k);
            if (lane > k) x = fma(-Ld[lane * DLD + k], xk, x);
          }
        } else {
#pragma unroll
          for (int k = SBK - 1; k >= 0; --k) {
            if (lane == k) x = squot(x, Ld[k * DLD + k], rinv);
            const T xk = __shfl_sync(0xffffffffu, x, k);
            if (lane < k) x = fma(-Ld[k * DLD + lane], xk, x);
          }
        }
        Ys[lane * YLD + c] = x;
      }
    } else {
      // diagonal block, more than 4 right-hand sides: thread (warp w, lane c) holds column c
      // of rows w, w + 8, w + 16, w + 24. Step k: warp k % 8 forms x_k for every column at
      // once and passes it on through shared memory (two buffers by step parity, so one
      // barrier per step), then each warp updates its rows below k (above k backward). An
      // FP64 instruction costs its SM sub-partition the same time with one active lane as
      // with 32, so this spends 32-wide instructions on all four sub-partitions where one
      // thread per column would spend them on one. Every x_i sees the operations of the
      // right-looking substitution in the same order (its updates by increasing k, then its
      // quotient; decreasing k backward).
      const int c = lane;
      T y[SBK / SNW];
#pragma unroll
      for (int j = 0; j < SBK / SNW; ++j) y[j] = c < cols ? Ys[(warp + SNW * j) * YLD + c] : T(0);
#pragma unroll
      for (int kk = 0; kk < SBK; ++kk) {
        const int k = REV ? SBK - 1 - kk : kk;
        if (warp == k % SNW) {
          const T x = squot(y[k / SNW], Ld[k * DLD + k], Rs[k]);
          y[k / SNW] = x;
          s_xk[kk & 1][c] = x;
        }
        __syncthreads();
        const T xk = s_xk[kk & 1][c];
#pragma unroll
        for (int j = 0; j < SBK / SNW; ++j) {
          const int i = warp + SNW * j;
          if (REV ? i < k : i > k) y[j] = fma(-(REV ? Ld[k * DLD + i] : Ld[i * DLD + k]), xk, y[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < SBK / SNW; ++j)
        if (c < cols) Ys[(warp + SNW * j) * YLD + c] = y[j];
    }
    __syncthreads();
    // write the solved block column by column (one warp per column: consecutive rows)
    for (int c = warp; c < cols; c += SNW)
#pragma unroll
      for (int rr = 0; rr < RPL; ++rr)
        if (lane + SB * rr < rows) __stcg(B + (int64_t)(c0 + c) * a.ldb + r0 + lane + SB * rr, Xo[(lane + SB * rr) * YLD + c]);
    __threadfence();
    __syncthreads();
    if (tid == 0) *(volatile int *)&a.flags[(int64_t)r * a.ngroups + g] = 1;
  }
}

__global__ void solve_info_kernel(const SolveCtrl *c0, const SolveCtrl *c1, int *dInfo) {
  if (threadIdx.x == 0) *dInfo = c0->info ? c0->info : (c1 ? c1->info : 0);
}
__global__ void solve_info_merge_kernel(const SolveCtrl *c0, int *dInfo) {
  if (threadIdx.x == 0 && *dInfo == 0) *dInfo = c0->info;
}

// workspace: two control blocks (one per sweep) and two flag arrays
static size_t flags_bytes(int n, int nrhs) {
  const int64_t nrb = (n + SB - 1) / SB;
  const int64_t ng = (nrhs + SG - 1) / SG;
  return align_up((size_t)std::max<int64_t>(1, nrb * ng) * 4, 256);
}
static size_t solve_ws(int n, int nrhs) { return 512 + 2 * flags_bytes(n, nrhs); }

size_t solve_workspace_bytes(int n, int nrhs) { return solve_ws(n, nrhs); }

// rows per item: 64 in FP32 (half the links of the chain), 32 in FP64 (exact substitution)
template <class T>
constexpr int item_rows() { return sizeof(T) == 4 ? 64 : 32; }

// the widest instances fit one block's shared memory (227 KB of dynamic shared memory per
// block, less the kernel's few static bytes)
static_assert(SolveSmem<float, SG, 64>::BYTES <= 227 * 1024 - 512, "FP32 sweep shared memory");
static_assert(SolveSmem<double, SG, 32>::BYTES <= 227 * 1024 - 512, "FP64 sweep shared memory");

template <class T, int NC, int MODE>
static cudaError_t launch_solve_mode(const SolveArgs &a, int grid, cudaStream_t s) {
  // one block per SM: the dynamic shared memory request (more than half an SM's) makes a
  // second block impossible
  constexpr int SBK = item_rows<T>();
  constexpr size_t bytes = SolveSmem<T, NC, SBK>::BYTES;
  const cudaError_t e = set_smem_attr((const void *)solve_kernel<T, NC, SBK, MODE>, (int)bytes);
  if (e != cudaSuccess) return e;
  solve_kernel<T, NC, SBK, MODE><<<grid, SNT, bytes, s>>>(a);
  return cudaGetLastError();
}

template <class T, int NC>
static cudaError_t launch_solve(const SolveArgs &a, int grid, cudaStream_t s) {
  if (a.trans == 0) return launch_solve_mode<T, NC, 0>(a, grid, s);
  if (a.trans == 1) return launch_solve_mode<T, NC, 1>(a, grid, s);
  if constexpr (sizeof(T) == 8) return launch_solve_mode<T, NC, 2>(a, grid, s);
  return cudaErrorInvalidValue;
}

template <class T>
static chol_status launch_sweep(int trans, int slot, int n, int nrhs, const T *dL, int lda, T *dB, int ldb,
                                void *dWork, const int *skip, cudaStream_t s, const int *prev_abort = nullptr) {
  SolveArgs a;
  a.L = dL; a.lda = lda; a.B = dB; a.ldb = ldb; a.n = n; a.nrhs = nrhs;
  a.nrb = (n + item_rows<T>() - 1) / item_rows<T>();  // flags are sized for 32-row blocks: enough
  a.ngroups = (nrhs + SG - 1) / SG;
  a.nitems = (int64_t)a.nrb * a.ngroups;
  a.trans = trans;
  a.timeout_ns = 10000000000ll;
  a.skip = skip;
  unsigned char *ws = static_cast<unsigned char *>(dWork);
  a.ctrl = reinterpret_cast<SolveCtrl *>(ws + 256 * slot);
  a.prev_abort = prev_abort ? prev_abort : slot == 1 ? &reinterpret_cast<SolveCtrl *>(ws)->abort : nullptr;
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

// U X = B in place (one backward sweep, U read from the upper triangle of the tiles, as the
// tile LU leaves it). The sweep's items are skipped once *prev_abort is set (nullable).
chol_status solve_upper_f64(int n, int nrhs, const double *dU, int lda, double *dB, int ldb, void *dWork,
                            const int *prev_abort, cudaStream_t s) {
  if (n == 0 || nrhs == 0) return CHOL_OK;
  return launch_sweep<double>(2, 0, n, nrhs, dU, lda, dB, ldb, dWork, nullptr, s, prev_abort);
}

// *dInfo = the upper sweep's info (0 or CHOL_INFO_TIMEOUT), unless it is already nonzero.
chol_status solve_upper_info(void *dWork, int *dInfo, cudaStream_t s) {
  unsigned char *ws = static_cast<unsigned char *>(dWork);
  solve_info_merge_kernel<<<1, 32, 0, s>>>(reinterpret_cast<const SolveCtrl *>(ws), dInfo);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

}  // namespace chol

using namespace chol;

extern "C" size_t chol_solve_workspace_size(int n, int nrhs) {
  if (n < 0 || nrhs < 0) return 0;
  return solve_ws(n, nrhs);
}

extern "C" chol_status chol_solve_f32(int n, int nrhs, const float *dL, int lda, float *dB, int ldb, void *dWork,
                                      size_t work_bytes, int *dInfo, void *stream) {
  const chol_status st = check_args(n, nrhs, dL, lda, dB, ldb, dWork, work_bytes);
  if (st != CHOL_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0 || nrhs == 0) {
    if (dInfo) CHOL_CUDA_TRY(cudaMemsetAsync(dInfo, 0, sizeof(int), s));
    return CHOL_OK;
  }
  const chol_status r = solve_f32(n, nrhs, dL, lda, dB, ldb, dWork, nullptr, s);
  if (r != CHOL_OK) return r;
  return write_info(dWork, 2, dInfo, s);
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
  // the argument rules of chol_solve first, then the size limit of the fixed array
  if (n < 0 || nrhs < 0) return CHOL_ERR_INVALID_ARG;
  if (lda < std::max(1, n) || ldb < std::max(1, n)) return CHOL_ERR_INVALID_ARG;
  if (n > 0 && nrhs > 0 && (!dL || !dB)) return CHOL_ERR_INVALID_ARG;
  if (n == 0 || nrhs == 0) {
    if (dInfo) CHOL_CUDA_TRY(cudaMemsetAsync(dInfo, 0, sizeof(int), (cudaStream_t)stream));
    return CHOL_OK;
  }
  if (solve_ws(n, nrhs) > SOLVE_NOALLOC_BYTES) return CHOL_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CHOL_ERR_CUDA;
  cudaError_t err = cudaSuccess;
  void *scratch = noalloc_scratch(dev, &err);
  if (!scratch) return CHOL_ERR_CUDA;
  // the sweeps clear the control blocks and flags they use before every launch
  return chol_solve(n, nrhs, dL, lda, dB, ldb, scratch, SOLVE_NOALLOC_BYTES, dInfo, stream);
}
