// Solve A X = B with the factors of the tile LU with incremental pivoting (chol_lu_factor).
//
// The factorization recorded, tile column by tile column, the transformation of GETRF(k)
// and then those of TSTRF(i, k), i > k, each a sequence of inner blocks (interchanges, unit
// lower L11, multipliers L21). Applying them to B in the same order gives U X = M B with U
// the upper triangle of the tiles (diagonal tiles' upper parts and the tiles right of the
// diagonal); back substitution with U finishes the solve.
//
// The transformations form a graph of their own: node (k, k) applies GETRF(k) to the tile
// row Y_k, node (i, k), i > k, applies TSTRF(i, k) to [Y_k; Y_i]. Node (i, k) needs node
// (i - 1, k) (the previous TSTRF of column k, or GETRF(k), left Y_k as it must be) and node
// (i, k - 1) (the last transformation that touched Y_i); (k, k) needs (k, k - 1). Its longest
// path has about 2T nodes against T(T + 1)/2 in all, so lu_fwd_kernel runs it as a wavefront:
// thread blocks (one per SM) claim (node, group of right-hand sides) items from an atomic
// counter with the nodes ordered by anti-diagonal s = i + k (then by k), wait on the ready
// flags of the two predecessors (both on diagonal s - 1, so claimed earlier; bounded waits),
// apply the node's inner blocks to the staged rows and publish a flag. Claiming along the
// diagonals keeps the in-flight items on the front of the wavefront; in column order the
// blocks would hold a few tile columns at a time and every later column would start late. Everything that does not depend on Y -- the pivots, the L11
// blocks, the first inner block's L21 rows -- is loaded before the wait. The back
// substitution is the backward sweep of the Cholesky solve with U (solve_upper_f64).
#include <algorithm>
#include <cmath>
#include "common.cuh"
#include "internal.cuh"
#include "tiles_lu.cuh"

namespace chol {

constexpr int LG = 8;                       // right-hand sides per item
constexpr int LNB = LU_NB_MAX / LU_IB;      // inner blocks per tile, at most
constexpr int L11LD = LU_IB + 1;
constexpr int LPOS = LU_IB + LU_NB_MAX;     // positions an inner block's interchanges address
constexpr int LMOV = 2 * LU_IB;              // moves of one inner block's interchanges, at most
constexpr int LU_FWD_SMEM_BYTES =
    (2 * LU_NB_MAX * LG + LNB * LU_IB * L11LD) * 8 + LU_NB_MAX * 4 + LNB * LPOS * 2 + LNB * LMOV * 4 + LNB * 4;
constexpr int LU_FWD_EXCL_SMEM = 120 * 1024;  // request at least this much: one block per SM
constexpr int LU_FWD_SMEM_REQ = LU_FWD_SMEM_BYTES > LU_FWD_EXCL_SMEM ? LU_FWD_SMEM_BYTES : LU_FWD_EXCL_SMEM;

struct LuFwdCtrl {
  unsigned int next_item;
  int abort;
  int info;
  int pad[61];
};

struct LuFwdArgs {
  int n, nb, T, nrhs, ngroups;
  int64_t nnodes, nitems;
  const double *F;
  int64_t lda;
  const int *piv;
  const double *lw;
  double *B;
  int64_t ldb;
  LuFwdCtrl *ctrl;
  int *flags;  // per (node, group): 1 once the node's transformation of that group is stored
  int64_t timeout_ns;
};

// Nodes (i, k), 0 <= k <= i < T, ordered by s = i + k, then by k. lu_diag_offset(T, s) is the
// number of nodes with i + k < s: sum over s' < s of (floor(s'/2) + 1 - max(0, s' - T + 1)).
__host__ __device__ __forceinline__ int64_t lu_diag_offset(int T, int s) {
  const int64_t h = s / 2;
  const int64_t a = (int64_t)s + (s % 2 == 0 ? h * (h - 1) : h * h);
  const int64_t e = s > T ? (int64_t)(s - T) * (s - T + 1) / 2 : 0;
  return a - e;
}
__device__ __forceinline__ int64_t lu_node_index(int T, int i, int k) {
  const int s = i + k;
  return lu_diag_offset(T, s) + (k - max(0, s - T + 1));
}
__device__ __forceinline__ void lu_node_decode(int T, int64_t node, int &i, int &k) {
  // largest s with lu_diag_offset(T, s) <= node (binary search over 0 .. 2T - 2)
  int lo = 0, hi = 2 * T - 2;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (lu_diag_offset(T, mid) <= node) lo = mid; else hi = mid - 1;
  }
  const int s = lo;
  k = max(0, s - T + 1) + (int)(node - lu_diag_offset(T, s));
  i = s - k;
}

// Wait (thread 0) until flag f is set; returns false if the run aborted or the wait expired.
__device__ bool lu_wait_flag(const LuFwdArgs &a, const int *f) {
  const uint64_t t0 = globaltimer_ns();
  int64_t spins = 0;
  unsigned slp = 32;
  while (ld_volatile(f) == 0) {
    if (ld_volatile(&a.ctrl->abort)) return false;
    if (globaltimer_ns() - t0 > (uint64_t)a.timeout_ns || ++spins > (a.timeout_ns >> 7) + 100000) {
      atomicCAS(&a.ctrl->info, 0, CHOL_INFO_TIMEOUT);
      atomicExch(&a.ctrl->abort, 1);
      return false;
    }
    __nanosleep(slp);
    slp = slp < 256 ? slp * 2 : 256;
  }
  return true;
}

__global__ void __launch_bounds__(NT, 1) lu_fwd_kernel(const __grid_constant__ LuFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *Yk = reinterpret_cast<double *>(smem_raw);    // [LG][LU_NB_MAX] column-major
  double *Yi = Yk + LU_NB_MAX * LG;
  double *L11 = Yi + LU_NB_MAX * LG;                     // [LNB][LU_IB][L11LD] row-major
  int *spiv = reinterpret_cast<int *>(L11 + LNB * LU_IB * L11LD);
  short *pmap = reinterpret_cast<short *>(spiv + LU_NB_MAX);    // [LNB][LPOS]
  short2 *moves = reinterpret_cast<short2 *>(pmap + LNB * LPOS); // [LNB][LMOV] (dst, src)
  int *nmoves = reinterpret_cast<int *>(moves + LNB * LMOV);     // [LNB]
  __shared__ long long s_item;
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = a.nb, T = a.T;
  const int64_t lda = a.lda, ldb = a.ldb;
  auto tile = [&](int r, int c) { return a.F + (int64_t)c * nb * lda + (int64_t)r * nb; };
  auto dim = [&](int t) { return min(nb, a.n - t * nb); };
  while (true) {
    if (tid == 0) s_item = ld_volatile(&a.ctrl->abort) ? -1 : (long long)atomicAdd(&a.ctrl->next_item, 1u);
    __syncthreads();
    const long long item = s_item;
    if (item < 0 || item >= a.nitems) break;
    const int64_t node = item / a.ngroups;
    const int g = (int)(item - node * a.ngroups);
    int i, k;
    lu_node_decode(T, node, i, k);
    const bool getrf = i == k;
    const int nk = dim(k), mi = getrf ? 0 : dim(i);
    const int c0g = g * LG, gc = min(LG, a.nrhs - c0g);
    const int nblk = (nk + LU_IB - 1) / LU_IB;
    const double *Akk = tile(k, k);
    const double *Aik = getrf ? nullptr : tile(i, k);
    const double *lwp = getrf ? nullptr : a.lw + ((int64_t)k * T + i) * LU_IB * nb;
    // --- independent of Y: pivots, L11 of every inner block, L21 rows of the first block
    const int *pv = a.piv + ((int64_t)k * T + i) * nb;
    for (int e = tid; e < nk; e += NT) spiv[e] = __ldcg(pv + e);
    for (int e = tid; e < nblk * LU_IB * LU_IB; e += NT) {
      const int b = e / (LU_IB * LU_IB), q = e - b * LU_IB * LU_IB;
      const int r = q & (LU_IB - 1), c = q >> 5;
      const int w = min(LU_IB, nk - b * LU_IB);
      double v = 0.0;
      if (r < w && c < r)
        v = getrf ? __ldcg(Akk + (int64_t)(b * LU_IB + c) * lda + b * LU_IB + r)
                  : __ldcg(lwp + (int64_t)(b * LU_IB + c) * LU_IB + r);
      L11[(b * LU_IB + r) * L11LD + c] = v;
    }
    // the interchanges of each inner block as one permutation of the positions they touch
    // (position p < w: row p of X1, else row p - w of X2): the sequence of swaps is replayed on
    // position labels, one thread per block, and the moved positions are listed as (dst, src)
    // pairs -- applied after the wait in one parallel gather instead of w dependent swaps
    for (int e = tid; e < nblk * LPOS; e += NT) pmap[e] = (short)(e % LPOS);
    __syncthreads();
    if (tid < nblk) {
      const int b = tid, c0 = b * LU_IB, w = min(LU_IB, nk - c0);
      const int m2 = getrf ? nk - c0 - w : mi;
      short *mp = pmap + b * LPOS;
      short2 *mv = moves + b * LMOV;
      int cnt = 0;
      for (int j = 0; j < w; ++j) {
        const int q = spiv[c0 + j];
        if (q == j || q < 0 || q >= w + m2) continue;
        const short t = mp[j];
        mp[j] = mp[q];
        mp[q] = t;
        if (q >= w) mv[w + cnt++] = make_short2((short)q, 0);  // X2 positions touched (may repeat)
      }
      // X1 positions first (all w of them), then the touched X2 positions
      for (int j = 0; j < w; ++j) mv[j] = make_short2((short)j, mp[j]);
      for (int u = 0; u < cnt; ++u) mv[w + u].y = mp[mv[w + u].x];
      nmoves[b] = w + cnt;
    }
    // row of X2 this thread eliminates in block b: GETRF rows c1 + tid of the diagonal tile,
    // TSTRF row tid of A_ik; its L21 row (w values) is held in registers, the next block's
    // loaded while the current one is applied
    double lcur[LU_IB], lnext[LU_IB];
    auto load_l21 = [&](int b, double (&l)[LU_IB]) {
      const int c0 = b * LU_IB, w = min(LU_IB, nk - c0), c1 = c0 + w;
      const int m2 = getrf ? nk - c1 : mi;
      const double *base = getrf ? Akk + (int64_t)c0 * lda + c1 : Aik + (int64_t)c0 * lda;
#pragma unroll
      for (int j = 0; j < LU_IB; ++j) l[j] = (tid < m2 && j < w) ? __ldcg(base + (int64_t)j * lda + tid) : 0.0;
    };
    load_l21(0, lcur);
    // --- wait for the predecessors: (i - 1, k) and (i, k - 1)
    if (tid == 0) {
      bool ok = true;
      if (!getrf) ok = lu_wait_flag(a, &a.flags[lu_node_index(T, i - 1, k) * a.ngroups + g]);
      if (ok && k > 0) ok = lu_wait_flag(a, &a.flags[lu_node_index(T, i, k - 1) * a.ngroups + g]);
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    __threadfence();
    // --- stage the rows (column-major, ld LU_NB_MAX)
    for (int e = tid; e < nk * gc; e += NT) {
      const int c = e / nk, r = e - c * nk;
      Yk[c * LU_NB_MAX + r] = __ldcg(a.B + (int64_t)(c0g + c) * ldb + (int64_t)k * nb + r);
    }
    for (int e = tid; e < mi * gc; e += NT) {
      const int c = e / mi, r = e - c * mi;
      Yi[c * LU_NB_MAX + r] = __ldcg(a.B + (int64_t)(c0g + c) * ldb + (int64_t)i * nb + r);
    }
    // rows of Y_k past the tile, up to the last inner block's end, are read (times a zero
    // multiplier) by the eliminations below: they must hold finite values
    {
      const int pad = nblk * LU_IB - nk;
      for (int e = tid; e < pad * gc; e += NT) {
        const int c = e / pad, r = e - c * pad;
        Yk[c * LU_NB_MAX + nk + r] = 0.0;
      }
    }
    __syncthreads();
    for (int b = 0; b < nblk; ++b) {
      const int c0 = b * LU_IB, w = min(LU_IB, nk - c0), c1 = c0 + w;
      const int m2 = getrf ? nk - c1 : mi;
      double *X1 = Yk + c0;                      // w rows
      double *X2 = getrf ? Yk + c1 : Yi;         // m2 rows
      if (b + 1 < nblk) load_l21(b + 1, lnext);
      // the interchanges: gather every moved position's value, then store them (a repeated
      // X2 position is written twice with the same value)
      {
        const int nm = nmoves[b], tot = nm * gc;
        const short2 *mv = moves + b * LMOV;
        auto at = [&](int c, int pos) { return pos < w ? X1 + c * LU_NB_MAX + pos : X2 + c * LU_NB_MAX + (pos - w); };
        double v[(LMOV * LG + NT - 1) / NT];
#pragma unroll
        for (int u = 0; u < (LMOV * LG + NT - 1) / NT; ++u) {
          const int e = tid + u * NT;
          if (e < tot) v[u] = *at(e / nm, mv[e % nm].y);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < (LMOV * LG + NT - 1) / NT; ++u) {
          const int e = tid + u * NT;
          if (e < tot) *at(e / nm, mv[e % nm].x) = v[u];
        }
      }
      __syncthreads();
      // unit lower L11 solve, one warp per right-hand side (lane = row)
      const double *l11 = L11 + (size_t)b * LU_IB * L11LD;
      for (int c = warp; c < gc; c += NT / 32) {
        double y = lane < w ? X1[c * LU_NB_MAX + lane] : 0.0;
        for (int j = 0; j + 1 < w; ++j) {
          const double yj = __shfl_sync(0xffffffffu, y, j);
          if (lane > j) y = fma(-l11[lane * L11LD + j], yj, y);
        }
        if (lane < w) X1[c * LU_NB_MAX + lane] = y;
      }
      __syncthreads();
      // X2 -= L21 X1, one thread per row of X2, four partial sums per right-hand side
      if (tid < m2) {
        for (int c = 0; c < gc; ++c) {
          const double *x1 = X1 + c * LU_NB_MAX;
          double t[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
          for (int j = 0; j < LU_IB; ++j) t[j & 3] = fma(lcur[j], x1[j], t[j & 3]);
          X2[c * LU_NB_MAX + tid] -= (t[0] + t[1]) + (t[2] + t[3]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < LU_IB; ++j) lcur[j] = lnext[j];
    }
    // --- store and publish
    for (int e = tid; e < nk * gc; e += NT) {
      const int c = e / nk, r = e - c * nk;
      __stcg(a.B + (int64_t)(c0g + c) * ldb + (int64_t)k * nb + r, Yk[c * LU_NB_MAX + r]);
    }
    for (int e = tid; e < mi * gc; e += NT) {
      const int c = e / mi, r = e - c * mi;
      __stcg(a.B + (int64_t)(c0g + c) * ldb + (int64_t)i * nb + r, Yi[c * LU_NB_MAX + r]);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) *(volatile int *)&a.flags[node * a.ngroups + g] = 1;
  }
}

__global__ void lu_info_kernel(const LuFwdCtrl *c, int *dInfo) {
  if (threadIdx.x == 0) *dInfo = c->info;
}

struct LuSolveLayout {
  size_t ctrl, flags, sweep, total;
  int64_t nnodes;
  int ngroups;
};

static LuSolveLayout lu_solve_layout(int n, int nrhs, int nb) {
  LuSolveLayout L;
  const int T = n > 0 ? (n + nb - 1) / nb : 0;
  L.nnodes = (int64_t)T * (T + 1) / 2;
  L.ngroups = (nrhs + LG - 1) / LG;
  size_t o = 0;
  L.ctrl = o; o += 256;
  L.flags = o; o += align_up((size_t)std::max<int64_t>(1, L.nnodes * L.ngroups) * 4, 256);
  L.sweep = o; o += solve_workspace_bytes(n, nrhs);
  L.total = o;
  return L;
}

}  // namespace chol

using namespace chol;

extern "C" size_t chol_lu_solve_workspace_size(int n, int nrhs, const chol_opts *opts) {
  if (n < 0 || nrhs < 0) return 0;
  const int nb = lu_tile_size(n, opts);
  if (nb <= 0) return 0;
  return lu_solve_layout(n, nrhs, nb).total;
}

extern "C" chol_status chol_lu_solve(int n, int nrhs, const double *dF, int lda, const int *dPiv, const double *dLw,
                                     const chol_opts *opts, double *dB, int ldb, void *dWork, size_t work_bytes,
                                     int *dInfo, void *stream) {
  if (n < 0 || nrhs < 0) return CHOL_ERR_INVALID_ARG;
  const int nb = lu_tile_size(n, opts);
  if (nb <= 0) return CHOL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0 || nrhs == 0) {
    if (dInfo) CHOL_CUDA_TRY(cudaMemsetAsync(dInfo, 0, sizeof(int), s));
    return CHOL_OK;
  }
  if (lda < n || ldb < n || !dF || !dPiv || !dLw || !dB) return CHOL_ERR_INVALID_ARG;
  const LuSolveLayout L = lu_solve_layout(n, nrhs, nb);
  if (!dWork || work_bytes < L.total || ((uintptr_t)dWork & 255)) return CHOL_ERR_WORKSPACE;
  const DeviceInfo di = current_device_info();
  if (di.sms <= 0) return CHOL_ERR_CUDA;
  if (di.cc_major != 10 || di.cc_minor != 3) return CHOL_ERR_UNSUPPORTED;
  CHOL_CUDA_TRY(set_smem_attr((const void *)lu_fwd_kernel, LU_FWD_SMEM_REQ));
  unsigned char *ws = static_cast<unsigned char *>(dWork);
  LuFwdArgs a;
  a.n = n;
  a.nb = nb;
  a.T = (n + nb - 1) / nb;
  a.nrhs = nrhs;
  a.ngroups = L.ngroups;
  a.nnodes = L.nnodes;
  a.nitems = L.nnodes * L.ngroups;
  a.F = dF;
  a.lda = lda;
  a.piv = dPiv;
  a.lw = dLw;
  a.B = dB;
  a.ldb = ldb;
  a.ctrl = reinterpret_cast<LuFwdCtrl *>(ws + L.ctrl);
  a.flags = reinterpret_cast<int *>(ws + L.flags);
  a.timeout_ns = 10000000000ll;
  CHOL_CUDA_TRY(cudaMemsetAsync(ws, 0, L.sweep, s));  // control block and flags
  const int grid = (int)std::min<int64_t>(a.nitems, (int64_t)di.sms);
  lu_fwd_kernel<<<grid, NT, LU_FWD_SMEM_REQ, s>>>(a);
  CHOL_CUDA_TRY(cudaGetLastError());
  // U X = Y, skipped if the transformation aborted
  const chol_status st = solve_upper_f64(n, nrhs, dF, lda, dB, ldb, ws + L.sweep, &a.ctrl->abort, s);
  if (st != CHOL_OK) return st;
  if (dInfo) {
    lu_info_kernel<<<1, 32, 0, s>>>(a.ctrl, dInfo);
    CHOL_CUDA_TRY(cudaGetLastError());
    return solve_upper_info(ws + L.sweep, dInfo, s);
  }
  return CHOL_OK;
}
