// Tensor-core tile update for the low-precision factor: C (FP32) -= A B^T on the fifth-
// generation tensor cores (tcgen05), BF16 operands and FP32 accumulation in tensor memory.
//
// An FP32 operand x is rounded to NTERM BF16 terms, x ~ t0 + t1 + t2 with t0 = bf16(x),
// t1 = bf16(x - t0), t2 = bf16(x - t0 - t1):
//   NTERM = 1  plain BF16 operands (8-bit significands), the BF16 variant of the factor;
//   NTERM = 3  24 significant bits, so the split is exact for every FP32 value whose terms do
//              not underflow, and the six products t_i t_j with i + j <= 2 are accumulated
//              (the dropped ones are below 2^-24 relative): an FP32-accurate product.
//
// Block of C: 256 x 256 (two M = 128 halves, one MMA N = 256), accumulators in 512 TMEM
// columns (half h at columns 256 h, row r of the half in lane r). K is consumed in chunks of
// KC, double-buffered in shared memory: all 256 threads load a chunk (one row of A and one row
// of B per thread, coalesced over rows), split it and store it in the K-major core-matrix
// layout (8 rows x 16 bytes per core matrix, no swizzle); one thread issues the MMAs of the
// chunk and commits them to the chunk's mbarrier, and the threads refill a stage only after
// the MMAs that read it have completed. The epilogue reads the accumulators with tcgen05.ld
// (warp w: lanes 32 (w mod 4).., half w / 4, one row of C per thread) and writes C - acc.
//
// Every wait is bounded (globaltimer); on expiry the body reports an error and returns.
#pragma once
#include <stdint.h>
#include <cuda_bf16.h>

namespace chol {
namespace tc {

constexpr int NT = 256;
constexpr int TM = 256, TN = 256;
constexpr int TMEM_COLS = 512;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s

template <int NTERM>
struct Cfg {
  static constexpr int KC = 32;                    // k per stage
  static constexpr int OPB = TM * KC * 2;          // bytes of one term of one operand in a stage
  static constexpr int STAGE = 2 * NTERM * OPB;    // A and B, all terms
  static constexpr int SMEM = 2 * STAGE;           // two stages
  static constexpr int SBO = (KC / 8) * 128;       // byte stride between 8-row groups
  static constexpr int LBO = 128;                  // byte stride between K-adjacent core matrices
  static constexpr int NPROD = NTERM == 1 ? 1 : (NTERM == 2 ? 3 : 6);
};

// per-block state that lives across tasks (static shared memory, not the dynamic buffer the
// other bodies and the scheduler share)
struct State {
  uint64_t mbar[2];  // MMA completion of the chunks in stage 0 / 1 (tcgen05.commit)
  uint64_t full[2];  // bulk copies into stage 0 / 1 complete (transaction bytes)
  uint32_t tmem;
  uint32_t chunks;   // chunks issued so far by this block (stage = chunk & 1)
  uint32_t fb[2];    // phases of full[0] / full[1] used so far
  int err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte
// offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D FP32, A and B BF16, both K-major, N = 256, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint64_t *mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase of parity `par` of an mbarrier; false on expiry of the time limit
__device__ __forceinline__ bool mbar_wait(uint64_t *mb, uint32_t par) {
  if (mbar_try(mb, par)) return true;
  const uint64_t t0 = globaltimer();
  for (int64_t it = 0; it < (int64_t)1 << 34; ++it) {
    if (mbar_try(mb, par)) return true;
    if (globaltimer() - t0 > WAIT_LIMIT_NS) return false;
  }
  return false;
}

// wait until the commit of chunk q (barrier q & 1, phase (q >> 1) & 1) has arrived
__device__ __forceinline__ bool wait_chunk(State &s, uint32_t q) { return mbar_wait(&s.mbar[q & 1], (q >> 1) & 1u); }

// one thread: expect `bytes` on full[st] and copy them from global memory into the stage
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint64_t *mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

// Allocate the accumulators and set up the barriers; all threads of the block call it.
__device__ __forceinline__ void begin(State &s) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s.mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s.mbar[1])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s.full[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s.full[1])) : "memory");
    s.fb[0] = 0;
    s.fb[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s.chunks = 0;
    s.err = 0;
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

// Wait for any MMA still in flight (bounded), then free the accumulators; all threads call it.
__device__ __forceinline__ void end(State &s) {
  __syncthreads();
  if (s.chunks > 0) {
    const uint32_t last = s.chunks - 1;
    wait_chunk(s, last);
    if (last > 0) wait_chunk(s, last - 1);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "r"(TMEM_COLS) : "memory");
}

// the six (or three, or one) products t_a t_b, smallest first
template <int NTERM>
__device__ __forceinline__ void prod_terms(int i, int &ta, int &tb) {
  if (NTERM == 1) { ta = 0; tb = 0; return; }
  if (NTERM == 2) { ta = i == 0 ? 1 : 0; tb = i == 1 ? 1 : 0; return; }
  const int a_[6] = {2, 0, 1, 1, 0, 0}, b_[6] = {0, 2, 1, 0, 1, 0};
  ta = a_[i]; tb = b_[i];
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// Load k = k0 .. k0 + KC - 1 of row `row` of P (column-major, ld) into registers; rows at or
// past R and k at or past K read as zero.
template <int KC>
__device__ __forceinline__ void load_row(float (&v)[KC], const float *P, int64_t ld, int R, int row, int k0, int K) {
  const bool ok = row < R;
#pragma unroll
  for (int e = 0; e < KC; ++e) {
    const int k = k0 + e;
    v[e] = (ok && k < K) ? __ldcg(P + (int64_t)k * ld + row) : 0.f;
  }
}

// Store the NTERM BF16 terms of one row of a chunk into the stage buffer `dst` (term t at
// dst + t * OPB), K-major core-matrix layout.
template <int NTERM>
__device__ __forceinline__ void store_row(unsigned char *dst, const float (&v)[Cfg<NTERM>::KC], int row) {
  using C = Cfg<NTERM>;
#pragma unroll
  for (int g = 0; g < C::KC / 8; ++g) {
    const uint32_t off = (uint32_t)(((row >> 3) * (C::KC / 8) + g) * 128 + (row & 7) * 16);
    float r[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) r[e] = v[8 * g + e];
#pragma unroll
    for (int t = 0; t < NTERM; ++t) {
      float b[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        b[e] = __bfloat162float(__float2bfloat16_rn(r[e]));
        r[e] = r[e] - b[e];
      }
      uint4 w;
      w.x = pack2(b[0], b[1]);
      w.y = pack2(b[2], b[3]);
      w.z = pack2(b[4], b[5]);
      w.w = pack2(b[6], b[7]);
      *reinterpret_cast<uint4 *>(dst + t * C::OPB + off) = w;
    }
  }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// C[M x N] -= A[M x K] B[N x K]^T (column-major FP32); with `lower` only row >= column is
// written. Called by all NT threads with State from begin(); `smem` holds Cfg<NTERM>::SMEM
// bytes (16-byte aligned). Returns 0, or -1 when a wait expired (the caller aborts).
template <int NTERM>
__device__ __noinline__ int update_nt(float *Cm, int64_t ldc, const float *A, int64_t lda, const float *B,
                                      int64_t ldb, int M, int N, int K, bool lower, unsigned char *smem,
                                      State &s) {
  using C = Cfg<NTERM>;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(smem);
  for (int bn = 0; bn < N; bn += TN) {
    for (int bm = 0; bm < M; bm += TM) {
      if (lower && bm + TM <= bn) continue;
      const int mb = min(TM, M - bm), nbk = min(TN, N - bn);
      const int nchunk = (K + C::KC - 1) / C::KC;
      if (nchunk == 0) continue;
      const uint32_t c0 = s.chunks;  // same value in every thread (written before a barrier)
      // registers hold the raw values of the chunk being stored and of the next one, so the
      // loads of chunk ci + 1 are in flight while chunk ci is split, stored and multiplied
      float ra[C::KC], rb[C::KC], na[C::KC], nb[C::KC];
      load_row<C::KC>(ra, A + bm, lda, mb, tid, 0, K);
      load_row<C::KC>(rb, B + bn, ldb, nbk, tid, 0, K);
      for (int ci = 0; ci < nchunk; ++ci) {
        const uint32_t q = c0 + ci;
        const int st = q & 1;
        if (ci + 1 < nchunk) {
          load_row<C::KC>(na, A + bm, lda, mb, tid, (ci + 1) * C::KC, K);
          load_row<C::KC>(nb, B + bn, ldb, nbk, tid, (ci + 1) * C::KC, K);
        }
        // the MMAs of chunk q - 2 read this stage
        if (q >= 2 && !wait_chunk(s, q - 2)) s.err = 1;
        unsigned char *stg = smem + st * C::STAGE;
        store_row<NTERM>(stg, ra, tid);
        store_row<NTERM>(stg + NTERM * C::OPB, rb, tid);
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        if (s.err) {  // chunks before q were issued; end() waits for them
          if (tid == 0) s.chunks = q;
          return -1;
        }
        if (tid == 0) {
          fence_after_sync();
          const uint32_t sa = sbase + st * C::STAGE, sb = sa + NTERM * C::OPB;
#pragma unroll
          for (int ks = 0; ks < C::KC / 16; ++ks) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
              for (int pi = 0; pi < C::NPROD; ++pi) {
                int ta, tb;
                prod_terms<NTERM>(pi, ta, tb);
                const uint64_t ad = sdesc(sa + ta * C::OPB + h * 16 * C::SBO + ks * 256, C::LBO, C::SBO);
                const uint64_t bd = sdesc(sb + tb * C::OPB + ks * 256, C::LBO, C::SBO);
                mma_bf16(s.tmem + 256 * h, ad, bd, (ci > 0 || ks > 0 || pi > 0) ? 1u : 0u);
              }
            }
          }
          mma_commit(&s.mbar[st]);
        }
#pragma unroll
        for (int e = 0; e < C::KC; ++e) { ra[e] = na[e]; rb[e] = nb[e]; }
      }
      // epilogue: thread = one row of the block, 256 columns in 8 loads of 32; the C values of
      // the next 32 columns are loaded while the current ones are written
      const int qd = warp & 3, h = warp >> 2;
      const int r = 128 * h + 32 * qd + lane;
      const int ncb = (nbk + 31) / 32;
      float cv[32], cn[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const bool w = r < mb && j < nbk && (!lower || bm + r >= bn + j);
        cv[j] = w ? __ldcg(Cm + (int64_t)(bn + j) * ldc + bm + r) : 0.f;
      }
      const uint32_t last = c0 + nchunk - 1;
      const bool ok = wait_chunk(s, last);
      fence_after_sync();
      if (!ok) s.err = 1;
      __syncthreads();
      if (s.err) {
        if (tid == 0) s.chunks = c0 + nchunk;
        return -1;
      }
#pragma unroll 1
      for (int cb = 0; cb < ncb; ++cb) {
        if (cb + 1 < ncb) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int c = 32 * (cb + 1) + j;
            const bool w = r < mb && c < nbk && (!lower || bm + r >= bn + c);
            cn[j] = w ? __ldcg(Cm + (int64_t)(bn + c) * ldc + bm + r) : 0.f;
          }
        }
        uint32_t v[32];
        tmem_ld32(s.tmem + ((uint32_t)(32 * qd) << 16) + 256 * h + 32 * cb, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = 32 * cb + j;
          const bool w = r < mb && c < nbk && (!lower || bm + r >= bn + c);
          if (w) __stcg(Cm + (int64_t)(bn + c) * ldc + bm + r, cv[j] - __uint_as_float(v[j]));
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) cv[j] = cn[j];
      }
      fence_before_sync();
      __syncthreads();
      if (tid == 0) s.chunks = c0 + nchunk;
      __syncthreads();
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------------------
// Pre-split operands. The TRSM that produces a panel tile also writes its NTERM BF16 terms,
// already in the stage layout, to a side buffer: chunk c (tile columns 32 c .. 32 c + 31) is
// NTERM term blocks of OPB bytes, each the K-major core-matrix layout of 256 rows x 32 k. A
// GEMM/SYRK then moves a chunk of each operand into a stage with one bulk copy (the copy
// engine, completion counted in bytes on the stage's full barrier), and one thread keeps the
// tensor core fed while the copy of the next chunk runs.

template <int NTERM>
struct Split {
  static constexpr int CHUNK = NTERM * Cfg<NTERM>::OPB;
  static constexpr size_t tile_bytes(int nb) { return (size_t)(nb / Cfg<NTERM>::KC) * CHUNK; }
};

// Emitter for the row-per-thread TRSM: row r's values of tile columns 32 c .. 32 c + 31 are
// split into `buf` (two chunk buffers in shared memory, alternating), and after each column
// block one thread writes the chunk to the tile's side buffer with one bulk copy (shared ->
// global, bulk async-group). Before the task completes, finish() waits for the copies and
// orders them (async proxy) before the completion's release, so the updates that bulk-copy
// the tile see it.
// The BF16 terms of one band of 64 rows [r0, r0 + 64) of a panel tile, for f32::trsm_band:
// the 64 rows of one term form one contiguous 4 KiB range of a chunk (8-row groups of 512
// bytes), so the band is staged compactly (term t of chunk c at buf + ((c & 1) NTERM + t) 4 KiB)
// and each flush copies NTERM ranges to their place in the chunk.
template <int NTERM>
struct SplitEmitBand {
  static constexpr int ROWS = 64;
  static constexpr int BAND = ROWS / 8 * 512;  // bytes of one term of the band
  static constexpr int BYTES = 2 * NTERM * BAND;
  unsigned char *tile;  // global: the tile's chunks
  unsigned char *buf;   // shared: BYTES, 16-byte aligned
  int r0;               // first row of the band in the tile (a multiple of 64)
  __device__ void store(int r, int c, const float (&v)[32]) const {
    unsigned char *dst = buf + (c & 1) * NTERM * BAND;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const uint32_t off = (uint32_t)(((r >> 3) * 4 + g) * 128 + (r & 7) * 16);
      float x[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) x[e] = v[8 * g + e];
#pragma unroll
      for (int t = 0; t < NTERM; ++t) {
        float b[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          b[e] = __bfloat162float(__float2bfloat16_rn(x[e]));
          x[e] = x[e] - b[e];
        }
        uint4 w;
        w.x = pack2(b[0], b[1]);
        w.y = pack2(b[2], b[3]);
        w.z = pack2(b[4], b[5]);
        w.w = pack2(b[6], b[7]);
        *reinterpret_cast<uint4 *>(dst + t * BAND + off) = w;
      }
    }
  }
  __device__ void row(int r, int c, const float (&v)[32]) const { store(r, c, v); }
  __device__ void zero(int r, int c) const {
    float z[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) z[e] = 0.f;
    store(r, c, z);
  }
  __device__ void flush(int c) const {
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int t = 0; t < NTERM; ++t) {
        const size_t go = (size_t)c * Split<NTERM>::CHUNK + (size_t)t * Cfg<NTERM>::OPB + (size_t)(r0 / 8) * 512;
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(tile + go),
                     "r"(smem_u32(buf + ((c & 1) * NTERM + t) * BAND)), "r"((uint32_t)BAND)
                     : "memory");
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
    }
    __syncthreads();
  }
  __device__ void finish() const {
    if (threadIdx.x == 0) {
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
  }
};

// C[M x N] -= A B^T with both operands pre-split (sa, sb: their tiles in the side buffer), K a
// multiple of 32, M, N <= 256. Same accumulators and epilogue as update_nt. Returns 0, or -1
// when a wait expired.
template <int NTERM>
__device__ __noinline__ int update_nt_split(float *Cm, int64_t ldc, const unsigned char *sa, const unsigned char *sb,
                                            int M, int N, int K, bool lower, unsigned char *smem, State &s) {
  using C = Cfg<NTERM>;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(smem);
  const int nchunk = K / C::KC;
  const uint32_t c0 = s.chunks;  // same value in every thread (written before a barrier)
  __syncthreads();               // everyone has read it before thread 0 moves it on
  if (tid == 0) {
    // data written by other SMs with ordinary stores, read here by the copy engine
    asm volatile("fence.proxy.async.global;" ::: "memory");
    int issued = 0;
    for (int ci = 0; ci < nchunk; ++ci) {
      const uint32_t q = c0 + ci;
      const int st = q & 1;
      if (q >= 2 && !wait_chunk(s, q - 2)) { s.err = 1; break; }  // the MMAs that read this stage
      const uint32_t bytes = NTERM * C::OPB;
      const uint32_t sa_s = sbase + st * C::STAGE, sb_s = sa_s + bytes;
      mbar_expect_tx(&s.full[st], 2 * bytes);
      bulk_g2s(sa_s, sa + (size_t)ci * bytes, bytes, &s.full[st]);
      bulk_g2s(sb_s, sb + (size_t)ci * bytes, bytes, &s.full[st]);
      const bool ok = mbar_wait(&s.full[st], s.fb[st] & 1u);
      ++s.fb[st];
      if (!ok) { s.err = 1; break; }
      fence_after_sync();
#pragma unroll
      for (int ks = 0; ks < C::KC / 16; ++ks) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int pi = 0; pi < C::NPROD; ++pi) {
            int ta, tb;
            prod_terms<NTERM>(pi, ta, tb);
            const uint64_t ad = sdesc(sa_s + ta * C::OPB + h * 16 * C::SBO + ks * 256, C::LBO, C::SBO);
            const uint64_t bd = sdesc(sb_s + tb * C::OPB + ks * 256, C::LBO, C::SBO);
            mma_bf16(s.tmem + 256 * h, ad, bd, (ci > 0 || ks > 0 || pi > 0) ? 1u : 0u);
          }
        }
      }
      mma_commit(&s.mbar[st]);
      issued = ci + 1;
    }
    s.chunks = c0 + issued;
  }
  // epilogue: thread = one row of the block, 256 columns in 8 loads of 32; the C values of
  // the next 32 columns are loaded while the current ones are written
  const int qd = warp & 3, h = warp >> 2;
  const int r = 128 * h + 32 * qd + lane;
  const int ncb = (N + 31) / 32;
  float cv[32], cn[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const bool w = r < M && j < N && (!lower || r >= j);
    cv[j] = w ? __ldcg(Cm + (int64_t)j * ldc + r) : 0.f;
  }
  __syncthreads();
  if (s.err) return -1;
  const bool ok = wait_chunk(s, c0 + nchunk - 1);
  fence_after_sync();
  if (!ok) s.err = 1;
  __syncthreads();
  if (s.err) return -1;
#pragma unroll 1
  for (int cb = 0; cb < ncb; ++cb) {
    if (cb + 1 < ncb) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = 32 * (cb + 1) + j;
        const bool w = r < M && c < N && (!lower || r >= c);
        cn[j] = w ? __ldcg(Cm + (int64_t)c * ldc + r) : 0.f;
      }
    }
    uint32_t v[32];
    tmem_ld32(s.tmem + ((uint32_t)(32 * qd) << 16) + 256 * h + 32 * cb, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = 32 * cb + j;
      const bool w = r < M && c < N && (!lower || r >= c);
      if (w) __stcg(Cm + (int64_t)c * ldc + r, cv[j] - __uint_as_float(v[j]));
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) cv[j] = cn[j];
  }
  fence_before_sync();
  __syncthreads();
  return 0;
}

}  // namespace tc
}  // namespace chol
