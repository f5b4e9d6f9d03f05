// Throughput probes of the FP64 units: measurement support for the roofline of the FP64
// factor, not part of the method. One kernel keeps every SM's FP64 pipe busy with
// independent fused multiply-adds (DFMA, the instruction the FP64 tile bodies use); the
// others issue the FP64 warp-level MMA shapes (mma.sync ... .f64) back to back. The host
// times a launch on its stream; chol_probe_fp64_flops gives the flops of that launch.
//
// Every thread (DFMA: 16 chains) or warp (MMA: PROBE_CHAINS chains) runs independent
// accumulation chains, so the pipe, not the latency of one chain, bounds the rate. The
// operands are runtime values and the accumulators are stored (under a condition the compiler
// cannot decide), so no work is folded away; every product is about 2^-40, so the
// accumulators stay near 1 for any iteration count.
#include "common.cuh"

namespace chol {

constexpr int PROBE_CHAINS = 8;

// DFMA in the pattern of the factor's register tile: 4 x 4 accumulators acc[i][j] +=
// a[i] b[j], sixteen independent chains per thread with distinct operand registers.
__global__ void __launch_bounds__(256) probe_dfma_kernel(long long iters, double x, double y, double *out) {
  double a[4], b[4], acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[i] = y * (1.0 + 0.125 * i);
    b[i] = x * y * (1.0 + 0.0625 * i + 1e-9 * threadIdx.x);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 1.0;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += acc[i][j];
  if (s == -1.0) out[0] = s;  // never true (every accumulator stays >= 1)
}

// DFMA with every chain on its own three registers: x_c <- x_c y_c + z_c (y_c = 1 - 2^-20 c',
// z_c small), so no two FMAs of an iteration read a common operand register.
__global__ void __launch_bounds__(256) probe_dfma_free_kernel(long long iters, double x, double y, double *out) {
  double a[16], m[16], c[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    a[i] = 1.0 + 1e-3 * i + 1e-9 * threadIdx.x;
    m[i] = x - y * (double)i;
    c[i] = y * (1.0 + 0.0625 * i);
  }
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = fma(a[i], m[i], c[i]);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += a[i];
  if (s == -1.0) out[0] = s;  // never true (every chain stays near its fixed point, about 1)
}

// DFMA fed from shared memory as in the FP64 tile update: per step every thread reads four
// rows of A and four columns of B (k-major 32 x 64 panels) and updates its 4 x 4 register tile.
__global__ void __launch_bounds__(256) probe_dfma_smem_kernel(long long iters, double x, double y, double *out) {
  __shared__ double As[32 * 64], Bs[32 * 64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < 32 * 64; e += 256) {
    As[e] = y * (1.0 + 1e-3 * (e & 63));
    Bs[e] = x * y * (1.0 + 1e-3 * (e >> 6));
  }
  __syncthreads();
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 1.0;
  for (long long it = 0; it < iters; it += 32) {
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk * 64 + tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk * 64 + ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += acc[i][j];
  if (s == -1.0) out[0] = s;  // never true (every accumulator stays >= 1)
}

// Per shape: fragment sizes (doubles per thread) of A, B and C/D, and M, N, K.
template <int KIND>
struct MmaShape;
template <>
struct MmaShape<1> {  // m8n8k4
  static constexpr int NA = 1, NB = 1, NC = 2, M = 8, N = 8, K = 4;
  __device__ static void mma(double *d, const double *a, const double *b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a[0]), "d"(b[0]));
  }
};
template <>
struct MmaShape<2> {  // m16n8k4
  static constexpr int NA = 2, NB = 1, NC = 4, M = 16, N = 8, K = 4;
  __device__ static void mma(double *d, const double *a, const double *b) {
    asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0, %1, %2, %3}, {%4, %5}, {%6}, "
                 "{%0, %1, %2, %3};"
                 : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
                 : "d"(a[0]), "d"(a[1]), "d"(b[0]));
  }
};
template <>
struct MmaShape<3> {  // m16n8k8
  static constexpr int NA = 4, NB = 2, NC = 4, M = 16, N = 8, K = 8;
  __device__ static void mma(double *d, const double *a, const double *b) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
                 : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
  }
};
template <>
struct MmaShape<4> {  // m16n8k16
  static constexpr int NA = 8, NB = 4, NC = 4, M = 16, N = 8, K = 16;
  __device__ static void mma(double *d, const double *a, const double *b) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0, %1, %2, %3}, "
                 "{%4, %5, %6, %7, %8, %9, %10, %11}, {%12, %13, %14, %15}, {%0, %1, %2, %3};"
                 : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
                 : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
                   "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
  }
};

// The MMA chains multiply small operands (|a b| summed over K stays below 2^-10) into
// accumulators that start at 1, so they stay finite for any iteration count.
template <int KIND>
__global__ void __launch_bounds__(256) probe_mma_kernel(long long iters, double x, double y, double *out) {
  using S = MmaShape<KIND>;
  double a[S::NA], b[S::NB], d[PROBE_CHAINS][S::NC];
#pragma unroll
  for (int i = 0; i < S::NA; ++i) a[i] = y * (1.0 + 1e-3 * i);
#pragma unroll
  for (int i = 0; i < S::NB; ++i) b[i] = y * x;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c)
#pragma unroll
    for (int i = 0; i < S::NC; ++i) d[c][i] = 1.0 + 1e-7 * threadIdx.x;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) S::mma(d[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c)
#pragma unroll
    for (int i = 0; i < S::NC; ++i) s += d[c][i];
  if (s == -1.0) out[0] = s;  // never true (every accumulator stays >= 1)
}

static long long mma_flops_per_warp_iter(int kind) {
  switch (kind) {
    case 1: return 2ll * 8 * 8 * 4 * PROBE_CHAINS;
    case 2: return 2ll * 16 * 8 * 4 * PROBE_CHAINS;
    case 3: return 2ll * 16 * 8 * 8 * PROBE_CHAINS;
    case 4: return 2ll * 16 * 8 * 16 * PROBE_CHAINS;
    default: return 0;
  }
}

}  // namespace chol

using namespace chol;

extern "C" long long chol_probe_fp64_flops(int kind, int blocks, int threads, long long iters) {
  if (blocks < 1 || threads < 32 || threads > 256 || threads % 32 || iters < 0) return -1;
  if (kind == 0 || kind == 5) return 2ll * 16 * iters * threads * (long long)blocks;
  if (kind == 6) return 2ll * 16 * ((iters + 31) / 32 * 32) * threads * (long long)blocks;
  const long long per = mma_flops_per_warp_iter(kind);
  if (per == 0) return -1;
  return per * iters * (threads / 32) * (long long)blocks;
}

extern "C" chol_status chol_probe_fp64(int kind, int blocks, int threads, long long iters, double *dOut,
                                       void *stream) {
  if (chol_probe_fp64_flops(kind, blocks, threads, iters) < 0 || !dOut) return CHOL_ERR_INVALID_ARG;
  const DeviceInfo di = current_device_info();
  if (di.sms <= 0) return CHOL_ERR_CUDA;
  if (di.cc_major != 10 || di.cc_minor != 3) return CHOL_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const double x = 1.0 - 0x1p-20, y = 0x1p-20;
  switch (kind) {
    case 0: probe_dfma_kernel<<<blocks, threads, 0, s>>>(iters, x, y, dOut); break;
    case 5: probe_dfma_free_kernel<<<blocks, threads, 0, s>>>(iters, x, y, dOut); break;
    case 6:
      if (threads != 256) return CHOL_ERR_INVALID_ARG;  // the 16 x 16 thread tile
      probe_dfma_smem_kernel<<<blocks, threads, 0, s>>>(iters, x, y, dOut);
      break;
    case 1: probe_mma_kernel<1><<<blocks, threads, 0, s>>>(iters, x, y, dOut); break;
    case 2: probe_mma_kernel<2><<<blocks, threads, 0, s>>>(iters, x, y, dOut); break;
    case 3: probe_mma_kernel<3><<<blocks, threads, 0, s>>>(iters, x, y, dOut); break;
    case 4: probe_mma_kernel<4><<<blocks, threads, 0, s>>>(iters, x, y, dOut); break;
    default: return CHOL_ERR_INVALID_ARG;
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}
