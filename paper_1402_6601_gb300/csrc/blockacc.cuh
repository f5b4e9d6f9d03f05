// Thread layout for the products "32-row block x (32 x G right-hand-side block)" that the
// FP64 residual of the refinement accumulates, inside a 256-thread block: lane = row of the
// block, warp = slice.
//
// CPT columns per thread (compile time), CSP column slices (a power of two, CSP * CPT >= G)
// and KS = 8 / CSP k-slices: warp w owns columns (w % CSP) * CPT + q and the k values
// w / CSP + KS * t. Every fused multiply-add issued therefore works on a live column (or
// the zero padding of a ragged last group): predicated-off FP64 instructions would still
// occupy the FP64 pipe. With KS > 1 the k-slices are summed once at the end of a block.
#pragma once

namespace chol {

template <int CPT>
struct Slices {
  int csp, ks, cs, kslice;
  __device__ __forceinline__ Slices(int G, int warp) {
    const int need = (G + CPT - 1) / CPT;
    csp = 1;
    while (csp < need && csp < 8) csp <<= 1;
    ks = 8 / csp;
    cs = warp % csp;
    kslice = warp / csp;
  }
  __device__ __forceinline__ int col(int q) const { return cs * CPT + q; }
  __device__ __forceinline__ int width() const { return csp * CPT; }
};

// acc[q] -= sum_k Ls[rr][k] * Ys[k][col(q)] over this thread's k values.
template <class T, int CPT>
__device__ __forceinline__ void acc_step(T (&acc)[CPT], const T *Ls, int sld, const T *Ys, int sg, int rr,
                                         const Slices<CPT> &s) {
  const int nt = 32 / s.ks;
#pragma unroll 4
  for (int t = 0; t < nt; ++t) {
    const int k = s.kslice + s.ks * t;
    const T l = Ls[rr * sld + k];
#pragma unroll
    for (int q = 0; q < CPT; ++q) acc[q] = fma(-l, Ys[k * sg + s.col(q)], acc[q]);
  }
}

// Sum the k-slices and leave the 32 x G result in Out[row * sg + col]; Red must hold
// 32 * 8 * CPT values. Ends with the block synchronised.
template <class T, int CPT>
__device__ __forceinline__ void acc_finish(const T (&acc)[CPT], T *Out, int sg, T *Red, int rr, int G,
                                           const Slices<CPT> &s) {
  if (s.ks == 1) {
#pragma unroll
    for (int q = 0; q < CPT; ++q)
      if (s.col(q) < G) Out[rr * sg + s.col(q)] = acc[q];
    __syncthreads();
    return;
  }
  const int w = s.width();
#pragma unroll
  for (int q = 0; q < CPT; ++q) Red[(s.kslice * w + s.col(q)) * 32 + rr] = acc[q];
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * G; e += blockDim.x) {
    const int r = e & 31, c = e >> 5;
    T t = T(0);
    for (int k = 0; k < s.ks; ++k) t += Red[(k * w + c) * 32 + r];
    Out[r * sg + c] = t;
  }
  __syncthreads();
}

// columns per thread for a group of G right-hand sides
inline int cpt_for(int G) { return G >= 5 ? 8 : (G >= 3 ? 4 : (G == 2 ? 2 : 1)); }

}  // namespace chol
