// Device-side helpers shared by the kernel translation units.
#pragma once

#include "plam_common.cuh"

namespace plam {

// Deterministic sum over a block: every thread passes its value; the result is
// returned to every thread.  Fixed butterfly inside each warp, then warp
// results added in warp order by warp 0.  `scratch` holds >= 33 doubles.
__device__ inline double block_sum(double v, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += scratch[i];
    scratch[32] = s;
  }
  __syncthreads();
  return scratch[32];
}

__device__ inline float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ inline T fma_t(T a, T b, T c) { return fma(a, b, c); }

}  // namespace plam
