// Warp- and block-wide sums of field elements (device).
#pragma once
#include "fr.cuh"

namespace vl {

__device__ __forceinline__ Fr shfl_xor_fr(const Fr& x, int off) {
  Fr y;
#pragma unroll
  for (int l = 0; l < 8; l++) y.v[l] = __shfl_xor_sync(0xffffffffu, x.v[l], off);
  return y;
}

__device__ __forceinline__ Fr warp_sum_fr(Fr x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x = fr_add(x, shfl_xor_fr(x, off));
  return x;
}

// Sum over the block of NV field elements per thread; the result is valid in
// every thread of warp 0.  `sh` needs NV * (blockDim.x / 32) entries.
template <int NV>
__device__ __forceinline__ void block_sum_fr(Fr (&x)[NV], Fr* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; q++) x[q] = warp_sum_fr(x[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) sh[q * nw + warp] = x[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) {
      x[q] = lane < nw ? sh[q * nw + lane] : fr_zero();
      x[q] = warp_sum_fr(x[q]);
    }
  }
  __syncthreads();
}

}  // namespace vl
