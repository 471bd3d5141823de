// Warp- and block-wide sums of field elements (device).
#pragma once
#include "fr.cuh"
#include "fr_dev.cuh"

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

// Sum a[32] over the 32 lanes of a warp; lane L returns the total of a[L].
__device__ __forceinline__ unsigned long long warp_transpose_sum(unsigned long long (&a)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; i++) {
      unsigned long long send = upper ? a[i] : a[i + off];
      unsigned long long keep = upper ? a[i + off] : a[i];
      unsigned long long recv = __shfl_xor_sync(0xffffffffu, send, off);
      a[i] = keep + recv;
    }
  }
  return a[0];
}

// Sum of NV field elements per thread (Montgomery form) over the block, as
// canonical values: the eight 32-bit limbs are summed as 64-bit integers
// (exact for up to 2^32 terms; no modular reduction per level), and one
// REDC of the column sums gives (sum x.R) . R^-1 = sum x mod r.  Results in
// out[0..NV).  sh: NV * 8 * (blockDim.x / 32) 64-bit slots.  Block-wide.
template <int NV>
__device__ __forceinline__ void block_sum_canonical(const Fr (&x)[NV], Fr* out, unsigned long long* sh) {
  static_assert(NV * 8 <= 32, "at most 4 values");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long a[32];
#pragma unroll
  for (int i = 0; i < 32; i++) a[i] = i < NV * 8 ? (unsigned long long)x[i / 8].v[i % 8] : 0ull;
  const unsigned long long s = warp_transpose_sum(a);
  if (lane < NV * 8) sh[warp * NV * 8 + lane] = s;
  __syncthreads();
  if (warp == 0) {
    unsigned long long t = 0;
    if (lane < NV * 8)
      for (int w = 0; w < nw; w++) t += sh[w * NV * 8 + lane];
    U64x8 col;
#pragma unroll
    for (int l = 0; l < 8; l++) col.v[l] = __shfl_sync(0xffffffffu, t, (lane * 8 + l) & 31);
    if (lane < NV) out[lane] = redc_columns_ni(col);
  }
  __syncthreads();
}

}  // namespace vl
