// Out-of-line field operations for the latency-bound kernels (prologue,
// rounds).  Their loops do little arithmetic in total, but inlining the
// ~550-instruction Montgomery product at every call site makes those kernels
// larger than the instruction cache; one shared copy per module avoids it.
#pragma once
#include "fr.cuh"

namespace vl {

struct U64x8 {
  uint64_t v[8];
};

static __device__ __noinline__ Fr mont_mul_ni(Fr a, Fr b) { return mont_mul(a, b); }

static __device__ __noinline__ Fr redc_columns_ni(U64x8 acc) { return redc_columns(acc.v); }

__device__ __forceinline__ Fr to_mont_ni(const Fr& a) { return mont_mul_ni(a, fr_r2()); }
__device__ __forceinline__ Fr from_mont_ni(const Fr& a) { return mont_mul_ni(a, fr_small(1)); }

// (lo + hi . 2^256) mod r, canonical (hi . 2^256 = mont_mul(hi, R^2)).
__device__ __forceinline__ Fr reduce_512_ni(const Fr& lo, const Fr& hi) {
  const Fr h = mont_mul_ni(hi, fr_r2());
  Fr l = lo;
  cond_sub_r(l.v, 0);
  cond_sub_r(l.v, 0);
  return fr_add(l, h);
}

}  // namespace vl
