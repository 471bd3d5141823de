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

// N independent Montgomery products in one out-of-line call: the compiler
// interleaves the N carry chains, so the call costs about the latency of one
// product instead of N.
template <int N>
struct FrN {
  Fr x[N];
};

template <int N>
static __device__ __noinline__ FrN<N> mont_mul_batch(FrN<N> a, FrN<N> b) {
  FrN<N> c;
#pragma unroll
  for (int q = 0; q < N; q++) c.x[q] = mont_mul(a.x[q], b.x[q]);
  return c;
}

// N independent REDCs of 64-bit column sums, interleaved the same way.
template <int N>
struct U64x8N {
  U64x8 x[N];
};

template <int N>
static __device__ __noinline__ FrN<N> redc_batch(U64x8N<N> a) {
  FrN<N> c;
#pragma unroll
  for (int q = 0; q < N; q++) c.x[q] = redc_columns(a.x[q].v);
  return c;
}

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
