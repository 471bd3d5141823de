// BLS12-381 scalar field F_r, 8 x 32-bit little-endian limbs, Montgomery
// arithmetic with R = 2^256 (host and device).
//
// The field is the one Sec. V fixes for the protocol (BLS12-381, |F| ~ 2^254):
//   r = 0x73eda753299d7d483339d80809a1d80553bda402fffe5bfeffffffff00000001.
// r < 2^255, so a sum of two reduced elements never overflows 256 bits.
// Limb constants below were derived from r by modular exponentiation:
//   R1 = 2^256 mod r, R2 = 2^512 mod r, R3 = 2^768 mod r, n' = -r^-1 mod 2^32.
//
// Representations used by the prover:
//   canonical      x in [0, r)                 (ABI, proofs, transcript)
//   Montgomery     x.R mod r                   (device arithmetic)
//   double-Mont.   x.R^2 mod r                 (eq-table weights of the int16
//                  fold: one REDC of sum(E.R^2 . p) lands in Montgomery form)
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define VL_HD __host__ __device__ __forceinline__
#else
#define VL_HD inline
#endif

namespace vl {

struct Fr {
  uint32_t v[8];
};

VL_HD constexpr uint32_t r_limb(int i) {
  return i == 0 ? 0x00000001u : i == 1 ? 0xffffffffu : i == 2 ? 0xfffe5bfeu
       : i == 3 ? 0x53bda402u : i == 4 ? 0x09a1d805u : i == 5 ? 0x3339d808u
       : i == 6 ? 0x299d7d48u : 0x73eda753u;
}
VL_HD constexpr uint32_t r1_limb(int i) {  // R mod r  (Montgomery form of 1)
  return i == 0 ? 0xfffffffeu : i == 1 ? 0x00000001u : i == 2 ? 0x00034802u
       : i == 3 ? 0x5884b7fau : i == 4 ? 0xecbc4ff5u : i == 5 ? 0x998c4fefu
       : i == 6 ? 0xacc5056fu : 0x1824b159u;
}
VL_HD constexpr uint32_t r2_limb(int i) {  // R^2 mod r
  return i == 0 ? 0xf3f29c6du : i == 1 ? 0xc999e990u : i == 2 ? 0x87925c23u
       : i == 3 ? 0x2b6cedcbu : i == 4 ? 0x7254398fu : i == 5 ? 0x05d31496u
       : i == 6 ? 0x9f59ff11u : 0x0748d9d9u;
}
VL_HD constexpr uint32_t r3_limb(int i) {  // R^3 mod r
  return i == 0 ? 0x439b73afu : i == 1 ? 0xc62c1807u : i == 2 ? 0x8cf06990u
       : i == 3 ? 0x1b3e0d18u : i == 4 ? 0xc7b5f418u : i == 5 ? 0x73d13c71u
       : i == 6 ? 0xc8db33e9u : 0x6e2a5bb9u;
}
static constexpr uint32_t NPRIME = 0xffffffffu;  // -r^-1 mod 2^32 (r = 1 mod 2^32)

VL_HD Fr fr_zero() { Fr z; for (int i = 0; i < 8; i++) z.v[i] = 0; return z; }
VL_HD Fr fr_small(uint32_t x) { Fr z = fr_zero(); z.v[0] = x; return z; }
VL_HD Fr fr_r1() { Fr z; for (int i = 0; i < 8; i++) z.v[i] = r1_limb(i); return z; }
VL_HD Fr fr_r2() { Fr z; for (int i = 0; i < 8; i++) z.v[i] = r2_limb(i); return z; }
VL_HD Fr fr_r3() { Fr z; for (int i = 0; i < 8; i++) z.v[i] = r3_limb(i); return z; }

VL_HD bool fr_is_zero(const Fr& a) {
  uint32_t o = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) o |= a.v[i];
  return o == 0;
}

VL_HD bool fr_eq(const Fr& a, const Fr& b) {
  uint32_t o = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) o |= a.v[i] ^ b.v[i];
  return o == 0;
}

// t - r if t >= r else t  (t < 2^256 given as 8 limbs plus an overflow limb hi).
VL_HD void cond_sub_r(uint32_t t[8], uint32_t hi) {
  uint32_t d[8];
  uint64_t borrow = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    uint64_t x = (uint64_t)t[i] - r_limb(i) - borrow;
    d[i] = (uint32_t)x;
    borrow = (x >> 63) & 1;
  }
  // t >= r iff no borrow out of the 256-bit subtraction, or hi is set.
  bool take = (hi != 0) || (borrow == 0);
#pragma unroll
  for (int i = 0; i < 8; i++) t[i] = take ? d[i] : t[i];
}

VL_HD bool lt_r(const Fr& a) {
  uint64_t borrow = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    uint64_t x = (uint64_t)a.v[i] - r_limb(i) - borrow;
    borrow = (x >> 63) & 1;
  }
  return borrow != 0;
}

VL_HD Fr fr_add(const Fr& a, const Fr& b) {
  Fr s;
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    c += (uint64_t)a.v[i] + b.v[i];
    s.v[i] = (uint32_t)c;
    c >>= 32;
  }
  cond_sub_r(s.v, (uint32_t)c);
  return s;
}

VL_HD Fr fr_sub(const Fr& a, const Fr& b) {
  Fr d;
  uint64_t borrow = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    uint64_t x = (uint64_t)a.v[i] - b.v[i] - borrow;
    d.v[i] = (uint32_t)x;
    borrow = (x >> 63) & 1;
  }
  // Add r back when the subtraction wrapped.
  uint32_t mask = borrow ? 0xffffffffu : 0u;
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    c += (uint64_t)d.v[i] + (r_limb(i) & mask);
    d.v[i] = (uint32_t)c;
    c >>= 32;
  }
  return d;
}

VL_HD Fr fr_neg(const Fr& a) { return fr_sub(fr_zero(), a); }
VL_HD Fr fr_dbl(const Fr& a) { return fr_add(a, a); }

// Montgomery product a.b.R^-1 mod r (CIOS, 32-bit limbs).  Inputs a < 2^256,
// b < r; the output is reduced (< r).
VL_HD Fr mont_mul(const Fr& a, const Fr& b) {
  uint32_t t[10];
#pragma unroll
  for (int j = 0; j < 10; j++) t[j] = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      c += (uint64_t)a.v[j] * b.v[i] + t[j];
      t[j] = (uint32_t)c;
      c >>= 32;
    }
    c += t[8];
    t[8] = (uint32_t)c;
    t[9] = (uint32_t)(c >> 32);
    uint32_t m = t[0] * NPRIME;
    c = ((uint64_t)m * r_limb(0) + t[0]) >> 32;
#pragma unroll
    for (int j = 1; j < 8; j++) {
      c += (uint64_t)m * r_limb(j) + t[j];
      t[j - 1] = (uint32_t)c;
      c >>= 32;
    }
    c += t[8];
    t[7] = (uint32_t)c;
    t[8] = t[9] + (uint32_t)(c >> 32);
  }
  Fr out;
#pragma unroll
  for (int j = 0; j < 8; j++) out.v[j] = t[j];
  cond_sub_r(out.v, t[8]);
  return out;
}

VL_HD Fr to_mont(const Fr& a) { return mont_mul(a, fr_r2()); }
VL_HD Fr from_mont(const Fr& a) { return mont_mul(a, fr_small(1)); }

// Montgomery reduction of a wide value V = sum_l acc[l] . 2^(32 l) given as
// eight unsigned 64-bit column sums: returns V . R^-1 mod r (reduced).
// V < 2^289, so the REDC result is below 2r before the final subtraction.
VL_HD Fr redc_columns(const uint64_t acc[8]) {
  uint32_t t[18];
  uint64_t carry = 0;
#pragma unroll
  for (int l = 0; l < 8; l++) {
    uint64_t s = (acc[l] & 0xffffffffull) + carry;
    t[l] = (uint32_t)s;
    carry = (acc[l] >> 32) + (s >> 32);
  }
  t[8] = (uint32_t)carry;
  t[9] = (uint32_t)(carry >> 32);
#pragma unroll
  for (int j = 10; j < 18; j++) t[j] = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    uint32_t m = t[i] * NPRIME;
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      c += (uint64_t)m * r_limb(j) + t[i + j];
      t[i + j] = (uint32_t)c;
      c >>= 32;
    }
#pragma unroll
    for (int j = i + 8; j < 18; j++) {
      c += t[j];
      t[j] = (uint32_t)c;
      c >>= 32;
    }
  }
  Fr out;
#pragma unroll
  for (int j = 0; j < 8; j++) out.v[j] = t[8 + j];
  cond_sub_r(out.v, t[16]);
  return out;
}

// Reduce a 512-bit little-endian value (lo + hi.2^256) mod r; canonical out.
VL_HD Fr reduce_512(const Fr& lo, const Fr& hi) {
  // hi.2^256 = hi.R = mont_mul(hi, R^2) (valid for unreduced hi < 2^256).
  Fr h = mont_mul(hi, fr_r2());
  Fr l = lo;
  cond_sub_r(l.v, 0);
  cond_sub_r(l.v, 0);  // 2^256 < 3r: two subtractions reduce any 256-bit value
  return fr_add(l, h);
}

// Inverse of a canonical nonzero a (canonical result), by the binary
// extended Euclidean algorithm on (a, r): invariants x1.a = u and x2.a = v
// (mod r); halving keeps them (x/2 mod r = (x + r)/2 for odd x; x + r < 2^256
// since r < 2^255), subtracting the smaller of u, v from the larger shrinks
// them until one is 1.  Each step removes at least one bit of u or v, so at
// most 2 . 256 steps run; the cap only guards a zero input (returns 0).
VL_HD bool fr_is_one(const Fr& a) {
  uint32_t acc = a.v[0] ^ 1u;
  for (int i = 1; i < 8; i++) acc |= a.v[i];
  return acc == 0;
}
VL_HD void fr_half_mod(Fr& x) {  // x <- x / 2 mod r, x < r
  uint32_t carry = 0;
  if (x.v[0] & 1u) {
    uint64_t c = 0;
    for (int i = 0; i < 8; i++) {
      c += (uint64_t)x.v[i] + r_limb(i);
      x.v[i] = (uint32_t)c;
      c >>= 32;
    }
    carry = (uint32_t)c;  // always 0 (x + r < 2^256); kept for the shift
  }
  for (int i = 0; i < 7; i++) x.v[i] = (x.v[i] >> 1) | (x.v[i + 1] << 31);
  x.v[7] = (x.v[7] >> 1) | (carry << 31);
}
VL_HD bool fr_geq_raw(const Fr& a, const Fr& b) {
  for (int i = 7; i >= 0; i--)
    if (a.v[i] != b.v[i]) return a.v[i] > b.v[i];
  return true;
}
VL_HD Fr fr_sub_raw(const Fr& a, const Fr& b) {  // a - b for a >= b (integers)
  Fr d;
  uint64_t borrow = 0;
  for (int i = 0; i < 8; i++) {
    const uint64_t x = (uint64_t)a.v[i] - b.v[i] - borrow;
    d.v[i] = (uint32_t)x;
    borrow = (x >> 63) & 1u;
  }
  return d;
}
VL_HD Fr fr_inv_canonical(const Fr& a) {
  if (fr_is_zero(a)) return fr_zero();
  Fr u = a, v, x1 = fr_small(1), x2 = fr_zero();
  for (int i = 0; i < 8; i++) v.v[i] = r_limb(i);
  for (int step = 0; step < 4 * 256 && !fr_is_one(u) && !fr_is_one(v); step++) {
    while (!(u.v[0] & 1u)) {
      for (int i = 0; i < 7; i++) u.v[i] = (u.v[i] >> 1) | (u.v[i + 1] << 31);
      u.v[7] >>= 1;
      fr_half_mod(x1);
    }
    while (!(v.v[0] & 1u)) {
      for (int i = 0; i < 7; i++) v.v[i] = (v.v[i] >> 1) | (v.v[i + 1] << 31);
      v.v[7] >>= 1;
      fr_half_mod(x2);
    }
    if (fr_geq_raw(u, v)) {
      u = fr_sub_raw(u, v);
      x1 = fr_sub(x1, x2);
    } else {
      v = fr_sub_raw(v, u);
      x2 = fr_sub(x2, x1);
    }
  }
  return fr_is_one(u) ? x1 : x2;
}
// Inverse in Montgomery form (x.R -> x^-1.R): from_mont, canonical inverse, to_mont.
VL_HD Fr fr_inv_mont(const Fr& a) { return to_mont(fr_inv_canonical(from_mont(a))); }

// Signed integer x (|x| < 2^63) as a canonical field element.
VL_HD Fr fr_from_i64(int64_t x) {
  uint64_t mag = x < 0 ? (uint64_t)(-(x + 1)) + 1u : (uint64_t)x;
  Fr a = fr_zero();
  a.v[0] = (uint32_t)mag;
  a.v[1] = (uint32_t)(mag >> 32);
  return x < 0 ? fr_neg(a) : a;
}

}  // namespace vl
