// Prologue of each proof: transcript start, the squeezes of u (d0 row
// challenges) and v (d2 column challenges), and the eq tables
//   E_u[i] = eq(u, bits(i)),  E_v[j] = eq(v, bits(j))
// of Eq. eq:MLE (Sec. II-B), written only for the real (unpadded) indices.
//
// eq(x, bits(i)) = prod_t (x_t if b_t else 1 - x_t), b_1 the MSB.  Split the d
// variables into a high block (first d - s) and a low block (last s): then
// E[i] = E_hi[i >> s] . E_lo[i mod 2^s], each factor table small enough for
// shared memory, and every output entry costs one Montgomery product.
// E_hi is kept in Montgomery form, E_lo in double-Montgomery form, so the
// product lands in double-Montgomery form (x.R^2), the weight format the
// int16 fold needs.  The kernel also writes 2^15 . sum_i E[i] (Montgomery),
// the correction for the +2^15 offset that the int16 fold applies.
#pragma once
#include "common.cuh"
#include "reduce.cuh"
#include "transcript.cuh"
#include "fr_dev.cuh"
#include "transcript_dev.cuh"

namespace vl {

static constexpr int MAX_VARS = 16;      // log2 of VL_MAX_REDUCE
static constexpr int MAX_HALF = 1 << 8;  // 2^(MAX_VARS / 2)

// Two fp16 values from bytes of w selected by `sel` (0x64bb is 1024 + bb).
__device__ __forceinline__ uint32_t pro_bytes_f16x2(uint32_t w, uint32_t sel) {
  const uint32_t v = __byte_perm(w, 0x64646464u, sel);
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(0x64006400u));
  return r;
}

// Entry i of the tensor-core weight table: the 32 bytes of e as fp16 values,
// at row i % 64 of its 4 KB chunk (MN-major core matrices: [i / 8 % 8][byte
// group][i % 8][8 bytes]).
__device__ __forceinline__ void store_w8(uint32_t* w8, int i, const Fr& e) {
  uint4* chunk = reinterpret_cast<uint4*>(w8) + (size_t)(i >> 6) * 256;
  const int kk = i & 63;
#pragma unroll
  for (int g = 0; g < 4; g++) {
    const uint32_t a = e.v[2 * g], b = e.v[2 * g + 1];
    chunk[(kk >> 3) * 32 + g * 8 + (kk & 7)] = make_uint4(pro_bytes_f16x2(a, 0x4140), pro_bytes_f16x2(a, 0x4342),
                                                          pro_bytes_f16x2(b, 0x4140), pro_bytes_f16x2(b, 0x4342));
  }
}

__device__ static Fr build_eq(const Fr* x, int d, int size, int tabs, Fr* out, uint32_t* out_soa, int pitch,
                              uint32_t* w8, Fr* lo, Fr* hi, Fr* red) {
  const int tid = threadIdx.x;
  const int s = (d + 1) >> 1;          // low-block variables
  const int dh = d - s;                // high-block variables
  const int nlo = 1 << s;
  const int nhi = (size + nlo - 1) >> s;
  for (int j = tid; j < nlo; j += blockDim.x) {
    Fr acc = fr_r2();  // 1 in double-Montgomery form
    for (int t = 0; t < s; t++) {
      const Fr& xt = x[dh + t];
      int b = (j >> (s - 1 - t)) & 1;
      acc = mont_mul_ni(acc, b ? xt : fr_sub(fr_r1(), xt));
    }
    lo[j] = acc;
  }
  for (int j = tid; j < nhi; j += blockDim.x) {
    Fr acc = fr_r1();  // 1 in Montgomery form
    for (int t = 0; t < dh; t++) {
      const Fr& xt = x[t];
      int b = (j >> (dh - 1 - t)) & 1;
      acc = mont_mul_ni(acc, b ? xt : fr_sub(fr_r1(), xt));
    }
    hi[j] = acc;
  }
  __syncthreads();
  Fr sum[1] = {fr_zero()};
  for (int i = tid; i < size; i += blockDim.x) {
    Fr e = mont_mul_ni(hi[i >> s], lo[i & (nlo - 1)]);
    if (tabs & TAB_LIMBS) {
      out[i] = e;
#pragma unroll
      for (int l = 0; l < 8; l++) out_soa[l * pitch + i] = e.v[l];
    }
    if (tabs & TAB_BYTES) store_w8(w8, i, e);
    sum[0] = fr_add(sum[0], e);
  }
  if (tabs & TAB_BYTES) {
    const int end = (size + 127) & ~127;  // whole 128-entry stages of the tensor-core fold
    for (int i = size + tid; i < end; i += blockDim.x) store_w8(w8, i, fr_zero());
  }
  block_sum_fr<1>(sum, red);
  // sum = sum_i E_i . R^2; one Montgomery product with the plain integer 2^15
  // gives 2^15 . sum_i E_i . R.
  return mont_mul_ni(sum[0], fr_small(1u << 15));
}

// Squeeze `count` challenges with `label` from the state Sw (big-endian
// words): thread 2t + h hashes half h of challenge t, thread 2 count the
// closing update.  Writes the challenges (Montgomery) to x and the new state
// to Sn.  Block-wide (two barriers).
__device__ static void squeeze_dev(const uint32_t* Sw, uint32_t label, int count, Fr* x, uint32_t* Sn,
                                   uint32_t (*dig)[8]) {
  const int tid = threadIdx.x;
  if (tid <= 2 * count) {
    uint32_t st[8], d[8];
#pragma unroll
    for (int i = 0; i < 8; i++) st[i] = Sw[i];
    if (tid < 2 * count) {
      dev_squeeze_block(st, label, (uint32_t)(tid >> 1), tid & 1, d);
#pragma unroll
      for (int i = 0; i < 8; i++) dig[tid][i] = d[i];
    } else {
      dev_squeeze_block(st, label, (uint32_t)count, 2, d);
#pragma unroll
      for (int i = 0; i < 8; i++) Sn[i] = d[i];
    }
  }
  __syncthreads();
  // challenge i = (lo + hi . 2^256) mod r in Montgomery form (lo = digest 2i,
  // hi = digest 2i + 1) = lo . R + hi . R^2: REDC(lo . R^2) and REDC(hi . R^3)
  // by two threads at once, then one addition
  Fr part;
  if (tid < 2 * count) part = mont_mul_ni(digest_le(dig[tid]), (tid & 1) ? fr_r3() : fr_r2());
  __syncthreads();
  if (tid < 2 * count) {
#pragma unroll
    for (int i = 0; i < 8; i++) dig[tid][i] = part.v[i];
  }
  __syncthreads();
  if (tid < count) {
    Fr lo, hi;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      lo.v[i] = dig[2 * tid][i];
      hi.v[i] = dig[2 * tid + 1][i];
    }
    x[tid] = fr_add(lo, hi);
  }
  __syncthreads();
}

// Transcript start and the squeezes of u, v into shared memory, or, for a
// proof with a given point, the given start state and point; the state after
// them goes to P.scr->state.  Block-wide.
__device__ static void start_or_given(const DevProof& P, uint32_t* S0, uint32_t* S1, uint32_t* S2,
                                      uint32_t (*dig)[8], Fr* u, Fr* v) {
  const int tid = threadIdx.x;
  if (P.given) {
    for (int i = tid; i < P.d0 + P.d2; i += blockDim.x) {
      if (i < P.d0) u[i] = P.given->u[i];
      else v[i - P.d0] = P.given->v[i - P.d0];
    }
    if (tid < 32) P.scr->state[tid] = P.given->state[tid];
    __syncthreads();
    return;
  }
  if (tid == 0) {
    uint8_t b[32];
    if (P.member1 > 0)
      ts_start_member(b, P.seed, (uint32_t)P.nmembers, (uint32_t)(P.member1 - 1), P.m, P.k, P.n, P.tp, P.tq, P.binds);
    else
      ts_start(b, P.seed, P.m, P.k, P.n, P.tp, P.tq, P.binds);
    for (int i = 0; i < 8; i++)
      S0[i] = ((uint32_t)b[4 * i] << 24) | ((uint32_t)b[4 * i + 1] << 16) | ((uint32_t)b[4 * i + 2] << 8) | b[4 * i + 3];
  }
  __syncthreads();
  squeeze_dev(S0, LBL_U, P.d0, u, S1, dig);
  squeeze_dev(S1, LBL_V, P.d2, v, S2, dig);
  if (tid < 32) P.scr->state[tid] = (uint8_t)(S2[tid >> 2] >> (24 - 8 * (tid & 3)));
}

// Shared memory the prologue needs (PRO_SMEM bytes), laid out below.
static_assert(PRO_SMEM == 128 + 2 * MAX_VARS * 32 + 2 * MAX_VARS * 32 + 2 * MAX_HALF * 32 + 8 * 32, "layout");

// Prologue of one proof by the whole block (any multiple of 32 threads, at
// least 64): transcript start, squeezes of u and v, eq tables, corrections.
static __device__ void prologue_block(const DevProof& P, uint8_t* smem) {
  uint32_t* S0 = reinterpret_cast<uint32_t*>(smem);
  uint32_t* S1 = S0 + 8;
  uint32_t* S2 = S0 + 16;
  uint32_t(*dig)[8] = reinterpret_cast<uint32_t(*)[8]>(smem + 128);
  Fr* u = reinterpret_cast<Fr*>(smem + 128 + 2 * MAX_VARS * 32);
  Fr* v = u + MAX_VARS;
  Fr* lo = v + MAX_VARS;
  Fr* hi = lo + MAX_HALF;
  Fr* red = hi + MAX_HALF;
  const int tid = threadIdx.x;

  start_or_given(P, S0, S1, S2, dig, u, v);

  Fr ca = build_eq(u, P.d0, P.m, P.tabA, P.eqA, P.eqA_soa, P.soa_pitchA, P.w8A, lo, hi, red);
  __syncthreads();
  Fr cb = build_eq(v, P.d2, P.n, P.tabB, P.eqB, P.eqB_soa, P.soa_pitchB, P.w8B, lo, hi, red);
  if (tid == 0) {
    P.scr->corrA = P.dtypeA == VL_I16 ? ca : fr_zero();
    P.scr->corrB = P.dtypeB == VL_I16 ? cb : fr_zero();
    P.scr->status = VL_OK;
  }
  __syncthreads();
}

// Factor tables of one side into global memory: lo[j] (2^s entries,
// double-Montgomery) and hi[j] (ceil(size / 2^s) entries, Montgomery), with
// E[i] = hi[i >> s] . lo[i mod 2^s] and s = ceil(d / 2).  Block-wide.
__device__ static void eq_factors(const Fr* x, int d, int size, Fr* lo, Fr* hi) {
  const int tid = threadIdx.x;
  const int s = (d + 1) >> 1, dh = d - s;
  const int nlo = 1 << s, nhi = (size + nlo - 1) >> s;
  for (int j = tid; j < nlo + nhi; j += blockDim.x) {
    const bool is_lo = j < nlo;
    const int jj = is_lo ? j : j - nlo, nv = is_lo ? s : dh, base = is_lo ? dh : 0;
    Fr acc = is_lo ? fr_r2() : fr_r1();
    for (int t = 0; t < nv; t++) {
      const Fr& xt = x[base + t];
      acc = mont_mul_ni(acc, ((jj >> (nv - 1 - t)) & 1) ? xt : fr_sub(fr_r1(), xt));
    }
    (is_lo ? lo : hi)[jj] = acc;
  }
}

// sum_{i < size} eq(x, bits(i)) (Montgomery), in closed form: i < size
// exactly when, at the first bit (from the top) where i and size differ, i
// has 0 and size has 1; the bits below are free and their eq factors sum to
// 1.  So the sum runs over the 1-bits t of size: prod of the factors of size's
// bits above t, times (1 - x_t).  O(d) products, one thread.
__device__ static Fr eq_prefix_sum(const Fr* x, int d, int size) {
  if (size >= (1 << d)) return fr_r1();  // the whole cube: sum 1
  Fr sum = fr_zero(), pre = fr_r1();
  for (int t = 0; t < d; t++) {
    const int b = (size >> (d - 1 - t)) & 1;
    const Fr one_minus = fr_sub(fr_r1(), x[t]);
    if (b) sum = fr_add(sum, mont_mul_ni(pre, one_minus));
    pre = mont_mul_ni(pre, b ? x[t] : one_minus);
  }
  return sum;
}

// First launch of the prologue, one proof per block (any multiple of 32
// threads, at least 64): transcript start, squeezes of u and v, the factor
// tables of both eq tables (to P.fac) and the offset corrections
// 2^15 . sum_i E[i] (Montgomery).
static __device__ void transcript_block(const DevProof& P, uint8_t* smem) {
  uint32_t* S0 = reinterpret_cast<uint32_t*>(smem);
  uint32_t* S1 = S0 + 8;
  uint32_t* S2 = S0 + 16;
  uint32_t(*dig)[8] = reinterpret_cast<uint32_t(*)[8]>(smem + 128);
  Fr* u = reinterpret_cast<Fr*>(smem + 128 + 2 * MAX_VARS * 32);
  Fr* v = u + MAX_VARS;
  const int tid = threadIdx.x;
  start_or_given(P, S0, S1, S2, dig, u, v);
  eq_factors(u, P.d0, P.m, P.fac, P.fac + EQ_FAC);
  eq_factors(v, P.d2, P.n, P.fac + 2 * EQ_FAC, P.fac + 3 * EQ_FAC);
  if (tid == 0 || tid == 32) {
    const bool a = tid == 0;
    const Fr sum = a ? eq_prefix_sum(u, P.d0, P.m) : eq_prefix_sum(v, P.d2, P.n);
    // sum . R times 2^15 . R, reduced once: 2^15 . sum (Montgomery)
    const Fr corr = mont_mul_ni(sum, to_mont_ni(fr_small(1u << 15)));
    const bool i16 = (a ? P.dtypeA : P.dtypeB) == VL_I16;
    (a ? P.scr->corrA : P.scr->corrB) = i16 ? corr : fr_zero();
  }
  if (tid == 0) P.scr->status = VL_OK;
  __syncthreads();
}

// Second launch: entries [i0, i1) of one eq table, E[i] = hi[i >> s] . lo[i
// mod 2^s] (double-Montgomery), written in the formats the side's fold
// engines read; tensor-core tables are zero from the last entry to their
// padded end.
static __device__ void eq_chunk(const EqItem& it, const DevProof& P) {
  const bool b = it.side != 0;
  const int d = b ? P.d2 : P.d0, size = b ? P.n : P.m, tabs = b ? P.tabB : P.tabA;
  const int s = (d + 1) >> 1, mask = (1 << s) - 1;
  const Fr* lo = P.fac + (b ? 2 * EQ_FAC : 0);
  const Fr* hi = lo + EQ_FAC;
  Fr* out = b ? P.eqB : P.eqA;
  uint32_t* soa = b ? P.eqB_soa : P.eqA_soa;
  const int pitch = b ? P.soa_pitchB : P.soa_pitchA;
  uint32_t* w8 = b ? P.w8B : P.w8A;
  for (int i = it.i0 + threadIdx.x; i < it.i1; i += blockDim.x) {
    const Fr e = i < size ? mont_mul_ni(hi[i >> s], lo[i & mask]) : fr_zero();
    if ((tabs & TAB_LIMBS) && i < size) {
      out[i] = e;
#pragma unroll
      for (int l = 0; l < 8; l++) soa[l * pitch + i] = e.v[l];
    }
    if (tabs & TAB_BYTES) store_w8(w8, i, e);
  }
}

}  // namespace vl
