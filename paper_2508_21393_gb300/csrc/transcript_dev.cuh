// Device transcript with the message blocks built in registers.
//
// Same transcript as transcript.cuh (start, absorb, counter-mode squeeze),
// specialised for the messages the device hashes: the state S is kept as
// the eight big-endian digest words, which are also the first eight message
// words of the next hash, so no byte buffer is needed.  The byte after S is
// the label; field elements follow as little-endian limbs, one byte out of
// word alignment, so message word 8 + i is (limb[i-1].byte3, limb[i].byte0,
// limb[i].byte1, limb[i].byte2) with the label standing in for byte 3 of
// limb[-1].  Every block is a fixed-index register array (no local memory).
#pragma once
#include <stdint.h>

#include "fr.cuh"
#include "sha256.cuh"
#include "transcript.cuh"

namespace vl {

__device__ __forceinline__ uint32_t rotr_dev(uint32_t x, int n) { return __funnelshift_r(x, x, n); }

struct ShaState {
  uint32_t h[8];
};
struct ShaBlock {
  uint32_t w[16];
};

// One SHA-256 compression, fully unrolled with the round constants as
// immediates, kept out of line (one copy per kernel module): the transcript
// is a serial chain of compressions, and an inlined copy at every call site
// makes the latency-bound kernels larger than the instruction cache.  h + K +
// W is formed off the e-chain, Ch and Maj use their two-operation forms.
static __device__ __noinline__ ShaState sha256_block_ni(ShaState st, ShaBlock m) {
  uint32_t a = st.h[0], b = st.h[1], c = st.h[2], d = st.h[3], e = st.h[4], f = st.h[5], g = st.h[6],
           h = st.h[7];
#pragma unroll
  for (int i = 0; i < 64; i++) {
    if (i >= 16) {
      const uint32_t x = m.w[(i - 15) & 15], y = m.w[(i - 2) & 15];
      m.w[i & 15] += (rotr_dev(x, 7) ^ rotr_dev(x, 18) ^ (x >> 3)) + m.w[(i - 7) & 15] +
                     (rotr_dev(y, 17) ^ rotr_dev(y, 19) ^ (y >> 10));
    }
    const uint32_t hkw = h + (sha_k(i) + m.w[i & 15]);
    const uint32_t s1 = rotr_dev(e, 6) ^ rotr_dev(e, 11) ^ rotr_dev(e, 25);
    const uint32_t ch = g ^ (e & (f ^ g));
    const uint32_t t1 = hkw + ch + s1;
    const uint32_t s0 = rotr_dev(a, 2) ^ rotr_dev(a, 13) ^ rotr_dev(a, 22);
    const uint32_t mj = (a & b) | (c & (a | b));
    h = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + (s0 + mj);
  }
  st.h[0] += a; st.h[1] += b; st.h[2] += c; st.h[3] += d;
  st.h[4] += e; st.h[5] += f; st.h[6] += g; st.h[7] += h;
  return st;
}

// One compression of a 16-word block into the chaining value st.
__device__ __forceinline__ void sha256_block(uint32_t st[8], const uint32_t blk[16]) {
  ShaState s;
  ShaBlock m;
#pragma unroll
  for (int i = 0; i < 8; i++) s.h[i] = st[i];
#pragma unroll
  for (int i = 0; i < 16; i++) m.w[i] = blk[i];
  s = sha256_block_ni(s, m);
#pragma unroll
  for (int i = 0; i < 8; i++) st[i] = s.h[i];
}

__device__ __forceinline__ void sha256_iv(uint32_t st[8]) {
  st[0] = 0x6a09e667u; st[1] = 0xbb67ae85u; st[2] = 0x3c6ef372u; st[3] = 0xa54ff53au;
  st[4] = 0x510e527fu; st[5] = 0x9b05688cu; st[6] = 0x1f83d9abu; st[7] = 0x5be0cd19u;
}

// S <- SHA256(S || label || x_0 || ... || x_{N-1}) for N canonical field elements.
// Message length 33 + 32N bytes; each 16-word block is built just before
// its compression (all indices are compile-time constants).
template <int N>
__device__ __forceinline__ void dev_absorb_fr(uint32_t S[8], uint32_t label, const Fr (&x)[N]) {
  constexpr int LEN = 33 + 32 * N;
  constexpr int NB = (LEN + 9 + 63) / 64;
  uint32_t st[8];
  sha256_iv(st);
#pragma unroll
  for (int b = 0; b < NB; b++) {
    uint32_t m[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
      const int gi = 16 * b + i;  // word index in the padded message
      uint32_t w = 0;
      if (gi < 8) {
        w = S[gi];
      } else if (gi < 8 + 8 * N) {
        const int q = gi - 8;
        const uint32_t cur = x[q / 8].v[q % 8];
        // the label sits where byte 3 of a previous limb would
        const uint32_t prev = q == 0 ? (label << 24) : x[(q - 1) / 8].v[(q - 1) % 8];
        w = __byte_perm(cur, prev, 0x7012);
      } else if (gi == 8 + 8 * N) {
        w = (x[N - 1].v[7] & 0xff000000u) | 0x00800000u;  // last data byte, then the 0x80 pad byte
      }
      if (gi == 16 * NB - 1) w = (uint32_t)LEN * 8u;
      m[i] = w;
    }
    sha256_block(st, m);
  }
#pragma unroll
  for (int i = 0; i < 8; i++) S[i] = st[i];
}

// One-block messages of a squeeze, from the state S before the squeeze:
//   kind 0/1: challenge t, half `kind`:  S || label || t u32le || kind   (38 bytes)
//   kind 2  : closing state update:      S || label || count u32le       (37 bytes)
// Returns the digest in out[8] (big-endian words).
__device__ __forceinline__ void dev_squeeze_block(const uint32_t S[8], uint32_t label, uint32_t t_or_count, int kind,
                                                  uint32_t out[8]) {
  uint32_t m[16];
#pragma unroll
  for (int i = 0; i < 8; i++) m[i] = S[i];
  const uint32_t v = t_or_count;
  // bytes 32..: label, v.b0, v.b1, v.b2 | v.b3, then (kind byte, 0x80) or 0x80
  m[8] = (label << 24) | ((v & 0xffu) << 16) | (((v >> 8) & 0xffu) << 8) | ((v >> 16) & 0xffu);
  if (kind == 2) {
    m[9] = ((v >> 24) << 24) | 0x00800000u;
    m[15] = 37u * 8u;
  } else {
    m[9] = ((v >> 24) << 24) | ((uint32_t)kind << 16) | 0x00008000u;
    m[15] = 38u * 8u;
  }
#pragma unroll
  for (int i = 10; i < 15; i++) m[i] = 0;
  sha256_iv(out);
  sha256_block(out, m);
}

// A 32-byte digest (big-endian words) read as a little-endian 256-bit integer.
__device__ __forceinline__ Fr digest_le(const uint32_t d[8]) {
  Fr x;
#pragma unroll
  for (int i = 0; i < 8; i++) x.v[i] = __byte_perm(d[i], 0, 0x0123);
  return x;
}

}  // namespace vl
