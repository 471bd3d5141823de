// Fiat-Shamir transcript over SHA-256 (host and device, one thread per call).
//
// The paper turns each verifier challenge into a hash of everything the
// prover sent before it (Sec. IV-A, footnote on Fiat-Shamir; Sec. V).  It
// fixes no byte format; this library's format is:
//   S0      = SHA256(DOMAIN || seed u64le || m,k,n u32le || transP,transQ u8
//                    || bindP || bindQ || bindC)            (binds: 32 B each)
//   absorb  : S <- SHA256(S || label || data)
//   squeeze : x_t = LE512(SHA256(S||label||t u32le||0x00) ||
//                         SHA256(S||label||t u32le||0x01)) mod r, t < count,
//             then S <- SHA256(S || label || count u32le)
// Field elements are serialised canonical, 32 bytes little-endian.  A
// sumcheck round absorbs g(0) || g(2): g(1) is fixed by the running claim.
// Squeezed challenges of one label depend only on the state before the
// squeeze, so they can be derived in parallel (one thread per t).
#pragma once
#include <stdint.h>

#include "fr.cuh"
#include "sha256.cuh"

namespace vl {

static constexpr uint8_t LBL_U = 'u', LBL_V = 'v', LBL_R = 'r';
static constexpr uint8_t LBL_C = 'c', LBL_G = 'g', LBL_F = 'f';

VL_HD void fr_to_le_bytes(const Fr& a, uint8_t out[32]) {
  for (int i = 0; i < 8; i++) {
    out[4 * i] = (uint8_t)a.v[i];
    out[4 * i + 1] = (uint8_t)(a.v[i] >> 8);
    out[4 * i + 2] = (uint8_t)(a.v[i] >> 16);
    out[4 * i + 3] = (uint8_t)(a.v[i] >> 24);
  }
}

VL_HD Fr fr_from_le_bytes(const uint8_t b[32]) {
  Fr a;
  for (int i = 0; i < 8; i++)
    a.v[i] = (uint32_t)b[4 * i] | ((uint32_t)b[4 * i + 1] << 8) |
             ((uint32_t)b[4 * i + 2] << 16) | ((uint32_t)b[4 * i + 3] << 24);
  return a;
}

VL_HD void ts_start(uint8_t S[32], uint64_t seed, uint32_t m, uint32_t k, uint32_t n,
                    uint32_t trans_p, uint32_t trans_q, const uint8_t binds[96]) {
  const uint8_t dom[23] = {'v', 'e', 'r', 'i', 'l', 'o', 'r', 'a', '-', 'g', 'b', '3',
                           '0', '0', '/', 'z', 'k', 'm', 'a', 't', '/', 'v', '1'};
  Sha256 h;
  h.init();
  h.update(dom, 23);
  h.u32le((uint32_t)seed);
  h.u32le((uint32_t)(seed >> 32));
  h.u32le(m);
  h.u32le(k);
  h.u32le(n);
  h.byte((uint8_t)(trans_p & 1));
  h.byte((uint8_t)(trans_q & 1));
  h.update(binds, 96);
  h.finish(S);
}

// Start of a linear zkMat transcript:
//   S0 = SHA256("verilora-gb300/zklin/v1" || seed u64le || rows, cols, q u32le
//               || coeffs (q x 32 B, canonical) || binds (q x 32 B))
VL_HD void ts_start_linear(uint8_t S[32], uint64_t seed, uint32_t rows, uint32_t cols, int q, const Fr* coeffs,
                           const uint8_t (*binds)[32]) {
  const uint8_t dom[23] = {'v', 'e', 'r', 'i', 'l', 'o', 'r', 'a', '-', 'g', 'b', '3',
                           '0', '0', '/', 'z', 'k', 'l', 'i', 'n', '/', 'v', '1'};
  Sha256 h;
  h.init();
  h.update(dom, 23);
  h.u32le((uint32_t)seed);
  h.u32le((uint32_t)(seed >> 32));
  h.u32le(rows);
  h.u32le(cols);
  h.u32le((uint32_t)q);
  for (int i = 0; i < q; i++) {
    uint8_t b[32];
    fr_to_le_bytes(coeffs[i], b);
    h.update(b, 32);
  }
  for (int i = 0; i < q; i++) h.update(binds[i], 32);
  h.finish(S);
}

// Member transcript of a product in a batched proof:
//   M_i = SHA256("verilora-gb300/zkbatch/v1/member" || seed u64le || K, i u32le
//                || m, k, n u32le || transP, transQ u8 || bindP || bindQ || bindC)
VL_HD void ts_start_member(uint8_t S[32], uint64_t seed, uint32_t K, uint32_t i, uint32_t m, uint32_t k, uint32_t n,
                           uint32_t trans_p, uint32_t trans_q, const uint8_t binds[96]) {
  const uint8_t dom[32] = {'v', 'e', 'r', 'i', 'l', 'o', 'r', 'a', '-', 'g', 'b', '3', '0', '0', '/', 'z',
                           'k', 'b', 'a', 't', 'c', 'h', '/', 'v', '1', '/', 'm', 'e', 'm', 'b', 'e', 'r'};
  Sha256 h;
  h.init();
  h.update(dom, 32);
  h.u32le((uint32_t)seed);
  h.u32le((uint32_t)(seed >> 32));
  h.u32le(K);
  h.u32le(i);
  h.u32le(m);
  h.u32le(k);
  h.u32le(n);
  h.byte((uint8_t)(trans_p & 1));
  h.byte((uint8_t)(trans_q & 1));
  h.update(binds, 96);
  h.finish(S);
}

// Batch transcript start: SHA256("verilora-gb300/zkbatch/v1" || seed u64le || K u32le || root)
VL_HD void ts_start_batch(uint8_t S[32], uint64_t seed, uint32_t K, const uint8_t root[32]) {
  const uint8_t dom[25] = {'v', 'e', 'r', 'i', 'l', 'o', 'r', 'a', '-', 'g', 'b', '3', '0',
                           '0', '/', 'z', 'k', 'b', 'a', 't', 'c', 'h', '/', 'v', '1'};
  Sha256 h;
  h.init();
  h.update(dom, 25);
  h.u32le((uint32_t)seed);
  h.u32le((uint32_t)(seed >> 32));
  h.u32le(K);
  h.update(root, 32);
  h.finish(S);
}

// Merkle nodes: leaf = SHA256(0x00 || data), node = SHA256(0x01 || left || right).
VL_HD void merkle_node(uint8_t out[32], const uint8_t left[32], const uint8_t right[32]) {
  Sha256 h;
  h.init();
  h.byte(1);
  h.update(left, 32);
  h.update(right, 32);
  h.finish(out);
}

// Start of a lookup transcript:
//   S0 = SHA256("verilora-gb300/zklookup/v1" || seed u64le || n, log2 D, log2 N u32le
//               || t0 i64le || bind (32 B))
VL_HD void ts_start_lookup(uint8_t S[32], uint64_t seed, uint32_t n, uint32_t log2_d, uint32_t log2_n, int64_t t0,
                           const uint8_t bind[32]) {
  const uint8_t dom[26] = {'v', 'e', 'r', 'i', 'l', 'o', 'r', 'a', '-', 'g', 'b', '3', '0',
                           '0', '/', 'z', 'k', 'l', 'o', 'o', 'k', 'u', 'p', '/', 'v', '1'};
  Sha256 h;
  h.init();
  h.update(dom, 26);
  h.u32le((uint32_t)seed);
  h.u32le((uint32_t)(seed >> 32));
  h.u32le(n);
  h.u32le(log2_d);
  h.u32le(log2_n);
  const uint64_t tb = (uint64_t)t0;
  h.u32le((uint32_t)tb);
  h.u32le((uint32_t)(tb >> 32));
  h.update(bind, 32);
  h.finish(S);
}

// absorb(label, canonical field elements)
VL_HD void ts_absorb_fr(uint8_t S[32], uint8_t label, const Fr* vals, int count) {
  Sha256 h;
  h.init();
  h.update(S, 32);
  h.byte(label);
  for (int i = 0; i < count; i++) {
    uint8_t b[32];
    fr_to_le_bytes(vals[i], b);
    h.update(b, 32);
  }
  h.finish(S);
}

// Challenge t of a squeeze with this label, from the state before the squeeze.
VL_HD Fr ts_challenge(const uint8_t S[32], uint8_t label, uint32_t t) {
  uint8_t d0[32], d1[32];
  Sha256 h;
  h.init();
  h.update(S, 32);
  h.byte(label);
  h.u32le(t);
  h.byte(0);
  h.finish(d0);
  h.init();
  h.update(S, 32);
  h.byte(label);
  h.u32le(t);
  h.byte(1);
  h.finish(d1);
  return reduce_512(fr_from_le_bytes(d0), fr_from_le_bytes(d1));
}

// State update that closes a squeeze of `count` challenges.
VL_HD void ts_squeeze_done(uint8_t S[32], uint8_t label, uint32_t count) {
  Sha256 h;
  h.init();
  h.update(S, 32);
  h.byte(label);
  h.u32le(count);
  h.finish(S);
}

}  // namespace vl
