// Claim and sumcheck rounds of each proof (Sec. II-B; Eq. eq:zk-mle-matmul).
//
// One CTA per proof.  The fold accumulators become the vectors
// f_A[w] = A~(u, w), f_B[w] = B~(w, v) over the padded cube w < 2^d1 (zeros
// for w >= k).  Round i (h = 2^(d1 - i)) evaluates the degree-2 round
// polynomial at 0, 1, 2:
//   g(0) = sum_j a0 b0,  g(1) = sum_j a1 b1,  g(2) = sum_j (2a1 - a0)(2b1 - b0)
// with a0 = f_A[j], a1 = f_A[j + h] (likewise b), absorbs the three values,
// squeezes r_i and folds both vectors in place, f[j] <- f[j] + r_i (f[j+h] - f[j])
// (variables bound most-significant first).  Finally a_r = f_A[0],
// b_r = f_B[0] are absorbed and the proof is written in canonical form.
//
// Schedule (latency is what matters here: one proof's rounds are a serial
// chain of hashes):
//  * pass 0 reduces the accumulators and evaluates round 1 in the same loop;
//    the claim is c = g_1(0) + g_1(1) (for k = 1 it is a_r . b_r);
//  * each later pass folds with r_i and evaluates round i + 1 on the folded
//    values in the same loop (one memory pass and one block reduction per
//    round);
//  * the transcript runs on warp 0 with message blocks in registers; the two
//    halves of the challenge and the closing state update are three
//    independent hashes done by three lanes at once.
#pragma once
#include "common.cuh"
#include "reduce.cuh"
#include "fr_dev.cuh"
#include "transcript_dev.cuh"

namespace vl {

// Shared memory the rounds need (RND_SMEM bytes): state (32), the round
// message (3 x 32), the challenge (32), then block-reduction slots for up to
// 8 warps (3 x 8 x 8 x 8 bytes at offset 256).
static_assert(RND_SMEM == 256 + 3 * 8 * 8 * 8, "layout");

__device__ __forceinline__ Fr load_acc_fr(const unsigned long long* acc, int w, const Fr& corr) {
  U64x8 a;
#pragma unroll
  for (int l = 0; l < 8; l++) a.v[l] = acc[(size_t)w * 8 + l];
  return fr_sub(redc_columns_ni(a), corr);
}

__device__ __forceinline__ void store_fr(vl_fr* dst, const Fr& x) {
#pragma unroll
  for (int l = 0; l < 8; l++) dst->limb[l] = x.v[l];
}

__device__ __forceinline__ Fr fold1(const Fr& x0, const Fr& x1, const Fr& r) {
  return fr_add(x0, mont_mul_ni(r, fr_sub(x1, x0)));
}

__device__ __forceinline__ void accum_g(Fr (&g)[3], const Fr& a0, const Fr& a1, const Fr& b0, const Fr& b1) {
  g[0] = fr_add(g[0], mont_mul_ni(a0, b0));
  g[1] = fr_add(g[1], mont_mul_ni(a1, b1));
  g[2] = fr_add(g[2], mont_mul_ni(fr_sub(fr_dbl(a1), a0), fr_sub(fr_dbl(b1), b0)));
}

// Warp 0: absorb the round message in gsh (lane 0), then squeeze one
// challenge: lanes 0 and 1 hash the two halves, lane 2 the state update.
// Returns r (Montgomery) in lane 0; S (shared) is the new state.
__device__ __forceinline__ Fr round_transcript(uint32_t* S, const Fr* gsh, bool with_claim, vl_proof* pf, int round) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    uint32_t st[8];
#pragma unroll
    for (int i = 0; i < 8; i++) st[i] = S[i];
    if (with_claim) {
      const Fr c[1] = {fr_add(gsh[0], gsh[1])};
      store_fr(&pf->c, c[0]);
      dev_absorb_fr<1>(st, LBL_C, c);
    }
#pragma unroll
    for (int q = 0; q < 3; q++) store_fr(&pf->g[round][q], gsh[q]);
    const Fr g02[2] = {gsh[0], gsh[2]};  // g(1) is fixed by the running claim
    dev_absorb_fr<2>(st, LBL_G, g02);
#pragma unroll
    for (int i = 0; i < 8; i++) S[i] = st[i];
  }
  __syncwarp();
  uint32_t st[8], d[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    st[i] = S[i];
    d[i] = 0;
  }
  if (lane < 3) dev_squeeze_block(st, LBL_R, lane < 2 ? 0u : 1u, lane, d);
  __syncwarp();
  if (lane == 2) {
#pragma unroll
    for (int i = 0; i < 8; i++) S[i] = d[i];
  }
  // r = (lo + hi . 2^256) mod r, in Montgomery form (lo: lane 0's digest,
  // hi: lane 1's) = lo . R + hi . R^2 mod r: lane 0 forms REDC(lo . R^2) and
  // lane 1 REDC(hi . R^3) at once, one product on the serial chain instead of
  // the reduction's and the conversion's two
  Fr half = fr_zero();
  if (lane < 2) half = mont_mul_ni(digest_le(d), lane == 0 ? fr_r2() : fr_r3());
  Fr other;
#pragma unroll
  for (int i = 0; i < 8; i++) other.v[i] = __shfl_sync(0xffffffffu, half.v[i], 1);
  Fr r = fr_zero();
  if (lane == 0) r = fr_add(half, other);
  __syncwarp();
  return r;
}

// Claim, rounds and proof of one proof by the whole block (any multiple of
// 32 threads up to 256), from round t0 on.  t0 = 1: everything.  t0 > 1: the
// earlier rounds ran batched over many proofs (kernels_rounds.cu): their
// messages are in the proof already, the transcript state and r_(t0-1) are
// in the scratch, and the vectors hold the round-(t0-1) values, 2^(d1-t0+2)
// entries each.
static __device__ void rounds_block(const DevProof& P, vl_proof* pf, uint8_t* smem, int t0 = 1) {
  uint32_t* S = reinterpret_cast<uint32_t*>(smem);
  Fr* gsh = reinterpret_cast<Fr*>(smem + 32);
  Fr& r_sh = gsh[3];
  unsigned long long* red = reinterpret_cast<unsigned long long*>(smem + 256);
  const int tid = threadIdx.x, warp = tid >> 5, nthr = blockDim.x;
  if (tid < 8) {
    const uint8_t* b = P.scr->state + 4 * tid;
    S[tid] = ((uint32_t)b[0] << 24) | ((uint32_t)b[1] << 16) | ((uint32_t)b[2] << 8) | (uint32_t)b[3];
  }
  if (t0 == 1) {
    if (tid == 0) {
      pf->m = P.m; pf->k = P.k; pf->n = P.n;
      pf->d0 = P.d0; pf->d1 = P.d1; pf->d2 = P.d2;
      pf->reserved = 0;
    }
    for (int i = P.d1 * 3 + tid; i < VL_MAX_ROUNDS * 3; i += nthr) store_fr(&pf->g[i / 3][i % 3], fr_zero());
  }
  const int d1 = P.d1, K = 1 << d1;
  const Fr corrA = P.scr->corrA, corrB = P.scr->corrB;
  Fr* fA = P.fA;
  Fr* fB = P.fB;
  __syncthreads();

  if (d1 == 0) {  // k = 1: no rounds, c = a_r . b_r
    if (tid == 0) {
      const Fr a = P.fdirA ? fA[0] : load_acc_fr(P.accA, 0, corrA);
      const Fr b = P.fdirB ? fB[0] : load_acc_fr(P.accB, 0, corrB);
      const Fr fin[2] = {from_mont_ni(a), from_mont_ni(b)};
      const Fr c[1] = {from_mont_ni(mont_mul_ni(a, b))};
      store_fr(&pf->c, c[0]);
      store_fr(&pf->a_r, fin[0]);
      store_fr(&pf->b_r, fin[1]);
      uint32_t st[8];
#pragma unroll
      for (int i = 0; i < 8; i++) st[i] = S[i];
      dev_absorb_fr<1>(st, LBL_C, c);
      dev_absorb_fr<2>(st, LBL_F, fin);
#pragma unroll
      for (int i = 0; i < 8; i++) {
        pf->state[4 * i] = (uint8_t)(st[i] >> 24);
        pf->state[4 * i + 1] = (uint8_t)(st[i] >> 16);
        pf->state[4 * i + 2] = (uint8_t)(st[i] >> 8);
        pf->state[4 * i + 3] = (uint8_t)st[i];
      }
      pf->status = P.scr->status;
    }
    __syncthreads();
    return;
  }

  Fr g[3] = {fr_zero(), fr_zero(), fr_zero()};
  if (t0 > 1) {
    // fold the round-(t0-1) vectors with r_(t0-1) and evaluate round t0
    const Fr r = P.scr->r;
    const int h = K >> (t0 - 1), hh = h >> 1;
    for (int j = tid; j < hh; j += nthr) {
      const Fr a0 = fold1(fA[j], fA[j + h], r), a1 = fold1(fA[j + hh], fA[j + hh + h], r);
      const Fr b0 = fold1(fB[j], fB[j + h], r), b1 = fold1(fB[j + hh], fB[j + hh + h], r);
      fA[j] = a0; fA[j + hh] = a1;
      fB[j] = b0; fB[j + hh] = b1;
      accum_g(g, a0, a1, b0, b1);
    }
  } else {
    // Pass 0: f from the accumulators, and round 1 (pairs j, j + K/2).
    const int h = K >> 1;
    for (int j = tid; j < h; j += nthr) {
      // K/2 < k <= K, so j < k always; j + h may be padding.
      // f_A, f_B come reduced from the fold (fdir) or as column sums to reduce here
      const Fr a0 = P.fdirA ? fA[j] : load_acc_fr(P.accA, j, corrA);
      const Fr b0 = P.fdirB ? fB[j] : load_acc_fr(P.accB, j, corrB);
      Fr a1 = fr_zero(), b1 = fr_zero();
      if (j + h < P.k) {
        a1 = P.fdirA ? fA[j + h] : load_acc_fr(P.accA, j + h, corrA);
        b1 = P.fdirB ? fB[j + h] : load_acc_fr(P.accB, j + h, corrB);
      }
      fA[j] = a0; fA[j + h] = a1;
      fB[j] = b0; fB[j + h] = b1;
      accum_g(g, a0, a1, b0, b1);
    }
  }
  block_sum_canonical<3>(g, gsh, red);

  for (int i = t0 - 1; i < d1; i++) {
    if (warp == 0) {
      const Fr r = round_transcript(S, gsh, i == 0, pf, i);
      if ((tid & 31) == 0) {
        r_sh = r;
        if (P.rch) P.rch[i] = r;  // chained proofs continue from this point
      }
    }
    __syncthreads();
    const Fr r = r_sh;
    const int h = K >> (i + 1);  // the vectors hold 2h entries
    if (i + 1 < d1) {
      // Fold with r_i and evaluate round i + 1 (pairs j, j + h/2) in one pass.
      const int hh = h >> 1;
      Fr gn[3] = {fr_zero(), fr_zero(), fr_zero()};
      if (4 * hh <= nthr) {
        // Few pairs (the last rounds, latency-bound): four lanes of one warp
        // per pair, one fold each, then three of them one term each (two
        // products on the chain instead of seven).
        const int j = tid >> 2, q = tid & 3;
        if (j < hh) {
          Fr* f = q < 2 ? fA : fB;
          const int at = j + (q & 1) * hh;
          f[at] = fold1(f[at], f[at + h], r);
        }
        __syncwarp();
        if (j < hh && q < 3) {
          const Fr a0 = fA[j], a1 = fA[j + hh], b0 = fB[j], b1 = fB[j + hh];
          if (q == 0) gn[0] = mont_mul_ni(a0, b0);
          else if (q == 1) gn[1] = mont_mul_ni(a1, b1);
          else gn[2] = mont_mul_ni(fr_sub(fr_dbl(a1), a0), fr_sub(fr_dbl(b1), b0));
        }
      } else {
        for (int j = tid; j < hh; j += nthr) {
          const Fr a0 = fold1(fA[j], fA[j + h], r), a1 = fold1(fA[j + hh], fA[j + hh + h], r);
          const Fr b0 = fold1(fB[j], fB[j + h], r), b1 = fold1(fB[j + hh], fB[j + hh + h], r);
          fA[j] = a0; fA[j + hh] = a1;
          fB[j] = b0; fB[j + hh] = b1;
          accum_g(gn, a0, a1, b0, b1);
        }
      }
      block_sum_canonical<3>(gn, gsh, red);
    } else if (tid == 0) {
      // Last fold: a_r, b_r; absorb them and write the proof.
      const Fr fin[2] = {from_mont_ni(fold1(fA[0], fA[1], r)), from_mont_ni(fold1(fB[0], fB[1], r))};
      store_fr(&pf->a_r, fin[0]);
      store_fr(&pf->b_r, fin[1]);
      uint32_t st[8];
#pragma unroll
      for (int q = 0; q < 8; q++) st[q] = S[q];
      dev_absorb_fr<2>(st, LBL_F, fin);
#pragma unroll
      for (int q = 0; q < 8; q++) {
        pf->state[4 * q] = (uint8_t)(st[q] >> 24);
        pf->state[4 * q + 1] = (uint8_t)(st[q] >> 16);
        pf->state[4 * q + 2] = (uint8_t)(st[q] >> 8);
        pf->state[4 * q + 3] = (uint8_t)st[q];
      }
      pf->status = P.scr->status;
    }
  }
  __syncthreads();
}

}  // namespace vl
