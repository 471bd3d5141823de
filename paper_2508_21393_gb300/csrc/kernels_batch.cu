// Batched-claim matmul sumcheck (Sec. IV, composition of proving steps by
// random aggregation of claims under one Fiat-Shamir transcript).
//
// The products' prologues (member transcripts, eq tables) and folds are the
// single-proof kernels; then:
//   claims  (one CTA per product): c_i = sum_w f_A[w] f_B[w], its Merkle leaf
//           SHA256(0x00 || S_i || c_i);
//   start   (one CTA): the Merkle root, the batch transcript start, rho, the
//           weights rho^i, the combined claim sum_i rho^i c_i;
//   rounds  per variable: a pass over every product's pairs (fold with the
//           previous challenge, then rho^i-weighted sums of g(0), g(2)) and
//           one CTA for the transcript step (g(1) = claim - g(0));
//   finish  (one CTA per product) a_i, b_i and their leaves; (one CTA) the
//           root, absorb 'f', the proof.
#include "prologue_dev.cuh"
#include "rounds_dev.cuh"

namespace vl {

namespace {

constexpr int BT_THREADS = 256;
constexpr uint8_t LBL_P = 'p';

// f_A[w] (side 0) or f_B[w] (side 1) of the unfolded vectors; 0 past k.
__device__ __forceinline__ Fr bt_level0(const DevProof& P, int side, int w) {
  if (w >= P.k) return fr_zero();
  if (side == 0) return P.fdirA ? P.fA[w] : load_acc_fr(P.accA, w, P.scr->corrA);
  return P.fdirB ? P.fB[w] : load_acc_fr(P.accB, w, P.scr->corrB);
}

__device__ __forceinline__ void bt_bytes(uint8_t out[32], const Fr& canonical) { fr_to_le_bytes(canonical, out); }

// One block per product.
__global__ void __launch_bounds__(BT_THREADS) bt_claims_kernel(const DevProof* dp, BtState* B) {
  __shared__ Fr red[BT_THREADS / 32];
  const DevProof& P = dp[blockIdx.x];
  const int i = P.member1 - 1;
  Fr acc[1] = {fr_zero()};
  for (int w = threadIdx.x; w < P.k; w += blockDim.x)
    acc[0] = fr_add(acc[0], mont_mul_ni(bt_level0(P, 0, w), bt_level0(P, 1, w)));
  block_sum_fr<1>(acc, red);
  if (threadIdx.x == 0) {
    B->c[i] = acc[0];
    const Fr c = from_mont_ni(acc[0]);
    for (int l = 0; l < 8; l++) B->c_out[i].limb[l] = c.v[l];
    uint8_t cb[32];
    bt_bytes(cb, c);
    Sha256 h;
    h.init();
    h.byte(0);
    h.update(P.scr->state, 32);
    h.update(cb, 32);
    h.finish(B->tree + (size_t)(B->P2 + i) * 32);
    if (P.scr->status != VL_OK) atomicExch(&B->status, P.scr->status);
  }
}

// Root of the Merkle tree whose K leaves are in place (block-wide): zero
// padding leaves, then the levels bottom up.
__device__ void bt_tree(BtState* B) {
  uint8_t* t = B->tree;
  for (int i = B->K + threadIdx.x; i < B->P2; i += blockDim.x)
    for (int b = 0; b < 32; b++) t[(size_t)(B->P2 + i) * 32 + b] = 0;
  __syncthreads();
  for (int lvl = B->P2 >> 1; lvl >= 1; lvl >>= 1) {
    for (int j = lvl + threadIdx.x; j < 2 * lvl; j += blockDim.x)
      merkle_node(t + (size_t)j * 32, t + (size_t)(2 * j) * 32, t + (size_t)(2 * j + 1) * 32);
    __syncthreads();
  }
}

// One block: batch start, rho, weights, combined claim.
__global__ void __launch_bounds__(BT_THREADS) bt_start_kernel(BtState* B) {
  __shared__ uint32_t S0[8], S1[8];
  __shared__ uint32_t dig[3][8];
  __shared__ Fr ch[1];
  __shared__ Fr red[BT_THREADS / 32];
  bt_tree(B);
  if (threadIdx.x == 0) {
    uint8_t b[32];
    ts_start_batch(b, B->seed, (uint32_t)B->K, B->tree + 32);
    for (int i = 0; i < 8; i++)
      S0[i] = ((uint32_t)b[4 * i] << 24) | ((uint32_t)b[4 * i + 1] << 16) | ((uint32_t)b[4 * i + 2] << 8) | b[4 * i + 3];
  }
  __syncthreads();
  squeeze_dev(S0, LBL_P, 1, ch, S1, dig);
  const Fr rho = ch[0];
  Fr acc[1] = {fr_zero()};
  for (int i = threadIdx.x; i < B->K; i += blockDim.x) {
    Fr w = fr_r1(), base = rho;  // rho^i by squaring
    for (int e = i; e; e >>= 1) {
      if (e & 1) w = mont_mul_ni(w, base);
      base = mont_mul_ni(base, base);
    }
    B->w[i] = w;
    acc[0] = fr_add(acc[0], mont_mul_ni(w, B->c[i]));
  }
  block_sum_fr<1>(acc, red);
  if (threadIdx.x == 0) {
    B->rho = rho;
    B->claim = acc[0];
    for (int i = 0; i < 8; i++) B->St[i] = S1[i];
  }
}

// Round t over pairs [k0, k1) of one product (item.proof = its DevProof
// index): fold with r_{t-1} (the first round reads the unfolded vectors, the
// second folds them into fA/fB, later rounds fold in place), then the
// rho^i-weighted sums of a0 b0 and (2a1 - a0)(2b1 - b0).
__global__ void __launch_bounds__(BT_THREADS) bt_pass_kernel(const DevProof* dp, BtState* B, int t,
                                                              const LkItem* items) {
  __shared__ Fr red[2 * (BT_THREADS / 32)];
  const LkItem it = items[blockIdx.x];
  const DevProof& P = dp[it.proof];
  const int h = 1 << (B->d1 - t);
  Fr acc[2] = {fr_zero(), fr_zero()};
  for (int j = it.k0 + threadIdx.x; j < it.k1; j += blockDim.x) {
    Fr a0, a1, b0, b1;
    if (t == 1) {
      a0 = bt_level0(P, 0, j), a1 = bt_level0(P, 0, j + h);
      b0 = bt_level0(P, 1, j), b1 = bt_level0(P, 1, j + h);
    } else if (t == 2) {
      const Fr r = B->r[0];
      a0 = fold1(bt_level0(P, 0, j), bt_level0(P, 0, j + 2 * h), r);
      a1 = fold1(bt_level0(P, 0, j + h), bt_level0(P, 0, j + 3 * h), r);
      b0 = fold1(bt_level0(P, 1, j), bt_level0(P, 1, j + 2 * h), r);
      b1 = fold1(bt_level0(P, 1, j + h), bt_level0(P, 1, j + 3 * h), r);
      P.fA[j] = a0, P.fA[j + h] = a1, P.fB[j] = b0, P.fB[j + h] = b1;
    } else {
      const Fr r = B->r[t - 2];
      a0 = fold1(P.fA[j], P.fA[j + 2 * h], r);
      a1 = fold1(P.fA[j + h], P.fA[j + 3 * h], r);
      b0 = fold1(P.fB[j], P.fB[j + 2 * h], r);
      b1 = fold1(P.fB[j + h], P.fB[j + 3 * h], r);
      P.fA[j] = a0, P.fA[j + h] = a1, P.fB[j] = b0, P.fB[j + h] = b1;
    }
    acc[0] = fr_add(acc[0], mont_mul_ni(a0, b0));
    acc[1] = fr_add(acc[1], mont_mul_ni(fr_sub(fr_dbl(a1), a0), fr_sub(fr_dbl(b1), b0)));
  }
  block_sum_fr<2>(acc, red);
  if (threadIdx.x == 0) {
    const Fr w = B->w[P.member1 - 1];
    B->part[(size_t)it.slot * 2] = mont_mul_ni(w, acc[0]);
    B->part[(size_t)it.slot * 2 + 1] = mont_mul_ni(w, acc[1]);
  }
}

// One block: round t's polynomial from the partial sums, its values in the
// proof, absorb, squeeze r_t, new claim.
__global__ void __launch_bounds__(BT_THREADS) bt_round_kernel(BtState* B, int t) {
  __shared__ Fr red[2 * (BT_THREADS / 32)];
  __shared__ uint32_t Sw[8], Sn[8];
  __shared__ uint32_t dig[3][8];
  __shared__ Fr ch[1];
  __shared__ Fr gsh[3];
  Fr acc[2] = {fr_zero(), fr_zero()};
  for (int s = B->pbeg[t] + threadIdx.x; s < B->pend[t]; s += blockDim.x) {
    acc[0] = fr_add(acc[0], B->part[(size_t)s * 2]);
    acc[1] = fr_add(acc[1], B->part[(size_t)s * 2 + 1]);
  }
  block_sum_fr<2>(acc, red);
  if (threadIdx.x == 0) {
    const Fr g[3] = {acc[0], fr_sub(B->claim, acc[0]), acc[1]};
    Fr gc[3];
    for (int q = 0; q < 3; q++) {
      gsh[q] = g[q];
      gc[q] = from_mont_ni(g[q]);
      for (int l = 0; l < 8; l++) B->out->g[t - 1][q].limb[l] = gc[q].v[l];
    }
    uint32_t S[8];
    for (int i = 0; i < 8; i++) S[i] = B->St[i];
    const Fr m2[2] = {gc[0], gc[2]};
    dev_absorb_fr<2>(S, LBL_G, m2);
    for (int i = 0; i < 8; i++) Sw[i] = S[i];
  }
  __syncthreads();
  squeeze_dev(Sw, LBL_R, 1, ch, Sn, dig);
  if (threadIdx.x == 0) {
    const Fr r = ch[0];
    B->r[t - 1] = r;
    for (int i = 0; i < 8; i++) B->St[i] = Sn[i];
    // g(r) through (0, g0), (1, g1), (2, g2): g0 (r-1)(r-2)/2 - g1 r(r-2) + g2 r(r-1)/2
    const Fr one = fr_r1(), two = fr_add(one, one);
    const Fr r1 = fr_sub(r, one), r2 = fr_sub(r, two);
    const Fr l0 = mont_mul_ni(mont_mul_ni(r1, r2), B->inv2);
    const Fr l1 = fr_neg(mont_mul_ni(r, r2));
    const Fr l2 = mont_mul_ni(mont_mul_ni(r, r1), B->inv2);
    B->claim = fr_add(fr_add(mont_mul_ni(gsh[0], l0), mont_mul_ni(gsh[1], l1)), mont_mul_ni(gsh[2], l2));
  }
}

// One warp per product: a_i, b_i (the last pair folded with r_d1), their
// canonical outputs and Merkle leaf.
__global__ void __launch_bounds__(32) bt_final_kernel(const DevProof* dp, BtState* B) {
  if (threadIdx.x != 0) return;
  const DevProof& P = dp[blockIdx.x];
  const int i = P.member1 - 1, d1 = B->d1;
  Fr a, b;
  if (d1 == 0) {
    a = bt_level0(P, 0, 0);
    b = bt_level0(P, 1, 0);
  } else if (d1 == 1) {
    a = fold1(bt_level0(P, 0, 0), bt_level0(P, 0, 1), B->r[0]);
    b = fold1(bt_level0(P, 1, 0), bt_level0(P, 1, 1), B->r[0]);
  } else {
    a = fold1(P.fA[0], P.fA[1], B->r[d1 - 1]);
    b = fold1(P.fB[0], P.fB[1], B->r[d1 - 1]);
  }
  const Fr ac = from_mont_ni(a), bc = from_mont_ni(b);
  for (int l = 0; l < 8; l++) {
    B->a_out[i].limb[l] = ac.v[l];
    B->b_out[i].limb[l] = bc.v[l];
  }
  uint8_t ab[32], bb[32];
  bt_bytes(ab, ac);
  bt_bytes(bb, bc);
  Sha256 h;
  h.init();
  h.byte(0);
  h.u32le((uint32_t)i);
  h.update(ab, 32);
  h.update(bb, 32);
  h.finish(B->tree + (size_t)(B->P2 + i) * 32);
}

// One block: the root of the final values, absorb 'f', the proof.
__global__ void __launch_bounds__(BT_THREADS) bt_close_kernel(BtState* B, int k) {
  bt_tree(B);
  if (threadIdx.x != 0) return;
  uint8_t S[32];
  for (int i = 0; i < 32; i++) S[i] = (uint8_t)(B->St[i >> 2] >> (24 - 8 * (i & 3)));
  Sha256 h;
  h.init();
  h.update(S, 32);
  h.byte(LBL_F);
  h.update(B->tree + 32, 32);
  h.finish(S);
  vl_batch_proof* out = B->out;
  for (int i = 0; i < 32; i++) out->state[i] = S[i];
  for (int t = B->d1; t < VL_MAX_ROUNDS; t++)
    for (int q = 0; q < 3; q++)
      for (int l = 0; l < 8; l++) out->g[t][q].limb[l] = 0u;
  out->K = B->K;
  out->k = k;
  out->d1 = B->d1;
  out->status = B->status;
}

}  // namespace

cudaError_t launch_batch_claims(const DevProof* dp, int np, BtState* B, cudaStream_t st) {
  bt_claims_kernel<<<np, BT_THREADS, 0, st>>>(dp, B);
  bt_start_kernel<<<1, BT_THREADS, 0, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_batch_round(const DevProof* dp, BtState* B, int t, const LkItem* items, int nitems,
                               cudaStream_t st) {
  if (nitems) bt_pass_kernel<<<nitems, BT_THREADS, 0, st>>>(dp, B, t, items);
  bt_round_kernel<<<1, BT_THREADS, 0, st>>>(B, t);
  return cudaGetLastError();
}

cudaError_t launch_batch_finish(const DevProof* dp, int np, BtState* B, int k, cudaStream_t st) {
  bt_final_kernel<<<np, 32, 0, st>>>(dp, B);
  bt_close_kernel<<<1, BT_THREADS, 0, st>>>(B, k);
  return cudaGetLastError();
}

}  // namespace vl
