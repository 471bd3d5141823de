// Claim and sumcheck rounds of each proof (Sec. II-B; Eq. eq:zk-mle-matmul).
//
// One CTA per proof.  It first turns the fold accumulators into the vectors
// f_A[w] = A~(u, w), f_B[w] = B~(w, v) over the padded cube w < 2^d1 (zeros
// for w >= k), forms the claim c = sum_w f_A[w] f_B[w] and absorbs it.  Round
// i (h = 2^(d1 - i)) then evaluates the degree-2 round polynomial at 0, 1, 2:
//   g(0) = sum_j a0 b0,  g(1) = sum_j a1 b1,  g(2) = sum_j (2a1 - a0)(2b1 - b0)
// with a0 = f_A[j], a1 = f_A[j + h] (likewise b), absorbs the three values,
// squeezes r_i and folds both vectors in place, f[j] <- f[j] + r_i (f[j+h] - f[j])
// (variables bound most-significant first).  Finally a_r = f_A[0],
// b_r = f_B[0] are absorbed and the proof is written in canonical form.
#include "common.cuh"
#include "reduce.cuh"
#include "transcript.cuh"

namespace vl {

static constexpr int RND_THREADS = 128;

__device__ __forceinline__ Fr load_acc_fr(const unsigned long long* acc, int w, const Fr& corr) {
  uint64_t a[8];
#pragma unroll
  for (int l = 0; l < 8; l++) a[l] = acc[(size_t)w * 8 + l];
  return fr_sub(redc_columns(a), corr);
}

__device__ __forceinline__ void store_fr(vl_fr* dst, const Fr& x) {
#pragma unroll
  for (int l = 0; l < 8; l++) dst->limb[l] = x.v[l];
}

__global__ void __launch_bounds__(RND_THREADS, 7) rounds_kernel(const DevProof* __restrict__ proofs,
                                                             vl_proof* __restrict__ out) {
  const DevProof& P = proofs[blockIdx.x];
  vl_proof* pf = out + blockIdx.x;
  __shared__ uint8_t S[32];
  __shared__ Fr red[3 * (RND_THREADS / 32)];
  __shared__ Fr r_sh;
  const int tid = threadIdx.x;
  if (tid < 32) S[tid] = P.scr->state[tid];
  const int K = 1 << P.d1;
  const Fr corrA = P.scr->corrA, corrB = P.scr->corrB;
  Fr* fA = P.fA;
  Fr* fB = P.fB;

  Fr c[1] = {fr_zero()};
  for (int w = tid; w < K; w += RND_THREADS) {
    Fr a = fr_zero(), b = fr_zero();
    if (w < P.k) {
      a = load_acc_fr(P.accA, w, corrA);
      b = load_acc_fr(P.accB, w, corrB);
    }
    fA[w] = a;
    fB[w] = b;
    c[0] = fr_add(c[0], mont_mul(a, b));
  }
  block_sum_fr<1>(c, red);
  if (tid == 0) {
    pf->m = P.m; pf->k = P.k; pf->n = P.n;
    pf->d0 = P.d0; pf->d1 = P.d1; pf->d2 = P.d2;
    pf->reserved = 0;
    Fr cc = from_mont(c[0]);
    store_fr(&pf->c, cc);
    ts_absorb_fr(S, LBL_C, &cc, 1);
  }
  for (int i = P.d1 * 3 + tid; i < VL_MAX_ROUNDS * 3; i += RND_THREADS)
    store_fr(&pf->g[i / 3][i % 3], fr_zero());
  __syncthreads();

  for (int i = 0; i < P.d1; i++) {
    const int h = K >> (i + 1);
    Fr g[3] = {fr_zero(), fr_zero(), fr_zero()};
    for (int j = tid; j < h; j += RND_THREADS) {
      const Fr a0 = fA[j], a1 = fA[j + h], b0 = fB[j], b1 = fB[j + h];
      g[0] = fr_add(g[0], mont_mul(a0, b0));
      g[1] = fr_add(g[1], mont_mul(a1, b1));
      g[2] = fr_add(g[2], mont_mul(fr_sub(fr_dbl(a1), a0), fr_sub(fr_dbl(b1), b0)));
    }
    block_sum_fr<3>(g, red);
    if (tid == 0) {
      Fr gc[3] = {from_mont(g[0]), from_mont(g[1]), from_mont(g[2])};
      for (int q = 0; q < 3; q++) store_fr(&pf->g[i][q], gc[q]);
      ts_absorb_fr(S, LBL_G, gc, 3);
      Fr r = ts_challenge(S, LBL_R, 0);
      ts_squeeze_done(S, LBL_R, 1);
      r_sh = to_mont(r);
    }
    __syncthreads();
    const Fr r = r_sh;
    for (int j = tid; j < h; j += RND_THREADS) {
      const Fr a0 = fA[j], a1 = fA[j + h], b0 = fB[j], b1 = fB[j + h];
      fA[j] = fr_add(a0, mont_mul(r, fr_sub(a1, a0)));
      fB[j] = fr_add(b0, mont_mul(r, fr_sub(b1, b0)));
    }
    __syncthreads();
  }
  if (tid == 0) {
    Fr fin[2] = {from_mont(fA[0]), from_mont(fB[0])};
    store_fr(&pf->a_r, fin[0]);
    store_fr(&pf->b_r, fin[1]);
    ts_absorb_fr(S, LBL_F, fin, 2);
    for (int q = 0; q < 32; q++) pf->state[q] = S[q];
    pf->status = P.scr->status;
  }
}

cudaError_t launch_rounds(const DevProof* proofs, int nproofs, vl_proof* out, cudaStream_t st) {
  if (nproofs <= 0) return cudaSuccess;
  rounds_kernel<<<nproofs, RND_THREADS, 0, st>>>(proofs, out);
  return cudaGetLastError();
}

}  // namespace vl
