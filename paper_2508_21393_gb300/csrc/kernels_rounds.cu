// Rounds kernel: one CTA per proof (see rounds_dev.cuh).
#include <atomic>

#include "rounds_dev.cuh"

namespace vl {

template <int MINB, int THREADS>
__global__ void __launch_bounds__(THREADS, MINB) rounds_kernel(const DevProof* __restrict__ proofs,
                                                               vl_proof* __restrict__ out) {
  extern __shared__ __align__(128) uint8_t rnd_smem[];
  const DevProof& P = proofs[blockIdx.x];
  rounds_block(P, out + P.job, rnd_smem);
}

// variant: CTAs per SM.  7, 6, 5 and 4 set the register allocation (7: one
// wave of 1064 proofs, tighter registers; 4: more registers per thread).  3 and 2
// use the variant-4 code and cap residency by reserving shared memory, for
// fewer co-resident proofs competing for issue slots.  threads: 128, 192 or
// 256 per proof (more threads shorten the vector passes of large proofs; the
// register budget follows from variant x threads).
cudaError_t launch_rounds(const DevProof* proofs, int nproofs, vl_proof* out, int variant, int threads,
                          cudaStream_t st) {
  if (nproofs <= 0) return cudaSuccess;
  if (threads == 192) {
    rounds_kernel<4, 192><<<nproofs, 192, RND_SMEM, st>>>(proofs, out);
  } else if (threads == 256) {
    rounds_kernel<3, 256><<<nproofs, 256, RND_SMEM, st>>>(proofs, out);
  } else if (variant == 2 || variant == 3) {
    static std::atomic<int> set{0};  // launches come from several host threads
    const int smem = variant == 2 ? 100 * 1024 : 70 * 1024;
    if (set.load(std::memory_order_acquire) < smem) {
      cudaError_t e =
          cudaFuncSetAttribute(rounds_kernel<4, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
      if (e != cudaSuccess) return e;
      set.store(100 * 1024, std::memory_order_release);
    }
    rounds_kernel<4, 128><<<nproofs, 128, smem, st>>>(proofs, out);
  } else if (variant == 4) {
    rounds_kernel<4, 128><<<nproofs, 128, RND_SMEM, st>>>(proofs, out);
  } else if (variant == 5) {
    rounds_kernel<5, 128><<<nproofs, 128, RND_SMEM, st>>>(proofs, out);
  } else if (variant == 6) {
    rounds_kernel<6, 128><<<nproofs, 128, RND_SMEM, st>>>(proofs, out);
  } else {
    rounds_kernel<7, 128><<<nproofs, 128, RND_SMEM, st>>>(proofs, out);
  }
  return cudaGetLastError();
}

}  // namespace vl

// ----------------------------------------------------------- batched rounds --
//
// The same claim and rounds as rounds_block, with the heavy first rounds
// organised by round instead of by proof: while a proof's round has more
// than RB_TAIL pairs, the round's vector work (fold with the previous
// challenge, evaluation of g(0), g(1), g(2)) for all such proofs is one launch
// of many CTAs, each on a range of one proof's pairs, and the round's
// transcript step is one launch with one warp per proof.  The first rounds'
// vector work (three quarters of a proof's) then spreads over the whole GPU
// instead of one CTA per proof; the rounds after that, short vector passes
// between serial hashes, run as before, one CTA per proof (rounds_block from
// the proof's first unbatched round), in one launch.

namespace vl {
namespace {

// accum_g and fold1 of the batched passes (the one out-of-line copy of the
// Montgomery product: an inlined copy per call made the kernel larger than
// the instruction cache).
__device__ __forceinline__ void accum_g_inl(Fr (&g)[3], const Fr& a0, const Fr& a1, const Fr& b0, const Fr& b1) {
  const Fr p0 = mont_mul_ni(a0, b0), p1 = mont_mul_ni(a1, b1);
  const Fr p2 = mont_mul_ni(fr_sub(fr_dbl(a1), a0), fr_sub(fr_dbl(b1), b0));
  g[0] = fr_add(g[0], p0);
  g[1] = fr_add(g[1], p1);
  g[2] = fr_add(g[2], p2);
}

__device__ __forceinline__ Fr fold1_inl(const Fr& x0, const Fr& x1, const Fr& r) {
  return fr_add(x0, mont_mul_ni(r, fr_sub(x1, x0)));
}

__global__ void __launch_bounds__(RB_THREADS, 4) rounds_pass_kernel(const DevProof* __restrict__ proofs,
                                                                    const RoundItem* __restrict__ items,
                                                                    Fr* __restrict__ partials, int t) {
  __shared__ Fr gsh[4];
  __shared__ unsigned long long red[3 * 8 * (RB_THREADS / 32)];
  const RoundItem it = items[blockIdx.x];
  const DevProof& P = proofs[it.proof];
  const int tid = threadIdx.x, K = 1 << P.d1;
  Fr* fA = P.fA;
  Fr* fB = P.fB;
  Fr g[3] = {fr_zero(), fr_zero(), fr_zero()};
  if (t == 1) {
    // f from the fold (reduced, or column sums to reduce here), round 1 on
    // pairs (j, j + K/2); j + K/2 may be padding (written as zeros)
    const int h = K >> 1;
    const bool da = P.fdirA, db = P.fdirB;
    const Fr corrA = P.scr->corrA, corrB = P.scr->corrB;
    for (int j = it.j0 + tid; j < it.j1; j += RB_THREADS) {
      const Fr a0 = da ? fA[j] : load_acc_fr(P.accA, j, corrA);
      const Fr b0 = db ? fB[j] : load_acc_fr(P.accB, j, corrB);
      const bool real = j + h < P.k;
      Fr a1 = fr_zero(), b1 = fr_zero();
      if (real) {
        a1 = da ? fA[j + h] : load_acc_fr(P.accA, j + h, corrA);
        b1 = db ? fB[j + h] : load_acc_fr(P.accB, j + h, corrB);
      }
      if (!da) fA[j] = a0;
      if (!da || !real) fA[j + h] = a1;
      if (!db) fB[j] = b0;
      if (!db || !real) fB[j + h] = b1;
      accum_g_inl(g, a0, a1, b0, b1);
    }
  } else {
    // fold with r_(t-1) (vectors of 2h entries) and evaluate round t on the
    // folded pairs (j, j + hh)
    const Fr r = P.scr->r;
    const int h = K >> (t - 1), hh = h >> 1;
    for (int j = it.j0 + tid; j < it.j1; j += RB_THREADS) {
      const Fr a0 = fold1_inl(fA[j], fA[j + h], r), a1 = fold1_inl(fA[j + hh], fA[j + hh + h], r);
      const Fr b0 = fold1_inl(fB[j], fB[j + h], r), b1 = fold1_inl(fB[j + hh], fB[j + hh + h], r);
      fA[j] = a0; fA[j + hh] = a1;
      fB[j] = b0; fB[j + hh] = b1;
      accum_g_inl(g, a0, a1, b0, b1);
    }
  }
  block_sum_canonical<3>(g, gsh, red);
  if (tid < 3) partials[3 * (size_t)blockIdx.x + tid] = gsh[tid];
}

__device__ __forceinline__ void state_to_bytes(const uint32_t* S, uint8_t* out, int lane) {
  out[lane] = (uint8_t)(S[lane >> 2] >> (24 - 8 * (lane & 3)));
}

// Transcript step of round t for proofs [0, np) (each has more rounds after
// t: the last rounds are the tail's).
__global__ void __launch_bounds__(32 * RB_WARPS) rounds_hash_kernel(const DevProof* __restrict__ proofs, int np,
                                                                    const int* __restrict__ ibase,
                                                                    const Fr* __restrict__ partials,
                                                                    vl_proof* __restrict__ out, int t) {
  __shared__ uint32_t Ssh[RB_WARPS][8];
  __shared__ Fr gsh_all[RB_WARPS][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * RB_WARPS + warp;
  if (p >= np) return;  // whole warps leave together
  const DevProof& P = proofs[p];
  vl_proof* pf = out + P.job;
  uint32_t* S = Ssh[warp];
  Fr* gsh = gsh_all[warp];
  if (lane < 8) {
    const uint8_t* b = P.scr->state + 4 * lane;
    S[lane] = ((uint32_t)b[0] << 24) | ((uint32_t)b[1] << 16) | ((uint32_t)b[2] << 8) | (uint32_t)b[3];
  }
  if (t == 1) {
    if (lane == 0) {
      pf->m = P.m; pf->k = P.k; pf->n = P.n;
      pf->d0 = P.d0; pf->d1 = P.d1; pf->d2 = P.d2;
      pf->reserved = 0;
    }
    for (int i = P.d1 * 3 + lane; i < VL_MAX_ROUNDS * 3; i += 32) store_fr(&pf->g[i / 3][i % 3], fr_zero());
  }
  if (lane == 0) {
    Fr g[3] = {fr_zero(), fr_zero(), fr_zero()};
    for (int i = ibase[p]; i < ibase[p + 1]; i++)
#pragma unroll
      for (int q = 0; q < 3; q++) g[q] = fr_add(g[q], partials[3 * (size_t)i + q]);
#pragma unroll
    for (int q = 0; q < 3; q++) gsh[q] = g[q];
  }
  __syncwarp();
  const Fr r = round_transcript(S, gsh, t == 1, pf, t - 1);
  if (lane == 0) {
    P.scr->r = r;
    if (P.rch) P.rch[t - 1] = r;  // chained proofs continue from this point
  }
  __syncwarp();
  state_to_bytes(S, P.scr->state, lane);
}

// The rounds after the batched ones, one CTA per proof.
__global__ void __launch_bounds__(128, 4) rounds_tail_kernel(const DevProof* __restrict__ proofs,
                                                             vl_proof* __restrict__ out) {
  extern __shared__ __align__(128) uint8_t rnd_smem[];
  const DevProof& P = proofs[blockIdx.x];
  rounds_block(P, out + P.job, rnd_smem, 1 + batched_rounds(P.d1));
}

}  // namespace

cudaError_t launch_rounds_pass(const DevProof* proofs, const RoundItem* items, int nitems, Fr* partials, int t,
                               cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  rounds_pass_kernel<<<nitems, RB_THREADS, 0, st>>>(proofs, items, partials, t);
  return cudaGetLastError();
}

cudaError_t launch_rounds_hash(const DevProof* proofs, int nproofs, const int* ibase, const Fr* partials,
                               vl_proof* out, int t, cudaStream_t st) {
  if (nproofs <= 0) return cudaSuccess;
  rounds_hash_kernel<<<(nproofs + RB_WARPS - 1) / RB_WARPS, 32 * RB_WARPS, 0, st>>>(proofs, nproofs, ibase,
                                                                                    partials, out, t);
  return cudaGetLastError();
}

cudaError_t launch_rounds_tail(const DevProof* proofs, int nproofs, vl_proof* out, cudaStream_t st) {
  if (nproofs <= 0) return cudaSuccess;
  rounds_tail_kernel<<<nproofs, 128, RND_SMEM, st>>>(proofs, out);
  return cudaGetLastError();
}

}  // namespace vl
