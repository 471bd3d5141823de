// Lookup-argument sumcheck: the batched round passes (the rounds of every
// proof before its tail), one kernel instance per side set and round mode.
// Kept apart from kernels_lookup.cu so the two compile in parallel.
#include "lookup_dev.cuh"

namespace vl {

namespace {

// Round t over pairs [k0, k1) of one proof (the rounds before the proof's
// tail): the partial sums of lk_pair_a (and lk_pair_b in table rounds, JR)
// into the item's slot.  Warp w of the block takes the 32 LK_PPT pairs from
// k0 + 32 LK_PPT w, lanes strided by one (coalesced loads).  In a high round
// with 2^sE >= 32 LK_PPT the warp's pairs lie in one block of 2^sE pairs, so
// the block's hiP factor multiplies each lane's sums once; with smaller
// blocks it multiplies every pair's eq factor.
#ifndef LK_PASS_MINB
#define LK_PASS_MINB 2  // resident CTAs per SM the register budget of the passes allows
#endif
template <bool JR, int MODE>
__global__ void __launch_bounds__(LK_THREADS, LK_PASS_MINB) lk_pass_kernel(LkDev* Ls, int t, const LkItem* items) {
  __shared__ Fr red[6 * (LK_THREADS / 32)];
  const LkItem it = items[blockIdx.x];
  LkDev* L = Ls + it.proof;
  const int h = 1 << (L->L - t);
  const int tj = t - (L->L - L->log2_n);  // table round number (1-based) when JR
  const LkEq q(L, t);
  const bool lane_factor = q.high && L->sE >= LK_PPT_LOG + 5;  // the warp's pairs share one hiP entry
  const int kw = it.k0 + (threadIdx.x >> 5) * (32 * LK_PPT);
  Fr acc[6];
#pragma unroll
  for (int i = 0; i < 6; i++) acc[i] = fr_zero();
  Fr accb[6];
  if constexpr (JR) {
#pragma unroll
    for (int i = 0; i < 6; i++) accb[i] = fr_zero();
  }
#pragma unroll 1
  for (int k = kw + (threadIdx.x & 31); k < min(it.k1, kw + 32 * LK_PPT); k += 32) {
    Fr f = q.f_tab[k & q.f_mask];
    if (q.high && !lane_factor) f = mont_mul_ni(f, q.hi_tab[k >> L->sE]);
    lk_pair_a<MODE>(L, t, k, h, f, acc);
    if constexpr (JR) lk_pair_b(L, t, tj, k, h, f, accb);
  }
  if constexpr (MODE == 0) lk_mode0_sums(acc);
  if constexpr (JR)
    if (tj == 1) lk_mode0_sums(accb);
  if (lane_factor && kw < it.k1) {  // the eq factor over the remaining high variables
    const Fr hf = q.hi_tab[kw >> L->sE];
    for (int i = 0; i < 3; i++) acc[i] = mont_mul_ni(acc[i], hf);
    if constexpr (JR)
      for (int i = 0; i < 3; i++) accb[i] = mont_mul_ni(accb[i], hf);
  }
  block_sum_fr<6>(acc, red);
  if (threadIdx.x == 0)
    for (int i = 0; i < 6; i++) L->part[(size_t)it.slot * 12 + i] = acc[i];
  if constexpr (JR) {
    block_sum_fr<6>(accb, red);
    if (threadIdx.x == 0)
      for (int i = 0; i < 6; i++) L->part[(size_t)it.slot * 12 + 6 + i] = accb[i];
  }
}

}  // namespace

// Round t's passes: nhi items of proofs in their high rounds, then nlo items
// of proofs in their table rounds.
cudaError_t launch_lookup_passes(LkDev* Ls, int t, const LkItem* items, int nhi, int nlo, cudaStream_t st) {
  if (nhi) {
    if (t == 1) lk_pass_kernel<false, 0><<<nhi, LK_THREADS, 0, st>>>(Ls, t, items);
    else if (t == 2) lk_pass_kernel<false, 1><<<nhi, LK_THREADS, 0, st>>>(Ls, t, items);
    else lk_pass_kernel<false, 2><<<nhi, LK_THREADS, 0, st>>>(Ls, t, items);
  }
  if (nlo) {
    if (t == 1) lk_pass_kernel<true, 0><<<nlo, LK_THREADS, 0, st>>>(Ls, t, items + nhi);
    else if (t == 2) lk_pass_kernel<true, 1><<<nlo, LK_THREADS, 0, st>>>(Ls, t, items + nhi);
    else lk_pass_kernel<true, 2><<<nlo, LK_THREADS, 0, st>>>(Ls, t, items + nhi);
  }
  return cudaGetLastError();
}

}  // namespace vl
