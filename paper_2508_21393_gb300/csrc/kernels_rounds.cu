// Rounds kernel: one CTA per proof (see rounds_dev.cuh).
#include "rounds_dev.cuh"

namespace vl {

static constexpr int RND_THREADS = 128;

template <int MINB>
__global__ void __launch_bounds__(RND_THREADS, MINB) rounds_kernel(const DevProof* __restrict__ proofs,
                                                                   vl_proof* __restrict__ out) {
  extern __shared__ __align__(128) uint8_t rnd_smem[];
  const DevProof& P = proofs[blockIdx.x];
  rounds_block(P, out + P.job, rnd_smem);
}

// variant: CTAs per SM the register allocation targets (7: one wave of 1064
// proofs, tighter registers; 4: more registers per thread, more waves).
cudaError_t launch_rounds(const DevProof* proofs, int nproofs, vl_proof* out, int variant, cudaStream_t st) {
  if (nproofs <= 0) return cudaSuccess;
  if (variant == 4) rounds_kernel<4><<<nproofs, RND_THREADS, RND_SMEM, st>>>(proofs, out);
  else rounds_kernel<7><<<nproofs, RND_THREADS, RND_SMEM, st>>>(proofs, out);
  return cudaGetLastError();
}

}  // namespace vl
