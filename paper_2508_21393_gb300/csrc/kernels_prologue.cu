// Prologue kernels (see prologue_dev.cuh): the transcript part one CTA per
// proof, then the eq tables in chunks of EQ_CHUNK entries.
#include "prologue_dev.cuh"

namespace vl {

static constexpr int PRO_THREADS = 128;

__global__ void __launch_bounds__(PRO_THREADS, 8) transcript_kernel(const DevProof* __restrict__ proofs, int p0) {
  extern __shared__ __align__(128) uint8_t pro_smem[];
  transcript_block(proofs[p0 + blockIdx.x], pro_smem);
}

__global__ void __launch_bounds__(256) eq_kernel(const EqItem* __restrict__ items,
                                                  const DevProof* __restrict__ proofs) {
  const EqItem it = items[blockIdx.x];
  eq_chunk(it, proofs[it.proof]);
}

cudaError_t launch_prologue(const DevProof* proofs, int p0, int p1, const EqItem* items, int nitems,
                            cudaStream_t st) {
  if (p1 <= p0) return cudaSuccess;
  transcript_kernel<<<p1 - p0, PRO_THREADS, PRO_SMEM, st>>>(proofs, p0);
  if (nitems > 0) eq_kernel<<<nitems, 256, 0, st>>>(items, proofs);
  return cudaGetLastError();
}

}  // namespace vl
