// Prologue kernel: one CTA per proof (see prologue_dev.cuh).
#include "prologue_dev.cuh"

namespace vl {

static constexpr int PRO_THREADS = 128;

__global__ void __launch_bounds__(PRO_THREADS, 8) prologue_kernel(const DevProof* __restrict__ proofs) {
  extern __shared__ __align__(128) uint8_t pro_smem[];
  prologue_block(proofs[blockIdx.x], pro_smem);
}

cudaError_t launch_prologue(const DevProof* proofs, int nproofs, cudaStream_t st) {
  if (nproofs <= 0) return cudaSuccess;
  prologue_kernel<<<nproofs, PRO_THREADS, PRO_SMEM, st>>>(proofs);
  return cudaGetLastError();
}

}  // namespace vl
