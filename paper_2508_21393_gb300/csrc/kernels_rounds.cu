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

// variant: CTAs per SM.  7 and 4 set the register allocation (7: one wave of
// 1064 proofs, tighter registers; 4: more registers per thread).  3 and 2
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
  } else {
    rounds_kernel<7, 128><<<nproofs, 128, RND_SMEM, st>>>(proofs, out);
  }
  return cudaGetLastError();
}

}  // namespace vl
