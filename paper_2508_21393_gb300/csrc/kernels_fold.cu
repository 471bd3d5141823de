// Fold kernel: one CTA per fold tile (see fold_dev.cuh).
#include <mutex>

#include "fold_dev.cuh"

namespace vl {

__global__ void __launch_bounds__(FOLD_THREADS, 2) fold_kernel(const FoldTask* __restrict__ tasks,
                                                               const FoldTile* __restrict__ tiles,
                                                               const DevProof* __restrict__ proofs,
                                                               unsigned long long wait_ns) {
  extern __shared__ __align__(128) uint8_t fold_smem[];
  const FoldTile t = tiles[blockIdx.x];
  const FoldTask T = tasks[t.task];
  fold_tile(T, t, proofs[T.proof], fold_smem, wait_ns);
}

// The limit is per kernel and process-wide, so it only ever grows: a plan
// bound later with smaller tiles must not lower it under an earlier plan.
cudaError_t fold_set_smem(int smem_bytes) {
  static std::mutex mu;  // plans are bound from several host threads
  static int current = 48 * 1024;
  std::lock_guard<std::mutex> lk(mu);
  if (smem_bytes <= current) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fold_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e == cudaSuccess) current = smem_bytes;
  return e;
}

cudaError_t launch_fold(const FoldTask* tasks, const FoldTile* tiles, int ntiles, const DevProof* proofs,
                        int smem_bytes, unsigned long long wait_ns, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  fold_kernel<<<ntiles, FOLD_THREADS, smem_bytes, st>>>(tasks, tiles, proofs, wait_ns);
  return cudaGetLastError();
}

}  // namespace vl
