// The whole proving step in one persistent launch.
//
// The grid holds exactly as many CTAs as fit on the GPU at once; each CTA
// takes work items in queue order from a global counter:
//   * prologue item p: transcript start, u/v squeezes and eq tables of proof
//     p, then a release store of ready[p];
//   * fold tile t of proof p: acquire ready[p] (bounded wait), fold the tile
//     into the proof's accumulators, then count it in done[p].  The CTA that
//     counts the last tile of proof p runs p's claim and sumcheck rounds at
//     once, so rounds of finished proofs overlap the folds of later ones.
// A fold item only waits for a prologue queued before it, which some running
// CTA has already taken and finishes without waiting: the queue cannot
// deadlock.  Every wait is bounded (wait_ns of the global timer); one that
// runs out marks the proof VL_ETIMEOUT and skips the tile.  `never_ready`
// (a proof index, or -1) is a test hook: that proof's ready flag is never
// set, so its tiles exercise the timeout path.
#include <mutex>

#include "fold_dev.cuh"
#include "prologue_dev.cuh"
#include "rounds_dev.cuh"

namespace vl {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *flag != 0, at most wait_ns of the global timer.
static __device__ bool wait_flag(const int* flag, uint64_t wait_ns) {
  if (ld_acquire(flag)) return true;
  const uint64_t deadline = global_ns() + wait_ns;
  while (!ld_acquire(flag)) {
    if (global_ns() > deadline) return false;
    __nanosleep(256);
  }
  return true;
}

__global__ void __launch_bounds__(FOLD_THREADS, 2) step_kernel(const StepItem* __restrict__ items, int nitems,
                                                               const FoldTask* __restrict__ tasks,
                                                               const FoldTile* __restrict__ tiles,
                                                               const DevProof* __restrict__ proofs, int nproofs,
                                                               vl_proof* __restrict__ out, int* ctl,
                                                               unsigned long long wait_ns, int never_ready) {
  extern __shared__ __align__(128) uint8_t step_smem[];
  __shared__ int item_sh, flag_sh;
  int* head = ctl;
  int* ready = ctl + STEP_CTL_HEAD_INTS;
  int* done = ready + nproofs;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) item_sh = atomicAdd(head, 1);
    __syncthreads();
    const int it = item_sh;
    __syncthreads();
    if (it >= nitems) return;
    const StepItem I = items[it];
    if (I.kind == STEP_PROLOGUE) {
      prologue_block(proofs[I.idx], step_smem);
      __threadfence();
      __syncthreads();
      if (tid == 0 && I.idx != never_ready) st_release(&ready[I.idx], 1);
      continue;
    }
    const FoldTile t = tiles[I.idx];
    const FoldTask T = tasks[t.task];
    const int p = T.proof;
    const DevProof& P = proofs[p];
    if (tid == 0) {
      flag_sh = wait_flag(&ready[p], wait_ns) ? 1 : 0;
      if (!flag_sh) atomicExch(&P.scr->status, VL_ETIMEOUT);
    }
    __syncthreads();
    if (flag_sh) fold_tile(T, t, P, step_smem, wait_ns);
    __threadfence();
    __syncthreads();
    if (tid == 0) flag_sh = atomicAdd(&done[p], 1) == P.ntiles - 1;
    __syncthreads();
    if (flag_sh) {
      __threadfence();
      rounds_block(P, out + P.job, step_smem);
    }
  }
}

cudaError_t step_set_smem(int smem_bytes) {
  static std::mutex mu;  // plans are bound from several host threads
  static int current = 48 * 1024;
  std::lock_guard<std::mutex> lk(mu);
  if (smem_bytes <= current) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e == cudaSuccess) current = smem_bytes;
  return e;
}

cudaError_t step_grid(int smem_bytes, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel, FOLD_THREADS, smem_bytes);
  if (e != cudaSuccess) return e;
  *grid = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

cudaError_t launch_step(const StepItem* items, int nitems, const FoldTask* tasks, const FoldTile* tiles,
                        const DevProof* proofs, int nproofs, vl_proof* out, int* ctl, int grid, int smem_bytes,
                        unsigned long long wait_ns, int never_ready, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  step_kernel<<<grid, FOLD_THREADS, smem_bytes, st>>>(items, nitems, tasks, tiles, proofs, nproofs, out, ctl, wait_ns,
                                                      never_ready);
  return cudaGetLastError();
}

}  // namespace vl
