// Fixed-point to field encoding (Sec. II-C embeds integer tensors in F; a
// negative x maps to r - |x|): dst = (x mod r) . 2^256 mod r, the Montgomery
// form the Montgomery-operand fold reads.  Memory-bound: 2 bytes in, 32 out.
#include "common.cuh"

namespace vl {

__global__ void __launch_bounds__(256) encode_kernel(const int16_t* __restrict__ src, int64_t rows, int64_t cols,
                                                     int64_t ld, Fr* __restrict__ dst) {
  const int64_t total = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols, c = i - r * cols;
    const int16_t x = src[r * ld + c];
    const Fr v = to_mont(fr_from_i64(x));
    uint4* d = reinterpret_cast<uint4*>(dst + i);
    d[0] = make_uint4(v.v[0], v.v[1], v.v[2], v.v[3]);
    d[1] = make_uint4(v.v[4], v.v[5], v.v[6], v.v[7]);
  }
}

cudaError_t launch_encode(const int16_t* src, int64_t rows, int64_t cols, int64_t ld, Fr* dst, cudaStream_t st) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  encode_kernel<<<(int)blocks, 256, 0, st>>>(src, rows, cols, ld, dst);
  return cudaGetLastError();
}

}  // namespace vl
