// Linear zkMat: sum_q c_q M_q = 0 by MLE linearity (Sec. IV; Eq. eq:MLE).
//
// M~(x, y) = sum_i sum_j eq(x, i) M[i, j] eq(y, j) is computed as a fold
// over one dimension followed by a dot product over the other:
//   start:  per proof, transcript start over the statement, squeezes of x
//           (d0) and y (d1), the eq factor tables of both, the fold's offset
//           correction (closed form); then, in chunks, the reduced side's eq
//           table as the tensor-core fold's fp16 byte table and the lines
//           side's in Montgomery form;
//   (the tensor-core fold writes f_q = the reduced vector of every matrix)
//   finish: e_q = sum_w f_q[w] E_lines[w] in blocks of LIN_DOT lines, then
//           the partial sums, the absorb of 'e' and the proof.
#include "prologue_dev.cuh"

namespace vl {

namespace {

constexpr uint8_t LBL_X = 'x', LBL_Y = 'y', LBL_E = 'e';
constexpr int LIN_THREADS = 256;

// One block per proof.
__global__ void __launch_bounds__(LIN_THREADS) lin_start_kernel(LinDev* Ls) {
  LinDev* L = Ls + blockIdx.x;
  __shared__ uint32_t S0[8], S1[8], S2[8];
  __shared__ uint32_t dig[2 * MAX_VARS + 1][8];
  __shared__ Fr xs[MAX_VARS], ys[MAX_VARS];
  const int tid = threadIdx.x;
  if (tid == 0) {
    uint8_t b[32];
    ts_start_linear(b, L->seed, (uint32_t)L->rows, (uint32_t)L->cols, L->nmats, L->coeffs, L->binds);
    for (int i = 0; i < 8; i++)
      S0[i] = ((uint32_t)b[4 * i] << 24) | ((uint32_t)b[4 * i + 1] << 16) | ((uint32_t)b[4 * i + 2] << 8) | b[4 * i + 3];
  }
  __syncthreads();
  squeeze_dev(S0, LBL_X, L->d0, xs, S1, dig);
  squeeze_dev(S1, LBL_Y, L->d1, ys, S2, dig);
  if (tid < 8) L->S[tid] = S2[tid];
  eq_factors(xs, L->d0, L->rows, L->fac, L->fac + EQ_FAC);
  eq_factors(ys, L->d1, L->cols, L->fac + 2 * EQ_FAC, L->fac + 3 * EQ_FAC);
  if (tid == 0) {
    const Fr sum = L->red_rows ? eq_prefix_sum(xs, L->d0, L->rows) : eq_prefix_sum(ys, L->d1, L->cols);
    L->corr = mont_mul_ni(sum, to_mont_ni(fr_small(1u << 15)));
    L->scr->status = VL_OK;
  }
}

// Entries [i0, i1) of one proof's reduced-side table (fp16 bytes, zero up
// to a multiple of 128 entries) or lines-side table (Montgomery).
__global__ void __launch_bounds__(LIN_THREADS) lin_eq_kernel(const LinDev* Ls, const EqItem* items) {
  const EqItem it = items[blockIdx.x];
  const LinDev* L = Ls + it.proof;
  const bool red = it.side != 0;
  const bool xside = red == (L->red_rows != 0);
  const int d = xside ? L->d0 : L->d1, size = xside ? L->rows : L->cols;
  const int s = (d + 1) >> 1, mask = (1 << s) - 1;
  const Fr* lo = L->fac + (xside ? 0 : 2 * EQ_FAC);
  const Fr* hi = lo + EQ_FAC;
  for (int i = it.i0 + threadIdx.x; i < it.i1; i += blockDim.x) {
    const Fr e = i < size ? mont_mul_ni(hi[i >> s], lo[i & mask]) : fr_zero();  // eq . R^2
    if (red) store_w8(L->w8, i, e);
    else L->el[i] = mont_mul_ni(e, fr_small(1));  // eq . R
  }
}

// Block (b, q, proof): sum over lines [b LIN_DOT, (b + 1) LIN_DOT) of
// f_q[w] E[w]; blocks past the proof's matrices or lines return at once.
__global__ void __launch_bounds__(LIN_THREADS) lin_dot_kernel(LinDev* Ls) {
  __shared__ Fr red[LIN_THREADS / 32];
  LinDev* L = Ls + blockIdx.z;
  const int q = blockIdx.y, b = blockIdx.x, lines = L->lines;
  if (q >= L->nmats || b >= L->nblk) return;
  const int w1 = min(lines, (b + 1) * LIN_DOT);
  const Fr corr = L->corr;
  Fr acc[1] = {fr_zero()};
  for (int w = b * LIN_DOT + threadIdx.x; w < w1; w += blockDim.x) {
    const size_t i = (size_t)q * lines + w;
    Fr fw;
    if (L->acc) {
      U64x8 a;
#pragma unroll
      for (int l = 0; l < 8; l++) a.v[l] = L->acc[i * 8 + l];
      fw = fr_sub(redc_columns_ni(a), corr);
    } else {
      fw = L->f[i];
    }
    acc[0] = fr_add(acc[0], mont_mul_ni(fw, L->el[w]));
  }
  block_sum_fr<1>(acc, red);
  if (threadIdx.x == 0) L->part[(size_t)q * L->nblk + b] = acc[0];
}

// One block per proof.
__global__ void __launch_bounds__(LIN_THREADS) lin_finish_kernel(const LinDev* Ls, vl_lin_proof* outs) {
  __shared__ Fr ev[VL_LIN_MAX];
  const LinDev* L = Ls + blockIdx.x;
  vl_lin_proof* out = outs + blockIdx.x;
  const int tid = threadIdx.x, nm = L->nmats;
  if (tid < nm) {
    Fr s = fr_zero();
    for (int b = 0; b < L->nblk; b++) s = fr_add(s, L->part[(size_t)tid * L->nblk + b]);
    ev[tid] = from_mont_ni(s);
  }
  __syncthreads();
  if (tid == 0) {
    uint8_t S[32];
    for (int i = 0; i < 32; i++) S[i] = (uint8_t)(L->S[i >> 2] >> (24 - 8 * (i & 3)));
    ts_absorb_fr(S, LBL_E, ev, nm);
    out->rows = L->rows;
    out->cols = L->cols;
    out->d0 = L->d0;
    out->d1 = L->d1;
    out->nmats = nm;
    out->status = L->scr->status;
    for (int i = 0; i < 32; i++) out->state[i] = S[i];
  }
  for (int i = tid; i < VL_LIN_MAX * 8; i += blockDim.x)
    out->evals[i >> 3].limb[i & 7] = (i >> 3) < nm ? ev[i >> 3].v[i & 7] : 0u;
}

}  // namespace

cudaError_t launch_linear_start(LinDev* Ls, int nproofs, const EqItem* items, int nitems, cudaStream_t st) {
  lin_start_kernel<<<nproofs, LIN_THREADS, 0, st>>>(Ls);
  if (nitems > 0) lin_eq_kernel<<<nitems, LIN_THREADS, 0, st>>>(Ls, items);
  return cudaGetLastError();
}

cudaError_t launch_linear_finish(LinDev* Ls, int nproofs, int max_nblk, int max_nmats, vl_lin_proof* out,
                                 cudaStream_t st) {
  lin_dot_kernel<<<dim3(max_nblk, max_nmats, nproofs), LIN_THREADS, 0, st>>>(Ls);
  lin_finish_kernel<<<nproofs, LIN_THREADS, 0, st>>>(Ls, out);
  return cudaGetLastError();
}

}  // namespace vl
