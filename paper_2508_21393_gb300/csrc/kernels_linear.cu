// Linear zkMat: sum_q c_q M_q = 0 by MLE linearity (Sec. IV; Eq. eq:MLE).
//
// M~(x, y) = sum_i sum_j eq(x, i) M[i, j] eq(y, j) is computed as a fold
// over one dimension (the shorter, "reduced") followed by a dot product over
// the other ("lines"):
//   start:  per proof, transcript start over the statement, squeezes of x
//           (d0) and y (d1), the eq factor tables of both sides, the fold's
//           offset correction (closed form, in a warp of its own); then, in
//           chunks, the reduced side's eq table as the tensor-core fold's
//           fp16 byte table;
//   (the tensor-core fold writes f_q = the reduced vector of every matrix;
//   reductions of at most LIN_SHORT_MAX entries fold on CUDA cores instead,
//   one thread per line, from the table's limbs)
//   finish: the lines side's eq table is never formed: with
//           E[w] = hi[w >> s] . lo[w mod 2^s],
//             e_q = sum_j hi[j] . (sum_l f_q[j 2^s + l] . lo[l]),
//           one warp per inner sum (one Montgomery product per line), then
//           per proof the outer sums, the absorb of 'e' and the proof.
#include "prologue_dev.cuh"

namespace vl {

namespace {

constexpr uint8_t LBL_X = 'x', LBL_Y = 'y', LBL_E = 'e';
constexpr int LIN_THREADS = 256;
constexpr int LIN_FAC_THREADS = LIN_THREADS - 32;  // the last warp computes the correction

// Factor entry j of one side (lo entries first): a product of eq factors,
// starting from 1 in double-Montgomery (lo of the reduced side) or
// Montgomery form (everything else).
__device__ Fr lin_factor(const Fr* x, int d, int j, bool lo_double, bool* is_lo, int* idx) {
  const int s = (d + 1) >> 1, dh = d - s, nlo = 1 << s;
  *is_lo = j < nlo;
  const int jj = *is_lo ? j : j - nlo, nv = *is_lo ? s : dh, base = *is_lo ? dh : 0;
  *idx = jj;
  Fr acc = (*is_lo && lo_double) ? fr_r2() : fr_r1();
  for (int t = 0; t < nv; t++) {
    const Fr& xt = x[base + t];
    acc = mont_mul_ni(acc, ((jj >> (nv - 1 - t)) & 1) ? xt : fr_sub(fr_r1(), xt));
  }
  return acc;
}

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
  const bool rr = L->red_rows != 0;
  if (tid < LIN_FAC_THREADS) {
    // Both sides' factor tables in one loop: [x lo | x hi | y lo | y hi].
    const int sx = (L->d0 + 1) >> 1, sy = (L->d1 + 1) >> 1;
    const int nx = (1 << sx) + ((L->rows + (1 << sx) - 1) >> sx);
    const int ny = (1 << sy) + ((L->cols + (1 << sy) - 1) >> sy);
    for (int j = tid; j < nx + ny; j += LIN_FAC_THREADS) {
      const bool xside = j < nx;
      bool is_lo;
      int idx;
      const Fr v = xside ? lin_factor(xs, L->d0, j, rr, &is_lo, &idx) : lin_factor(ys, L->d1, j - nx, !rr, &is_lo, &idx);
      L->fac[(xside ? 0 : 2 * EQ_FAC) + (is_lo ? 0 : EQ_FAC) + idx] = v;
    }
  } else if (tid == LIN_FAC_THREADS) {
    const Fr sum = rr ? eq_prefix_sum(xs, L->d0, L->rows) : eq_prefix_sum(ys, L->d1, L->cols);
    L->corr = mont_mul_ni(sum, to_mont_ni(fr_small(1u << 15)));
    L->scr->status = VL_OK;
  }
}

// Entries [i0, i1) of one proof's reduced-side table (fp16 bytes, zero up
// to a multiple of 128 entries).
__global__ void __launch_bounds__(LIN_THREADS) lin_eq_kernel(const LinDev* Ls, const EqItem* items) {
  const EqItem it = items[blockIdx.x];
  const LinDev* L = Ls + it.proof;
  const bool xside = L->red_rows != 0;
  const int d = xside ? L->d0 : L->d1, size = xside ? L->rows : L->cols;
  const int s = (d + 1) >> 1, mask = (1 << s) - 1;
  const Fr* lo = L->fac + (xside ? 0 : 2 * EQ_FAC);
  const Fr* hi = lo + EQ_FAC;
  for (int i = it.i0 + threadIdx.x; i < it.i1; i += blockDim.x) {
    const Fr e = i < size ? mont_mul_ni(hi[i >> s], lo[i & mask]) : fr_zero();  // eq . R^2
    store_w8(L->w8, i, e);
    if (L->e2 && i < size) L->e2[i] = e;  // short reductions fold on CUDA cores with the limbs
  }
}

// Short reductions (red <= LIN_SHORT_MAX): thread w of the block folds line
// w0 + w of one matrix.  With p = x + 2^15 in [0, 2^16) and e = E R^2,
// sum_j e_j p_j is an exact integer, kept as eight 64-bit column sums of the
// limb products (each below 2^48, at most 128 of them); one REDC gives
// (sum_j E_j p_j) R, and subtracting 2^15 (sum_j E_j) R (the offset
// correction) leaves f_q[line] = sum_j E_j x_j in Montgomery form: the value
// the tensor-core fold writes for the same line.
__global__ void __launch_bounds__(LIN_SHORT_LINES) lin_short_kernel(const LinDev* Ls, const LinShort* items) {
  __shared__ __align__(16) Fr e2s[LIN_SHORT_MAX];
  const LinShort it = items[blockIdx.x];
  const LinDev* L = Ls + it.proof;
  for (int j = threadIdx.x; j < it.red; j += blockDim.x) e2s[j] = L->e2[j];
  __syncthreads();
  const int w = threadIdx.x;
  if (w >= it.nw) return;
  const int64_t line = it.w0 + w;
  unsigned long long acc[8];
#pragma unroll
  for (int l = 0; l < 8; l++) acc[l] = 0;
  // acc[l] += e_j[l] . p_j as one 32 x 32 -> 64-bit multiply-add per limb
  // (the weights as two 16-byte shared-memory loads)
  auto add = [&](int j, int16_t x) {
    const uint32_t p = (uint32_t)((int32_t)x + 32768);
    const uint4 e0 = reinterpret_cast<const uint4*>(&e2s[j])[0];
    const uint4 e1 = reinterpret_cast<const uint4*>(&e2s[j])[1];
    const uint32_t ev[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
    for (int l = 0; l < 8; l++) asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[l]) : "r"(ev[l]), "r"(p));
  };
  // Loads are issued in groups before their entries are used, so that each
  // thread has several in flight.
  if (it.mode == MODE_ROWDOT) {
    const int16_t* row = it.base + line * it.ld;
    int j = 0;
    if ((reinterpret_cast<uintptr_t>(row) & 15) == 0) {  // eight entries per 16-byte load
      for (; j + 32 <= it.red; j += 32) {
        uint4 v[4];
#pragma unroll
        for (int b = 0; b < 4; b++) v[b] = __ldg(reinterpret_cast<const uint4*>(row + j) + b);
#pragma unroll
        for (int b = 0; b < 4; b++) {
          const uint32_t wv[4] = {v[b].x, v[b].y, v[b].z, v[b].w};
#pragma unroll
          for (int i = 0; i < 4; i++) {
            add(j + 8 * b + 2 * i, (int16_t)(wv[i] & 0xffffu));
            add(j + 8 * b + 2 * i + 1, (int16_t)(wv[i] >> 16));
          }
        }
      }
      for (; j + 8 <= it.red; j += 8) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + j));
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
          add(j + 2 * i, (int16_t)(wv[i] & 0xffffu));
          add(j + 2 * i + 1, (int16_t)(wv[i] >> 16));
        }
      }
    }
    for (; j + 8 <= it.red; j += 8) {
      int16_t x[8];
#pragma unroll
      for (int i = 0; i < 8; i++) x[i] = __ldg(row + j + i);
#pragma unroll
      for (int i = 0; i < 8; i++) add(j + i, x[i]);
    }
    for (; j < it.red; j++) add(j, __ldg(row + j));
  } else {
    const int16_t* col = it.base + line;  // a warp reads consecutive columns of each row
    int j = 0;
    for (; j + 8 <= it.red; j += 8) {
      int16_t x[8];
#pragma unroll
      for (int i = 0; i < 8; i++) x[i] = __ldg(col + (int64_t)(j + i) * it.ld);
#pragma unroll
      for (int i = 0; i < 8; i++) add(j + i, x[i]);
    }
    for (; j < it.red; j++) add(j, __ldg(col + (int64_t)j * it.ld));
  }
  U64x8 a;
#pragma unroll
  for (int l = 0; l < 8; l++) a.v[l] = acc[l];
  L->f[(size_t)it.q * L->lines + line] = fr_sub(redc_columns_ni(a), L->corr);
}

// Warp w of block (b, q, proof) sums inner block j = 8 b + w of matrix q:
// part[q][j] = sum_l f_q[j 2^s + l] . lo[l] (Montgomery; f from the
// accumulators when the fold ran in several segments).
__global__ void __launch_bounds__(LIN_THREADS) lin_dot_kernel(LinDev* Ls) {
  LinDev* L = Ls + blockIdx.z;
  const int q = blockIdx.y, lane = threadIdx.x & 31;
  const int j = blockIdx.x * (LIN_THREADS / 32) + (threadIdx.x >> 5);
  if (q >= L->nmats || j >= L->nblk) return;
  const bool xside = L->red_rows == 0;  // the lines side
  const int d = xside ? L->d0 : L->d1, lines = L->lines;
  const int s = (d + 1) >> 1, hb = 1 << s;
  const Fr* lo = L->fac + (xside ? 0 : 2 * EQ_FAC);
  const Fr corr = L->corr;
  // f_q[w] (Montgomery), from the accumulators when the fold ran in several segments
  auto load_f = [&](int w) {
    const size_t i = (size_t)q * lines + w;
    if (!L->acc) return L->f[i];
    U64x8 a;
#pragma unroll
    for (int l = 0; l < 8; l++) a.v[l] = L->acc[i * 8 + l];
    return fr_sub(redc_columns_ni(a), corr);
  };
  Fr acc = fr_zero();
  const int w1 = min(lines, (j + 1) * hb);
  int w = j * hb + lane;
  // Two independent inline products per step: the carry chains interleave.
  for (; w + 32 < w1; w += 64) {
    const Fr f0 = load_f(w), f1 = load_f(w + 32);
    const Fr p0 = mont_mul(f0, lo[w & (hb - 1)]), p1 = mont_mul(f1, lo[(w + 32) & (hb - 1)]);
    acc = fr_add(acc, fr_add(p0, p1));
  }
  if (w < w1) acc = fr_add(acc, mont_mul_ni(load_f(w), lo[w & (hb - 1)]));
  acc = warp_sum_fr(acc);
  if (lane == 0) L->part[(size_t)q * L->nblk + j] = acc;
}

// One block per proof: e_q = sum_j part[q][j] . hi[j], absorb, proof.
__global__ void __launch_bounds__(LIN_THREADS) lin_finish_kernel(const LinDev* Ls, vl_lin_proof* outs) {
  __shared__ Fr red[LIN_THREADS / 32];
  __shared__ Fr ev[VL_LIN_MAX];
  const LinDev* L = Ls + blockIdx.x;
  vl_lin_proof* out = outs + blockIdx.x;
  const int tid = threadIdx.x, nm = L->nmats;
  const Fr* hi = L->fac + (L->red_rows ? 2 * EQ_FAC : 0) + EQ_FAC;  // the lines side's outer factors
  for (int q = 0; q < nm; q++) {
    Fr acc[1] = {fr_zero()};
    for (int j = tid; j < L->nblk; j += blockDim.x)
      acc[0] = fr_add(acc[0], mont_mul_ni(L->part[(size_t)q * L->nblk + j], hi[j]));
    block_sum_fr<1>(acc, red);
    if (tid == 0) ev[q] = from_mont_ni(acc[0]);
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

cudaError_t launch_linear_short(const LinDev* Ls, const LinShort* items, int nitems, cudaStream_t st) {
  if (nitems > 0) lin_short_kernel<<<nitems, LIN_SHORT_LINES, 0, st>>>(Ls, items);
  return cudaGetLastError();
}

cudaError_t launch_linear_finish(LinDev* Ls, int nproofs, int max_nblk, int max_nmats, vl_lin_proof* out,
                                 cudaStream_t st) {
  const int bx = (max_nblk + LIN_THREADS / 32 - 1) / (LIN_THREADS / 32);
  lin_dot_kernel<<<dim3(bx, max_nmats, nproofs), LIN_THREADS, 0, st>>>(Ls);
  lin_finish_kernel<<<nproofs, LIN_THREADS, 0, st>>>(Ls, out);
  return cudaGetLastError();
}

}  // namespace vl
