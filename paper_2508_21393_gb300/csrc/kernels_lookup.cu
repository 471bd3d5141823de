// Lookup-argument sumcheck (Sec. II, lookup arguments; Protocol 1; Eq.
// eq:lookup-sumcheck) for range tables T_j = t0 + j, j < N, over a batch of
// proofs.
//
// The sumcheck runs over k = (i, j) in {0,1}^L, L = log2 D, binding the most
// significant variable first, on
//   P(k) = alpha A(k) E(k) S'(k) + A(k) + (N/D)(alpha^2 B(j) Ej(j) T'(j) - B(j) m(j))
// with A = 1/(beta + S), E = eq(u, .), S' = S + beta, B = 1/(beta + T),
// Ej = eq(u_low, .), T' = T + beta.  The table side depends on the low
// log2 N variables only, so in the first L - log2 N rounds its contribution
// to g_t(X) is the constant 2^-t . Cb, Cb = alpha^2 sum B Ej T' - sum B m;
// in the last log2 N rounds its four vectors are folded like the others.
//
// E = eq(u, .) is never formed: folded by r_1 .. r_{t-1} it is
//   E_t(X, k) = c_t . eqf(u_t, X) . eq(u_{t+1..L}, k),
//   c_t = prod_{v<t} eqf(u_v, r_v), eqf(u, x) = u x + (1 - u)(1 - x),
// so a pass sums eq(u_{t+1..L}, k) . (A S')(X, k) and the transcript step
// multiplies by the scalar c_t eqf(u_t, X).  eq(u_{t+1..L}, k) is read from
// suffix tables: while t binds one of the first L - sE variables it is
// hiP[k >> sE] . loP_sE[k mod 2^sE], later loP_(L-t)[k].
//
// Launches: start (per proof: transcript, beta, alpha, u, N/D, claim),
// factors (the suffix eq tables and eq(u_low, .)), histogram
// (multiplicities, range check), table (batch inversion of beta + T per
// 1024-entry block, table-side vectors, partial sums of Cb); per round a
// pass over all proofs' pairs (fold with the previous challenge, then the
// partial sums of g(0), g(2), g(3)) and a transcript step per proof; finish.
// A never exists as a vector: its entries are gathered from B by value
// (A_k = B_{S_k - t0}), and S' from T'.
#include "lookup_dev.cuh"

namespace vl {

namespace {

// One block per proof.
__global__ void __launch_bounds__(LK_THREADS) lk_start_kernel(LkDev* Ls) {
  LkDev* L = Ls + blockIdx.x;
  __shared__ uint32_t S0[8], S1[8], S2[8], S3[8];
  __shared__ uint32_t dig[2 * LK_MAX_L + 1][8];
  __shared__ Fr ch[LK_MAX_L];
  __shared__ Fr beta_sh, alpha_sh;
  const int tid = threadIdx.x;
  if (tid == 0) {
    uint8_t b[32];
    ts_start_lookup(b, L->seed, (uint32_t)L->n, (uint32_t)L->L, (uint32_t)L->log2_n, L->t0, L->bind);
    for (int i = 0; i < 8; i++)
      S0[i] = ((uint32_t)b[4 * i] << 24) | ((uint32_t)b[4 * i + 1] << 16) | ((uint32_t)b[4 * i + 2] << 8) | b[4 * i + 3];
  }
  __syncthreads();
  squeeze_dev(S0, LBL_BETA, 1, ch, S1, dig);
  if (tid == 0) beta_sh = ch[0];
  __syncthreads();
  squeeze_dev(S1, LBL_ALPHA, 1, ch, S2, dig);
  if (tid == 0) alpha_sh = ch[0];
  __syncthreads();
  squeeze_dev(S2, LBL_U, L->L, ch, S3, dig);
  if (tid < L->L) L->u[tid] = ch[tid];
  if (tid < 8) L->St[tid] = S3[tid];
  if (tid == 0) {
    const Fr alpha = alpha_sh;
    L->beta = beta_sh;
    L->alpha = alpha;
    L->claim = fr_add(alpha, mont_mul(alpha, alpha));
    L->half_t = fr_r1();
    L->ct = fr_r1();
    L->ctj = fr_r1();
    Fr c = fr_r1();  // N / D = 2^-(L - log2 N)
    for (int i = 0; i < L->L - L->log2_n; i++) c = mont_mul(c, L->inv2);
    L->c_nd = c;
    L->scr->status = VL_OK;
    const uint32_t pad = (uint32_t)((1 << L->L) - L->n);  // padding entries hold t0: table index 0
    if (pad) atomicAdd(&L->counts[0], pad);
  }
}

// eq table over nv <= 8 variables x[0..nv) (MSB first) into tab[0..2^nv),
// block-wide: doubling, each level appending the next variable as the new
// lowest bit (one product per new entry).
__device__ void lk_eq_small(Fr* tab, const Fr* x, int nv) {
  if (threadIdx.x == 0) tab[0] = fr_r1();
  __syncthreads();
  for (int l = 0; l < nv; l++) {
    const int j = threadIdx.x;
    Fr a = fr_zero();
    if (j < (1 << l)) a = tab[j];
    __syncthreads();
    if (j < (1 << l)) {
      const Fr xl = x[l];
      tab[2 * j] = mont_mul_ni(a, fr_sub(fr_r1(), xl));
      tab[2 * j + 1] = mont_mul_ni(a, xl);
    }
    __syncthreads();
  }
}

// Suffix eq tables: item.slot 0 = loP (levels m = 0..sE: eq over the last
// m variables of u), 1 = hiP (levels m = 0..L-sE-1: eq over the last m of
// the first L - sE variables), 2 = eq(u_low, .) into WE (the last log2 N).
// Entry e of a pyramid is level m = floor(log2(e + 1)), index e + 1 - 2^m;
// its value is the product of x or 1 - x per bit (MSB first).
__global__ void __launch_bounds__(LK_THREADS) lk_factor_kernel(LkDev* Ls, const LkItem* items) {
  const LkItem it = items[blockIdx.x];
  LkDev* L = Ls + it.proof;
  if (it.slot == 2) {
    // eq(u_low, i) over the last n = log2 N variables, MSB first, as
    // hi[i >> s] . lo[i mod 2^s]: lo over the last s = min(n, 8) variables,
    // hi over the n - s before them (both at most 256 entries, built in
    // shared memory), then one product per entry instead of n.
    __shared__ Fr lo[256], hi[256];
    const int nb = L->log2_n, sl = nb < 8 ? nb : 8;
    lk_eq_small(lo, L->u + (L->L - sl), sl);
    lk_eq_small(hi, L->u + (L->L - nb), nb - sl);
    for (int e = it.k0 + threadIdx.x; e < it.k1; e += blockDim.x)
      L->WE[e] = mont_mul_ni(hi[e >> sl], lo[e & ((1 << sl) - 1)]);
    return;
  }
  Fr* out = it.slot == 0 ? L->loP : L->hiP;
  const int top = it.slot == 1 ? L->L - L->sE : L->L;  // the suffixes end at variable top - 1 (0-based)
  for (int e = it.k0 + threadIdx.x; e < it.k1; e += blockDim.x) {
    const int m = 31 - __clz(e + 1), i = e + 1 - (1 << m);
    Fr acc = fr_r1();
    for (int t = 0; t < m; t++) {
      const Fr& x = L->u[top - m + t];
      acc = mont_mul_ni(acc, ((i >> (m - 1 - t)) & 1) ? x : fr_sub(fr_r1(), x));
    }
    out[e] = acc;
  }
}

// Multiplicities of entries [k0, k1) of S; a value outside the table marks
// the proof VL_ELOOKUP.  Tables up to 4096 entries count in shared memory.
__global__ void __launch_bounds__(LK_THREADS) lk_hist_kernel(LkDev* Ls, const LkItem* items) {
  __shared__ uint32_t h[4096];
  const LkItem it = items[blockIdx.x];
  LkDev* L = Ls + it.proof;
  const int N = 1 << L->log2_n;
  const bool local = N <= 4096;
  if (local)
    for (int j = threadIdx.x; j < N; j += blockDim.x) h[j] = 0;
  __syncthreads();
  bool bad = false;
  for (int k = it.k0 + threadIdx.x; k < it.k1; k += blockDim.x) {
    const int row = k / (int)L->cols, col = k - row * (int)L->cols;
    const int64_t j = (int64_t)L->S[(int64_t)row * L->ld + col] - L->t0;
    if (j < 0 || j >= N) {
      bad = true;
      continue;
    }
    if (local) atomicAdd(&h[j], 1u);
    else atomicAdd(&L->counts[j], 1u);
  }
  if (bad) atomicExch(&L->scr->status, VL_ELOOKUP);
  __syncthreads();
  if (local)
    for (int j = threadIdx.x; j < N; j += blockDim.x)
      if (h[j]) atomicAdd(&L->counts[j], h[j]);
}

// Table entries [k0, k1) (at most 4 per thread): x_j = beta + t0 + j, its
// inverse by one batch inversion per block (prefix products, one field
// inversion, back substitution), the table-side vectors, and this block's
// share of X1 = sum B Ej T' and X2 = sum B m (slot: 12 Fr, the first two).
__global__ void __launch_bounds__(LK_THREADS) lk_table_kernel(LkDev* Ls, const LkItem* items) {
  __shared__ Fr pre[LK_THREADS], suf[LK_THREADS];
  __shared__ Fr inv_tot;
  __shared__ Fr red[2 * (LK_THREADS / 32)];
  const LkItem it = items[blockIdx.x];
  LkDev* L = Ls + it.proof;
  const int tid = threadIdx.x;
  const Fr beta = L->beta;
  Fr x[4], p[4];
  for (int e = 0; e < 4; e++) {
    const int j = it.k0 + 4 * tid + e;
    x[e] = j < it.k1 ? fr_add(beta, to_mont(fr_from_i64(L->t0 + j))) : fr_r1();
    p[e] = e == 0 ? x[0] : mont_mul(p[e - 1], x[e]);
  }
  // inclusive prefix and suffix products of the thread totals (Hillis-Steele)
  pre[tid] = p[3];
  suf[tid] = p[3];
  __syncthreads();
  for (int off = 1; off < LK_THREADS; off <<= 1) {
    const Fr a = tid >= off ? mont_mul(pre[tid - off], pre[tid]) : pre[tid];
    const Fr b = tid + off < LK_THREADS ? mont_mul(suf[tid], suf[tid + off]) : suf[tid];
    __syncthreads();
    pre[tid] = a;
    suf[tid] = b;
    __syncthreads();
  }
  if (tid == 0) inv_tot = fr_inv_mont(pre[LK_THREADS - 1]);
  __syncthreads();
  if (fr_is_zero(inv_tot)) {  // beta + t0 + j = 0 for some j (probability ~2^-239)
    if (tid == 0) atomicExch(&L->scr->status, VL_ELOOKUP);
    return;
  }
  const Fr qprev = tid > 0 ? pre[tid - 1] : fr_r1();
  // 1 / (prefix through this thread) = inv_tot . (product of the later threads' totals)
  Fr inv_f = tid + 1 < LK_THREADS ? mont_mul(inv_tot, suf[tid + 1]) : inv_tot;
  Fr inv_x[4];
  for (int e = 3; e >= 0; e--) {
    const Fr f_before = e > 0 ? mont_mul(qprev, p[e - 1]) : qprev;  // prefix before element e
    inv_x[e] = mont_mul(inv_f, f_before);
    inv_f = mont_mul(inv_f, x[e]);
  }
  Fr acc[2] = {fr_zero(), fr_zero()};
  for (int e = 0; e < 4; e++) {
    const int j = it.k0 + 4 * tid + e;
    if (j >= it.k1) break;
    const Fr m = to_mont(fr_small(L->counts[j]));
    L->Binv[j] = inv_x[e];
    L->WB[j] = inv_x[e];
    L->Tb[j] = x[e];
    L->WT[j] = x[e];
    L->WM[j] = m;
    acc[0] = fr_add(acc[0], mont_mul(mont_mul(inv_x[e], L->WE[j]), x[e]));
    acc[1] = fr_add(acc[1], mont_mul(inv_x[e], m));
  }
  block_sum_fr<2>(acc, red);
  if (tid == 0) {
    L->part[(size_t)it.slot * 12] = acc[0];
    L->part[(size_t)it.slot * 12 + 1] = acc[1];
  }
}

// The round polynomial of round t from the summed partials, by warp 0 (the
// sums valid in all its lanes): g(X) = alpha c_t eqf(u_t, X) T_X + A_X +
// table side for X = 0, 2, 3 by lanes 0..2 at once (the scalars they share
// formed in each), g(1) = claim - g(0); lanes 0..3 convert the four values
// for the proof; lane 0 absorbs ('g': g0, g2, g3) into Sw.  gsh[0..3]: the
// values (Montgomery), for lk_step_r.
__device__ void lk_step_g(LkDev* L, int t, const Fr (&acc)[6], const Fr (&accb)[6], bool jr, vl_lookup_proof* out,
                          Fr* gsh, uint32_t* Sw) {
  const int lane = threadIdx.x & 31, q = lane < 3 ? lane : 0;
  // eqf(u_t, X) for X = 0, 2, 3: eqf(u, X) = (1 - u) + X (2u - 1)
  const Fr ut = L->u[t - 1], one = fr_r1();
  const Fr e0 = fr_sub(one, ut), d = fr_sub(fr_add(ut, ut), one);
  const Fr eq = q == 0 ? e0 : (q == 1 ? fr_add(e0, fr_add(d, d)) : fr_add(fr_add(e0, fr_add(d, d)), d));
  const Fr half_t = L->half_t;
  Fr gq = fr_zero(), ht = fr_zero();
  if (lane < 3) {
    const Fr alpha = L->alpha;
    Fr tab;
    if (jr) {  // (N/D) (alpha^2 c'_t eqf(u_t, X) U_X - V_X)
      const Fr ac2 = mont_mul_ni(mont_mul_ni(alpha, alpha), L->ctj);
      tab = mont_mul_ni(L->c_nd, fr_sub(mont_mul_ni(mont_mul_ni(ac2, eq), accb[q]), accb[3 + q]));
    } else {
      ht = mont_mul_ni(half_t, L->inv2);
      tab = mont_mul_ni(ht, L->Cb);
    }
    const Fr ac = mont_mul_ni(alpha, L->ct);
    gq = fr_add(fr_add(mont_mul_ni(mont_mul_ni(ac, eq), acc[q]), acc[3 + q]), tab);
  }
  __syncwarp();
  if (!jr && lane == 0) L->half_t = ht;
  Fr G[4];
#pragma unroll
  for (int l = 0; l < 8; l++) {
    G[0].v[l] = __shfl_sync(0xffffffffu, gq.v[l], 0);
    G[2].v[l] = __shfl_sync(0xffffffffu, gq.v[l], 1);
    G[3].v[l] = __shfl_sync(0xffffffffu, gq.v[l], 2);
  }
  G[1] = fr_sub(L->claim, G[0]);
  const Fr mine = lane == 0 ? G[0] : (lane == 1 ? G[1] : (lane == 2 ? G[2] : G[3]));
  Fr c = fr_zero();
  if (lane < 4) {
    c = from_mont_ni(mine);
    for (int l = 0; l < 8; l++) out->g[t - 1][lane].limb[l] = c.v[l];
    gsh[lane] = mine;
  }
  Fr gc[3];
#pragma unroll
  for (int l = 0; l < 8; l++) {
    gc[0].v[l] = __shfl_sync(0xffffffffu, c.v[l], 0);
    gc[1].v[l] = __shfl_sync(0xffffffffu, c.v[l], 2);
    gc[2].v[l] = __shfl_sync(0xffffffffu, c.v[l], 3);
  }
  if (lane == 0) {
    uint32_t S[8];
    for (int i = 0; i < 8; i++) S[i] = L->St[i];
    dev_absorb_fr<3>(S, LBL_G, gc);
    for (int i = 0; i < 8; i++) Sw[i] = S[i];
  }
  __syncwarp();
}

// After the squeeze of r_t, by warp 0: store r_t and the state, fold c_t
// (and c'_t for a table variable) by eqf(u_t, r_t), and the new claim
// g(r_t) = sum_i g(i) L_i(r_t) over the nodes 0..3, lane i forming L_i and
// its term (the same products as a serial evaluation, in another order).
__device__ void lk_step_r(LkDev* L, int t, const Fr& r, const uint32_t* Sn, const Fr* gsh) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    L->r[t - 1] = r;
    for (int i = 0; i < 8; i++) L->St[i] = Sn[i];
  }
  const Fr ut = L->u[t - 1], one = fr_r1();
  // eqf(u_t, r) = u r + (1 - u)(1 - r): the two products on lanes 0, 1
  Fr part = fr_zero();
  if (lane < 2) part = lane == 0 ? mont_mul_ni(ut, r) : mont_mul_ni(fr_sub(one, ut), fr_sub(one, r));
  Fr ef;
#pragma unroll
  for (int l = 0; l < 8; l++) ef.v[l] = __shfl_sync(0xffffffffu, part.v[l], 1);
  ef = fr_add(part, ef);  // valid in lane 0
#pragma unroll
  for (int l = 0; l < 8; l++) ef.v[l] = __shfl_sync(0xffffffffu, ef.v[l], 0);
  const bool tabvar = t > L->L - L->log2_n;
  if (lane == 0) L->ct = mont_mul_ni(L->ct, ef);
  if (lane == 1 && tabvar) L->ctj = mont_mul_ni(L->ctj, ef);
  // Lagrange weights over the nodes 0..3 at r:
  //   L0 = -(r-1)(r-2)(r-3)/6, L1 = r(r-2)(r-3)/2, L2 = -r(r-1)(r-3)/2, L3 = r(r-1)(r-2)/6
  const Fr two = fr_add(one, one), three = fr_add(two, one);
  const Fr r1 = fr_sub(r, one), r2 = fr_sub(r, two), r3 = fr_sub(r, three);
  Fr term = fr_zero();
  if (lane < 4) {
    const Fr x = lane == 0 ? r1 : r, y = lane == 1 ? r2 : (lane == 0 ? r2 : r1);
    const Fr z = lane == 3 ? r2 : r3;
    const Fr inv = (lane == 0 || lane == 3) ? L->inv6 : L->inv2;
    Fr li = mont_mul_ni(mont_mul_ni(mont_mul_ni(x, y), z), inv);
    if (lane == 0 || lane == 2) li = fr_neg(li);
    term = mont_mul_ni(gsh[lane], li);
  }
  Fr t1, t2, t3;
#pragma unroll
  for (int l = 0; l < 8; l++) {
    t1.v[l] = __shfl_sync(0xffffffffu, term.v[l], 1);
    t2.v[l] = __shfl_sync(0xffffffffu, term.v[l], 2);
    t3.v[l] = __shfl_sync(0xffffffffu, term.v[l], 3);
  }
  if (lane == 0) L->claim = fr_add(fr_add(fr_add(term, t1), t2), t3);
  __syncwarp();
}

// The table side's cube sum Cb = alpha^2 X1 - X2 from the table kernel's
// partials (block-wide).
__device__ void lk_table_sum(LkDev* L, Fr* red) {
  Fr x[2] = {fr_zero(), fr_zero()};
  for (int s = L->xbeg + threadIdx.x; s < L->xend; s += blockDim.x) {
    x[0] = fr_add(x[0], L->part[(size_t)s * 12]);
    x[1] = fr_add(x[1], L->part[(size_t)s * 12 + 1]);
  }
  block_sum_fr<2>(x, red);
  if (threadIdx.x == 0) L->Cb = fr_sub(mont_mul_ni(mont_mul_ni(L->alpha, L->alpha), x[0]), x[1]);
  __syncthreads();
}

// Round t of one proof before its tail (one block each): the round
// polynomial from the partial sums, absorb, squeeze r_t, new claim.
__global__ void __launch_bounds__(LK_ROUND_THREADS) lk_round_kernel(LkDev* Ls, int t, vl_lookup_proof* outs) {
  __shared__ Fr red[6 * (LK_ROUND_THREADS / 32)];
  __shared__ uint32_t Sw[8], Sn[8];
  __shared__ uint32_t dig[3][8];
  __shared__ Fr rch[1];
  __shared__ Fr gsh[4];
  LkDev* L = Ls + blockIdx.x;
  if (t >= L->tail) return;
  const int tid = threadIdx.x;
  const bool jr = t > L->L - L->log2_n;
  if (t == 1) lk_table_sum(L, red);
  Fr acc[6], accb[6];
  for (int i = 0; i < 6; i++) acc[i] = accb[i] = fr_zero();
  for (int s = L->pbeg[t] + tid; s < L->pend[t]; s += blockDim.x) {
    for (int i = 0; i < 6; i++) acc[i] = fr_add(acc[i], L->part[(size_t)s * 12 + i]);
    if (jr)
      for (int i = 0; i < 6; i++) accb[i] = fr_add(accb[i], L->part[(size_t)s * 12 + 6 + i]);
  }
  block_sum_fr<6>(acc, red);
  if (jr) block_sum_fr<6>(accb, red);
  if (tid < 32) lk_step_g(L, t, acc, accb, jr, outs + blockIdx.x, gsh, Sw);
  __syncthreads();
  squeeze_dev(Sw, LBL_R, 1, rch, Sn, dig);
  if (tid < 32) lk_step_r(L, t, rch[0], Sn, gsh);
}

// The final evaluations (the last pair folded with r_L), absorb 'f', the
// proof (thread 0; the other threads zero the unused rounds first).
__device__ void lk_finish(LkDev* L, vl_lookup_proof* out) {
  for (int i = threadIdx.x; i < (VL_LOOKUP_MAX_LOG_D - L->L) * 32; i += blockDim.x)  // unused rounds
    out->g[L->L + i / 32][(i / 8) & 3].limb[i & 7] = 0u;
  if (threadIdx.x != 0) return;
  Fr a, s, b, m;
  const int Lp = L->L;
  if (Lp == 0) {
    lk_level0(*L, 0, a, s);
  } else if (Lp == 1) {
    Fr a1, s1;
    lk_level0(*L, 0, a, s);
    lk_level0(*L, 1, a1, s1);
    a = lk_fold(a, a1, L->r[0]);
    s = lk_fold(s, s1, L->r[0]);
  } else {
    a = lk_fold(L->VA[0], L->VA[1], L->r[Lp - 1]);
    s = lk_fold(L->VS[0], L->VS[1], L->r[Lp - 1]);
  }
  if (L->log2_n == 0) {
    b = L->WB[0];
    m = L->WM[0];
  } else {
    b = lk_fold(L->WB[0], L->WB[1], L->r[Lp - 1]);
    m = lk_fold(L->WM[0], L->WM[1], L->r[Lp - 1]);
  }
  s = fr_sub(s, L->beta);
  const Fr fin[4] = {from_mont_ni(a), from_mont_ni(s), from_mont_ni(b), from_mont_ni(m)};
  uint32_t S[8];
  for (int i = 0; i < 8; i++) S[i] = L->St[i];
  dev_absorb_fr<4>(S, LBL_F, fin);
  out->n = L->n;
  out->log2_d = Lp;
  out->log2_n = L->log2_n;
  out->t0 = L->t0;
  for (int l = 0; l < 8; l++) {
    out->a_r.limb[l] = fin[0].v[l];
    out->s_r.limb[l] = fin[1].v[l];
    out->b_r.limb[l] = fin[2].v[l];
    out->m_r.limb[l] = fin[3].v[l];
  }
  for (int i = 0; i < 32; i++) out->state[i] = (uint8_t)(S[i >> 2] >> (24 - 8 * (i & 3)));
  out->status = L->scr->status;
}

// One block per proof: its rounds from L->tail on (at most 2^LK_TAIL_LOG
// pairs each), each a pass over the pairs, a block reduction and the
// transcript step in this block, then the final evaluations and the proof.
#ifndef LK_TAIL_MINB
#define LK_TAIL_MINB 4  // resident tail CTAs per SM the register budget allows
#endif
__global__ void __launch_bounds__(LK_TAIL_THREADS, LK_TAIL_MINB) lk_tail_kernel(LkDev* Ls, vl_lookup_proof* outs) {
  __shared__ Fr red[6 * (LK_TAIL_THREADS / 32)];
  __shared__ uint32_t Sw[8], Sn[8];
  __shared__ uint32_t dig[3][8];
  __shared__ Fr rch[1];
  __shared__ Fr gsh[4];
  LkDev* L = Ls + blockIdx.x;
  vl_lookup_proof* out = outs + blockIdx.x;
  const int tid = threadIdx.x;
  if (L->tail == 1 && L->L >= 1) lk_table_sum(L, red);
  for (int t = L->tail; t <= L->L; t++) {
    const int h = 1 << (L->L - t);
    const bool jr = t > L->L - L->log2_n;
    const int tj = t - (L->L - L->log2_n);
    const LkEq q(L, t);
    Fr acc[6], accb[6];
    for (int i = 0; i < 6; i++) acc[i] = accb[i] = fr_zero();
    for (int k = tid; k < h; k += blockDim.x) {
      Fr f = q.f_tab[k & q.f_mask];
      if (q.high) f = mont_mul_ni(f, q.hi_tab[k >> L->sE]);
      if (t == 1) lk_pair_a<0>(L, t, k, h, f, acc);
      else if (t == 2) lk_pair_a<1>(L, t, k, h, f, acc);
      else lk_pair_a<2>(L, t, k, h, f, acc);
      if (jr) lk_pair_b(L, t, tj, k, h, f, accb);
    }
    if (t == 1) lk_mode0_sums(acc);
    if (jr && tj == 1) lk_mode0_sums(accb);
    block_sum_fr<6>(acc, red);
    if (jr) block_sum_fr<6>(accb, red);
    if (tid < 32) lk_step_g(L, t, acc, accb, jr, out, gsh, Sw);
    __syncthreads();
    squeeze_dev(Sw, LBL_R, 1, rch, Sn, dig);
    if (tid < 32) lk_step_r(L, t, rch[0], Sn, gsh);
    __syncthreads();  // r_t and the folded vectors are visible to the next round
  }
  lk_finish(L, out);
}

}  // namespace

cudaError_t launch_lookup_setup(LkDev* Ls, int np, const LkItem* fac_items, int nfac, const LkItem* hist_items,
                                int nhist, const LkItem* tab_items, int ntab, cudaStream_t st) {
  lk_start_kernel<<<np, LK_THREADS, 0, st>>>(Ls);
  if (nfac) lk_factor_kernel<<<nfac, LK_THREADS, 0, st>>>(Ls, fac_items);
  if (nhist) lk_hist_kernel<<<nhist, LK_THREADS, 0, st>>>(Ls, hist_items);
  if (ntab) lk_table_kernel<<<ntab, LK_THREADS, 0, st>>>(Ls, tab_items);
  return cudaGetLastError();
}

cudaError_t launch_lookup_round(LkDev* Ls, int np, int t, const LkItem* items, int nhi, int nlo,
                                vl_lookup_proof* out, cudaStream_t st) {
  const cudaError_t e = launch_lookup_passes(Ls, t, items, nhi, nlo, st);
  if (e != cudaSuccess) return e;
  lk_round_kernel<<<np, LK_ROUND_THREADS, 0, st>>>(Ls, t, out);
  return cudaGetLastError();
}

cudaError_t launch_lookup_finish(LkDev* Ls, int np, vl_lookup_proof* out, cudaStream_t st) {
  lk_tail_kernel<<<np, LK_TAIL_THREADS, 0, st>>>(Ls, out);
  return cudaGetLastError();
}

}  // namespace vl
