// Device helpers of the lookup-argument kernels (kernels_lookup.cu: start,
// tables, transcript steps, tails; kernels_lookup_pass.cu: the batched round
// passes), shared by both translation units.  Their Montgomery products are
// the one out-of-line copy (mont_mul_ni): inlined, the ten to fifteen products
// of a pair made each kernel larger than the instruction cache (measured on
// the 7B remainder lookups: batched rounds 9.28 ms inlined, 7.90 ms out of
// line).
#pragma once
#include "prologue_dev.cuh"


namespace vl {

namespace {

constexpr uint8_t LBL_BETA = 'b', LBL_ALPHA = 'a';
constexpr int LK_ROUND_THREADS = 64;  // transcript step: a few partial sums and one serial hash chain
constexpr int LK_TAIL_THREADS = 128;  // a proof's last rounds: four blocks per SM

__device__ __forceinline__ int lk_table_index(const LkDev& L, int k) {
  if (k >= L.n) return 0;  // padding entries hold t0
  const int row = k / (int)L.cols, col = k - row * (int)L.cols;
  const int64_t v = (int64_t)L.S[(int64_t)row * L.ld + col];
  const int64_t j = v - L.t0;
  const int N = 1 << L.log2_n;
  return j < 0 ? 0 : (j >= N ? N - 1 : (int)j);  // out-of-table values were reported; stay in bounds
}

// A and S' at entry k of the unfolded cube.
__device__ __forceinline__ void lk_level0(const LkDev& L, int k, Fr& a, Fr& s) {
  const int j = lk_table_index(L, k);
  a = L.Binv[j];
  s = L.Tb[j];
}

__device__ __forceinline__ Fr lk_fold(const Fr& x0, const Fr& x1, const Fr& r) {
  return fr_add(x0, mont_mul_ni(r, fr_sub(x1, x0)));
}

// One pair (k, k + h) of round t, A side: fold A and S' with r_{t-1} (the
// first round reads the unfolded cube, the second folds it on the fly and
// writes the folded vectors, later rounds fold them in place), then add
// f (A S')(X) to acc[0..2] and A(X) to acc[3..5] for X = 0, 2, 3, where f =
// eq(u_{t+1..L}, k).  MODE: 0 = first round, 1 = second round, 2 = later.
template <int MODE>
__device__ __forceinline__ void lk_pair_a(LkDev* L, int t, int k, int h, const Fr& f, Fr (&acc)[6]) {
  Fr a0, a1, s0, s1;
  if constexpr (MODE == 0) {
    lk_level0(*L, k, a0, s0);
    lk_level0(*L, k + h, a1, s1);
    // Unfolded entries have A . S' = 1, so along the line through them
    // (A S')(X) = (1-X)^2 + X^2 + X(1-X) w with w = a1 s0 + a0 s1:
    // (A S')(0) = 1, (A S')(2) = 5 - 2w, (A S')(3) = 13 - 6w.  Sum f and f w
    // here; lk_mode0_sums forms the three sums.
    // a0 s0 = a1 s1 = 1, so w = (a0 + a1)(s0 + s1) - 2: one product
    const Fr w = fr_sub(mont_mul_ni(fr_add(a0, a1), fr_add(s0, s1)), fr_dbl(fr_r1()));
    acc[0] = fr_add(acc[0], f);
    acc[1] = fr_add(acc[1], mont_mul_ni(f, w));
  } else {
    if constexpr (MODE == 1) {
      const Fr r = L->r[0];
      Fr xa, xs, ya, ys;
      lk_level0(*L, k, xa, xs);
      lk_level0(*L, k + 2 * h, ya, ys);
      a0 = lk_fold(xa, ya, r);
      s0 = lk_fold(xs, ys, r);
      lk_level0(*L, k + h, xa, xs);
      lk_level0(*L, k + 3 * h, ya, ys);
      a1 = lk_fold(xa, ya, r);
      s1 = lk_fold(xs, ys, r);
    } else {
      const Fr r = L->r[t - 2];
      a0 = lk_fold(L->VA[k], L->VA[k + 2 * h], r);
      s0 = lk_fold(L->VS[k], L->VS[k + 2 * h], r);
      a1 = lk_fold(L->VA[k + h], L->VA[k + 3 * h], r);
      s1 = lk_fold(L->VS[k + h], L->VS[k + 3 * h], r);
    }
    L->VA[k] = a0, L->VS[k] = s0;
    L->VA[k + h] = a1, L->VS[k + h] = s1;
    const Fr ds = fr_sub(s1, s0), da = fr_sub(a1, a0);
    const Fr s2 = fr_add(s1, ds), a2 = fr_add(a1, da);
    const Fr s3 = fr_add(s2, ds), a3 = fr_add(a2, da);
    acc[0] = fr_add(acc[0], mont_mul_ni(f, mont_mul_ni(a0, s0)));
    acc[1] = fr_add(acc[1], mont_mul_ni(f, mont_mul_ni(a2, s2)));
    acc[2] = fr_add(acc[2], mont_mul_ni(f, mont_mul_ni(a3, s3)));
  }
  const Fr da = fr_sub(a1, a0);
  const Fr a2 = fr_add(a1, da), a3 = fr_add(a2, da);
  acc[3] = fr_add(acc[3], a0);
  acc[4] = fr_add(acc[4], a2);
  acc[5] = fr_add(acc[5], a3);
}

// First-round sums from (sum f, sum f w): T_0 = sum f, T_2 = 5 sum f - 2 sum f w,
// T_3 = 13 sum f - 6 sum f w (linear: valid per thread before the reduction).
__device__ __forceinline__ void lk_mode0_sums(Fr (&acc)[6]) {
  const Fr sf = acc[0], sw = acc[1];
  const Fr sw2 = fr_add(sw, sw), sf4 = fr_add(fr_add(sf, sf), fr_add(sf, sf));
  acc[1] = fr_sub(fr_add(sf4, sf), sw2);
  acc[2] = fr_sub(fr_add(fr_add(sf4, sf4), fr_add(sf4, sf)), fr_add(sw2, fr_add(sw2, sw2)));
}

// One pair of a table round (round tj of the last log2 N).  eq(u_low, .)
// folded by the bound table variables is c'_t eqf(u_t, X) eq(u_{t+1..L}, k),
// the A side's factor f times a scalar of the transcript step, so only B,
// T' and m are folded (in place after the first table round).  Adds
// f (B T')(X) to accb[0..2] and (B m)(X) to accb[3..5]; in the first table
// round B T' = 1 on the unfolded entries, so as for the A side only f and
// f w' (w' = b1 u0 + b0 u1) are summed (lk_mode0_sums forms the three).
__device__ __forceinline__ void lk_pair_b(LkDev* L, int t, int tj, int k, int h, const Fr& f, Fr (&accb)[6]) {
  Fr b0, b1, u0, u1, m0, m1;  // B, T', m
  if (tj == 1) {
    b0 = L->WB[k], b1 = L->WB[k + h];
    u0 = L->WT[k], u1 = L->WT[k + h];
    m0 = L->WM[k], m1 = L->WM[k + h];
    // b0 u0 = b1 u1 = 1, so w' = (b0 + b1)(u0 + u1) - 2: one product
    const Fr w = fr_sub(mont_mul_ni(fr_add(b0, b1), fr_add(u0, u1)), fr_dbl(fr_r1()));
    accb[0] = fr_add(accb[0], f);
    accb[1] = fr_add(accb[1], mont_mul_ni(f, w));
  } else {
    const Fr r = L->r[t - 2];
    b0 = lk_fold(L->WB[k], L->WB[k + 2 * h], r);
    u0 = lk_fold(L->WT[k], L->WT[k + 2 * h], r);
    m0 = lk_fold(L->WM[k], L->WM[k + 2 * h], r);
    b1 = lk_fold(L->WB[k + h], L->WB[k + 3 * h], r);
    u1 = lk_fold(L->WT[k + h], L->WT[k + 3 * h], r);
    m1 = lk_fold(L->WM[k + h], L->WM[k + 3 * h], r);
    L->WB[k] = b0, L->WT[k] = u0, L->WM[k] = m0;
    L->WB[k + h] = b1, L->WT[k + h] = u1, L->WM[k + h] = m1;
    const Fr du = fr_sub(u1, u0), db = fr_sub(b1, b0);
    const Fr u2 = fr_add(u1, du), b2 = fr_add(b1, db);
    const Fr u3 = fr_add(u2, du), b3 = fr_add(b2, db);
    accb[0] = fr_add(accb[0], mont_mul_ni(f, mont_mul_ni(b0, u0)));
    accb[1] = fr_add(accb[1], mont_mul_ni(f, mont_mul_ni(b2, u2)));
    accb[2] = fr_add(accb[2], mont_mul_ni(f, mont_mul_ni(b3, u3)));
  }
  const Fr db = fr_sub(b1, b0), dm = fr_sub(m1, m0);
  const Fr b2 = fr_add(b1, db), m2 = fr_add(m1, dm);
  const Fr b3 = fr_add(b2, db), m3 = fr_add(m2, dm);
  accb[3] = fr_add(accb[3], mont_mul_ni(b0, m0));
  accb[4] = fr_add(accb[4], mont_mul_ni(b2, m2));
  accb[5] = fr_add(accb[5], mont_mul_ni(b3, m3));
}

// Where round t reads eq(u_{t+1..L}, k): hiP[k >> sE] . loP_sE[k mod 2^sE]
// while t binds one of the first L - sE variables (high), loP_(L-t)[k] after.
struct LkEq {
  const Fr* f_tab;
  const Fr* hi_tab;
  int f_mask;
  bool high;
  __device__ LkEq(const LkDev* L, int t) {
    high = t <= L->L - L->sE;
    const int mask = (1 << L->sE) - 1;
    f_tab = high ? L->loP + mask : L->loP + (1 << (L->L - t)) - 1;
    f_mask = high ? mask : (1 << (L->L - t)) - 1;
    hi_tab = L->hiP + (high ? (1 << (L->L - L->sE - t)) - 1 : 0);
  }
};

}  // namespace

}  // namespace vl
