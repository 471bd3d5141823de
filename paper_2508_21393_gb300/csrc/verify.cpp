// Host verifier of one matmul sumcheck proof (the verifier of Def. def:ip,
// checked for completeness in Sec. V-B and soundness in Sec. V-A).
//
// It replays the transcript from the public statement (seed, dims, transpose
// flags, binds), re-derives u, v and every r_i, checks g_i(0) + g_i(1)
// against the running claim, evaluates g_i(r_i) by Lagrange interpolation
// through 0, 1, 2, checks the final claim a_r . b_r, the final transcript
// state, and evaluates A~(u, r), B~(r, v), C~(u, v) directly from the
// matrices (the stand-in for polynomial-commitment openings, Sec. II-A).
#include <algorithm>
#include <cstring>
#include <vector>

#include "fr.cuh"
#include "transcript.cuh"
#include "verilora.h"
#include "abi_guard.h"

using namespace vl;

namespace {

int ceil_log2(int64_t x) {
  int d = 0;
  while ((int64_t(1) << d) < x) d++;
  return d;
}

Fr fr_from_api(const vl_fr& x) {
  Fr a;
  for (int i = 0; i < 8; i++) a.v[i] = x.limb[i];
  return a;
}

// Entry (i, j) of op(M) as a canonical field element.
struct HostMat {
  const vl_mat* M;
  int64_t rows() const { return M->trans ? M->cols : M->rows; }
  int64_t cols() const { return M->trans ? M->rows : M->cols; }
  Fr at(int64_t i, int64_t j) const {
    const int64_t r = M->trans ? j : i, c = M->trans ? i : j;
    const int64_t idx = r * M->ld + c;
    switch (M->dtype) {
      case VL_I16: return fr_from_i64(static_cast<const int16_t*>(M->data)[idx]);
      case VL_I64: return fr_from_i64(static_cast<const int64_t*>(M->data)[idx]);
      default: return from_mont(static_cast<const Fr*>(M->data)[idx]);
    }
  }
};

// eq table in Montgomery form, MSB-first variables, `size` leading entries.
std::vector<Fr> eq_table(const std::vector<Fr>& x, int64_t size) {
  std::vector<Fr> t(1, fr_r1());
  for (size_t v = 0; v < x.size(); v++) {
    std::vector<Fr> n(t.size() * 2);
    const Fr one_minus = fr_sub(fr_r1(), x[v]);
    for (size_t j = 0; j < t.size(); j++) {
      n[2 * j] = mont_mul(t[j], one_minus);
      n[2 * j + 1] = mont_mul(t[j], x[v]);
    }
    t.swap(n);
  }
  t.resize((size_t)size);
  return t;
}

// M~(x, y) = sum_{i,j} eq(x, i) M[i, j] eq(y, j) (Montgomery result).
Fr mle_eval(const HostMat& M, const std::vector<Fr>& x, const std::vector<Fr>& y) {
  const std::vector<Fr> ex = eq_table(x, M.rows()), ey = eq_table(y, M.cols());
  Fr total = fr_zero();
  for (int64_t i = 0; i < M.rows(); i++) {
    Fr row = fr_zero();
    for (int64_t j = 0; j < M.cols(); j++) row = fr_add(row, mont_mul(to_mont(M.at(i, j)), ey[j]));
    total = fr_add(total, mont_mul(row, ex[i]));
  }
  return total;
}

Fr inv2_mont() {
  // (r + 1) / 2 for odd r.
  Fr h;
  uint32_t carry = 0;
  for (int i = 7; i >= 0; i--) {
    const uint32_t l = r_limb(i);
    h.v[i] = (l >> 1) | (carry << 31);
    carry = l & 1;
  }
  Fr one = fr_small(1);
  return to_mont(fr_add(h, one));
}

// g(x) through (0, g0), (1, g1), (2, g2); all Montgomery.
Fr interp(const Fr& g0, const Fr& g1, const Fr& g2, const Fr& x) {
  const Fr one = fr_r1(), two = fr_add(one, one), i2 = inv2_mont();
  const Fr xm1 = fr_sub(x, one), xm2 = fr_sub(x, two);
  const Fr l0 = mont_mul(mont_mul(xm1, xm2), i2);
  const Fr l1 = fr_neg(mont_mul(x, xm2));
  const Fr l2 = mont_mul(mont_mul(x, xm1), i2);
  return fr_add(fr_add(mont_mul(g0, l0), mont_mul(g1, l1)), mont_mul(g2, l2));
}

int check_host_mat(const vl_mat* M) {
  if (!M || !M->data) return VL_EINVAL;
  if (M->space != VL_HOST || M->reserved != 0) return VL_EINVAL;
  if (M->dtype != VL_I16 && M->dtype != VL_I64 && M->dtype != VL_FR_MONT) return VL_EINVAL;
  if (M->trans != 0 && M->trans != 1) return VL_EINVAL;
  if (M->rows < 1 || M->cols < 1) return VL_ESHAPE;
  if (M->ld < M->cols) return VL_EINVAL;
  return VL_OK;
}

}  // namespace

extern "C" int32_t vl_verify_matmul(const vl_mat* P, const vl_mat* Q, const vl_mat* C, const vl_fs_init* fs,
                                    const vl_proof* proof) {
  VL_ABI_TRY
  int e;
  if ((e = check_host_mat(P)) != VL_OK || (e = check_host_mat(Q)) != VL_OK || (e = check_host_mat(C)) != VL_OK)
    return e;
  if (!fs || !proof) return VL_EINVAL;
  const HostMat A{P}, B{Q}, Cm{C};
  const int64_t m = A.rows(), k = A.cols(), n = B.cols();
  if (B.rows() != k || Cm.rows() != m || Cm.cols() != n) return VL_ESHAPE;
  if (m > VL_MAX_REDUCE || n > VL_MAX_REDUCE || k > (int64_t(1) << VL_MAX_ROUNDS)) return VL_ESHAPE;
  const int d0 = ceil_log2(m), d1 = ceil_log2(k), d2 = ceil_log2(n);
  if (proof->m != m || proof->k != k || proof->n != n || proof->d0 != d0 || proof->d1 != d1 || proof->d2 != d2)
    return VL_REJECT;
  if (proof->status != VL_OK) return VL_REJECT;
  // Every transmitted element must be canonical.
  if (!lt_r(fr_from_api(proof->c)) || !lt_r(fr_from_api(proof->a_r)) || !lt_r(fr_from_api(proof->b_r)))
    return VL_REJECT;
  for (int i = 0; i < d1; i++)
    for (int q = 0; q < 3; q++)
      if (!lt_r(fr_from_api(proof->g[i][q]))) return VL_REJECT;

  uint8_t S[32];
  ts_start(S, fs->seed, (uint32_t)m, (uint32_t)k, (uint32_t)n, (uint32_t)P->trans, (uint32_t)Q->trans,
           &fs->bind[0][0]);
  std::vector<Fr> u(d0), v(d2), rs;
  for (int t = 0; t < d0; t++) u[t] = to_mont(ts_challenge(S, LBL_U, t));
  ts_squeeze_done(S, LBL_U, d0);
  for (int t = 0; t < d2; t++) v[t] = to_mont(ts_challenge(S, LBL_V, t));
  ts_squeeze_done(S, LBL_V, d2);

  const Fr c = fr_from_api(proof->c);
  if (!fr_eq(to_mont(c), mle_eval(Cm, u, v))) return VL_REJECT;
  ts_absorb_fr(S, LBL_C, &c, 1);
  Fr claim = to_mont(c);
  for (int i = 0; i < d1; i++) {
    const Fr g[3] = {fr_from_api(proof->g[i][0]), fr_from_api(proof->g[i][1]), fr_from_api(proof->g[i][2])};
    if (!fr_eq(fr_add(g[0], g[1]), from_mont(claim))) return VL_REJECT;
    const Fr g02[2] = {g[0], g[2]};  // g(1) is fixed by the claim
    ts_absorb_fr(S, LBL_G, g02, 2);
    const Fr r = to_mont(ts_challenge(S, LBL_R, 0));
    ts_squeeze_done(S, LBL_R, 1);
    rs.push_back(r);
    claim = interp(to_mont(g[0]), to_mont(g[1]), to_mont(g[2]), r);
  }
  const Fr ar = fr_from_api(proof->a_r), br = fr_from_api(proof->b_r);
  if (!fr_eq(claim, mont_mul(to_mont(ar), to_mont(br)))) return VL_REJECT;
  const Fr fin[2] = {ar, br};
  ts_absorb_fr(S, LBL_F, fin, 2);
  if (std::memcmp(S, proof->state, 32) != 0) return VL_REJECT;
  if (!fr_eq(to_mont(ar), mle_eval(A, u, rs))) return VL_REJECT;
  if (!fr_eq(to_mont(br), mle_eval(B, rs, v))) return VL_REJECT;
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

// Host verifier of a linear zkMat proof (sum_q c_q op(M_q) = 0, Sec. IV):
// replays the transcript from the statement, checks sum_q c_q e_q = 0 and the
// final state, and evaluates every M_q~(x, y) from the matrices.
extern "C" int32_t vl_verify_linear(const vl_lin_job* job, const vl_lin_proof* proof) {
  VL_ABI_TRY
  if (!job || !proof || !job->mats || !job->coeffs || job->nmats < 1 || job->nmats > VL_LIN_MAX || job->reserved)
    return VL_EINVAL;
  const vl_mat* mats = job->mats;
  const int nmats = job->nmats;
  const uint8_t* binds = job->binds;
  const uint64_t seed = job->seed;
  const vl_fr* coeffs = job->coeffs;
  int e;
  for (int q = 0; q < nmats; q++)
    if ((e = check_host_mat(&mats[q])) != VL_OK) return e;
  const int64_t rows = HostMat{&mats[0]}.rows(), cols = HostMat{&mats[0]}.cols();
  for (int q = 1; q < nmats; q++)
    if (HostMat{&mats[q]}.rows() != rows || HostMat{&mats[q]}.cols() != cols) return VL_ESHAPE;
  if (rows > VL_MAX_REDUCE || cols > VL_MAX_REDUCE) return VL_ESHAPE;
  std::vector<Fr> c(nmats);
  uint8_t bind[VL_LIN_MAX][32] = {};
  for (int q = 0; q < nmats; q++) {
    c[q] = fr_from_api(coeffs[q]);
    if (!lt_r(c[q])) return VL_EINVAL;
    if (binds) std::memcpy(bind[q], binds + 32 * q, 32);
  }
  const int d0 = ceil_log2(rows), d1 = ceil_log2(cols);
  if (proof->rows != rows || proof->cols != cols || proof->d0 != d0 || proof->d1 != d1 || proof->nmats != nmats)
    return VL_REJECT;
  if (proof->status != VL_OK) return VL_REJECT;
  std::vector<Fr> ev(nmats);
  for (int q = 0; q < nmats; q++) {
    ev[q] = fr_from_api(proof->evals[q]);
    if (!lt_r(ev[q])) return VL_REJECT;
  }
  uint8_t S[32];
  ts_start_linear(S, seed, (uint32_t)rows, (uint32_t)cols, nmats, c.data(), bind);
  std::vector<Fr> x(d0), y(d1);
  for (int t = 0; t < d0; t++) x[t] = to_mont(ts_challenge(S, 'x', t));
  ts_squeeze_done(S, 'x', d0);
  for (int t = 0; t < d1; t++) y[t] = to_mont(ts_challenge(S, 'y', t));
  ts_squeeze_done(S, 'y', d1);
  Fr sum = fr_zero();
  for (int q = 0; q < nmats; q++) sum = fr_add(sum, mont_mul(to_mont(c[q]), to_mont(ev[q])));
  if (!fr_is_zero(sum)) return VL_REJECT;
  ts_absorb_fr(S, 'e', ev.data(), nmats);
  if (std::memcmp(S, proof->state, 32) != 0) return VL_REJECT;
  for (int q = 0; q < nmats; q++)
    if (!fr_eq(to_mont(ev[q]), mle_eval(HostMat{&mats[q]}, x, y))) return VL_REJECT;
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

namespace {

// g(x) for the cubic through (0, g0) .. (3, g3) (Lagrange); Montgomery.
Fr cubic_interp(const Fr (&g)[4], const Fr& x) {
  const Fr one = fr_r1(), two = fr_add(one, one), three = fr_add(two, one);
  const Fr inv2 = to_mont(fr_inv_canonical(fr_small(2))), inv6 = to_mont(fr_inv_canonical(fr_small(6)));
  const Fr x1 = fr_sub(x, one), x2 = fr_sub(x, two), x3 = fr_sub(x, three);
  const Fr l0 = fr_neg(mont_mul(mont_mul(mont_mul(x1, x2), x3), inv6));
  const Fr l1 = mont_mul(mont_mul(mont_mul(x, x2), x3), inv2);
  const Fr l2 = fr_neg(mont_mul(mont_mul(mont_mul(x, x1), x3), inv2));
  const Fr l3 = mont_mul(mont_mul(mont_mul(x, x1), x2), inv6);
  return fr_add(fr_add(mont_mul(g[0], l0), mont_mul(g[1], l1)), fr_add(mont_mul(g[2], l2), mont_mul(g[3], l3)));
}

}  // namespace

// Host verifier of a lookup proof (Protocol 1, Eq. eq:lookup-sumcheck):
// replays the transcript, checks every round against the running claim and
// the final claim against the sent evaluations (eq(u, r), eq(u_low, r_low)
// and T~(r_low) computed here), then checks the evaluations against A, S, B
// and m recomputed from S and T (the stand-in for commitment openings).
extern "C" int32_t vl_verify_lookup(const vl_lookup_job* job, const vl_lookup_proof* proof) {
  VL_ABI_TRY
  if (!job || !proof) return VL_EINVAL;
  const vl_mat* M = &job->S;
  int e;
  if ((e = check_host_mat(M)) != VL_OK) return e;
  if (M->trans != 0 || M->dtype == VL_FR_MONT || job->reserved != 0) return VL_EINVAL;
  if (job->log2_n < 0 || job->log2_n > VL_LOOKUP_MAX_LOG_N) return VL_EINVAL;
  if (job->t0 < -(int64_t(1) << 40) || job->t0 > (int64_t(1) << 40)) return VL_EINVAL;  // the prover's bound
  const int64_t maxd = int64_t(1) << VL_LOOKUP_MAX_LOG_D;
  if (M->rows > maxd || M->cols > maxd || M->rows * M->cols > maxd) return VL_ESHAPE;
  const int64_t n = M->rows * M->cols;
  const int ln = job->log2_n, L = std::max(ln, ceil_log2(n));
  const int64_t N = int64_t(1) << ln, D = int64_t(1) << L, t0 = job->t0;
  if (proof->n != n || proof->log2_d != L || proof->log2_n != ln || proof->t0 != t0) return VL_REJECT;
  if (proof->status != VL_OK) return VL_REJECT;
  for (int t = 0; t < L; t++)
    for (int q = 0; q < 4; q++)
      if (!lt_r(fr_from_api(proof->g[t][q]))) return VL_REJECT;
  const Fr a_r = fr_from_api(proof->a_r), s_r = fr_from_api(proof->s_r), b_r = fr_from_api(proof->b_r),
           m_r = fr_from_api(proof->m_r);
  if (!lt_r(a_r) || !lt_r(s_r) || !lt_r(b_r) || !lt_r(m_r)) return VL_REJECT;
  // S padded with t0, as table indices; values outside the table reject
  std::vector<int32_t> idx((size_t)D, 0);
  std::vector<uint64_t> counts((size_t)N, 0);
  for (int64_t k = 0; k < D; k++) {
    int64_t v = t0;
    if (k < n) {
      const int64_t row = k / M->cols, col = k % M->cols, at = row * M->ld + col;
      v = M->dtype == VL_I16 ? static_cast<const int16_t*>(M->data)[at] : static_cast<const int64_t*>(M->data)[at];
    }
    if (v < t0 || v - t0 >= N) return VL_REJECT;
    idx[(size_t)k] = (int32_t)(v - t0);
    counts[(size_t)(v - t0)]++;
  }
  uint8_t S[32];
  ts_start_lookup(S, job->seed, (uint32_t)n, (uint32_t)L, (uint32_t)ln, t0, job->bind);
  const Fr beta = to_mont(ts_challenge(S, 'b', 0));
  ts_squeeze_done(S, 'b', 1);
  const Fr alpha = to_mont(ts_challenge(S, 'a', 0));
  ts_squeeze_done(S, 'a', 1);
  std::vector<Fr> u(L), r(L);
  for (int t = 0; t < L; t++) u[t] = to_mont(ts_challenge(S, 'u', t));
  ts_squeeze_done(S, 'u', L);
  Fr claim = fr_add(alpha, mont_mul(alpha, alpha));
  for (int t = 0; t < L; t++) {
    Fr g[4], gc[3];
    for (int q = 0; q < 4; q++) g[q] = to_mont(fr_from_api(proof->g[t][q]));
    if (!fr_eq(fr_add(g[0], g[1]), claim)) return VL_REJECT;
    gc[0] = fr_from_api(proof->g[t][0]);
    gc[1] = fr_from_api(proof->g[t][2]);
    gc[2] = fr_from_api(proof->g[t][3]);
    ts_absorb_fr(S, 'g', gc, 3);
    r[t] = to_mont(ts_challenge(S, 'r', 0));
    ts_squeeze_done(S, 'r', 1);
    claim = cubic_interp(g, r[t]);
  }
  // eq(u, r), eq(u_low, r_low), T~(r_low) = t0 + sum_t 2^(ln-1-t) r_low_t
  Fr e_r = fr_r1(), ej_r = fr_r1(), t_r = to_mont(fr_from_i64(t0)), w = fr_r1();
  for (int t = 0; t < L; t++) {
    const Fr f = fr_add(mont_mul(u[t], r[t]), mont_mul(fr_sub(fr_r1(), u[t]), fr_sub(fr_r1(), r[t])));
    e_r = mont_mul(e_r, f);
    if (t >= L - ln) ej_r = mont_mul(ej_r, f);
  }
  for (int t = L - 1; t >= L - ln; t--) {  // weights 1, 2, 4, .. from the least significant bit
    t_r = fr_add(t_r, mont_mul(w, r[t]));
    w = fr_add(w, w);
  }
  const Fr inv2 = to_mont(fr_inv_canonical(fr_small(2)));
  Fr c = fr_r1();
  for (int i = 0; i < L - ln; i++) c = mont_mul(c, inv2);
  const Fr am = to_mont(a_r), sm = to_mont(s_r), bm = to_mont(b_r), mm = to_mont(m_r);
  const Fr a2 = mont_mul(alpha, alpha);
  Fr fin = fr_add(mont_mul(mont_mul(mont_mul(alpha, am), e_r), fr_add(sm, beta)), am);
  const Fr tab = fr_sub(mont_mul(mont_mul(mont_mul(a2, bm), ej_r), fr_add(t_r, beta)), mont_mul(bm, mm));
  fin = fr_add(fin, mont_mul(c, tab));
  if (!fr_eq(fin, claim)) return VL_REJECT;
  const Fr f4[4] = {a_r, s_r, b_r, m_r};
  ts_absorb_fr(S, 'f', f4, 4);
  if (std::memcmp(S, proof->state, 32) != 0) return VL_REJECT;
  // Openings: B by one batch inversion, A gathered from B, eq tables by doubling.
  std::vector<Fr> B((size_t)N), pre((size_t)N);
  Fr acc = fr_r1();
  for (int64_t j = 0; j < N; j++) {
    B[(size_t)j] = fr_add(beta, to_mont(fr_from_i64(t0 + j)));
    acc = mont_mul(acc, B[(size_t)j]);
    pre[(size_t)j] = acc;
  }
  Fr inv = fr_inv_mont(acc);
  if (fr_is_zero(inv)) return VL_REJECT;
  for (int64_t j = N - 1; j >= 0; j--) {
    const Fr before = j > 0 ? pre[(size_t)j - 1] : fr_r1();
    const Fr x = B[(size_t)j];
    B[(size_t)j] = mont_mul(inv, before);
    inv = mont_mul(inv, x);
  }
  const std::vector<Fr> er = eq_table(r, D);
  const std::vector<Fr> rl(r.begin() + (L - ln), r.end());
  const std::vector<Fr> erl = eq_table(rl, N);
  Fr ea = fr_zero(), es = fr_zero(), eb = fr_zero(), em = fr_zero();
  for (int64_t k = 0; k < D; k++) {
    const int32_t j = idx[(size_t)k];
    ea = fr_add(ea, mont_mul(B[(size_t)j], er[(size_t)k]));
    es = fr_add(es, mont_mul(to_mont(fr_from_i64(t0 + j)), er[(size_t)k]));
  }
  for (int64_t j = 0; j < N; j++) {
    eb = fr_add(eb, mont_mul(B[(size_t)j], erl[(size_t)j]));
    em = fr_add(em, mont_mul(to_mont(fr_from_i64((int64_t)counts[(size_t)j])), erl[(size_t)j]));
  }
  if (!fr_eq(ea, am) || !fr_eq(es, sm) || !fr_eq(eb, bm) || !fr_eq(em, mm)) return VL_REJECT;
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

namespace {

// Root of the Merkle tree over 32-byte leaves, zero-padded to a power of two.
std::vector<uint8_t> merkle_root_host(std::vector<uint8_t> level, size_t nleaves) {
  size_t size = 1;
  while (size < nleaves) size <<= 1;
  level.resize(32 * size, 0);
  while (size > 1) {
    std::vector<uint8_t> next(32 * (size / 2));
    for (size_t j = 0; j < size / 2; j++) merkle_node(&next[32 * j], &level[64 * j], &level[64 * j + 32]);
    level.swap(next);
    size /= 2;
  }
  level.resize(32);
  return level;
}

}  // namespace

// Host verifier of a batched proof: member transcripts and claims (checked
// against the claimed products), the claims' root, rho, the rounds against
// the combined claim, the final combination, the final values' root and
// state, and the final values against the operands.
extern "C" int32_t vl_verify_matmul_batched(const vl_job* jobs, const vl_mat* C, int32_t njobs, uint64_t seed,
                                            const vl_batch_proof* proof, const vl_fr* claims, const vl_fr* a,
                                            const vl_fr* b) {
  VL_ABI_TRY
  if (!jobs || !C || !proof || !claims || !a || !b || njobs < 1 || njobs > 65535) return VL_EINVAL;
  int e;
  int64_t k = -1;
  for (int i = 0; i < njobs; i++) {
    if ((e = check_host_mat(&jobs[i].P)) != VL_OK || (e = check_host_mat(&jobs[i].Q)) != VL_OK ||
        (e = check_host_mat(&C[i])) != VL_OK)
      return e;
    const HostMat A{&jobs[i].P}, B{&jobs[i].Q}, Cm{&C[i]};
    if (A.cols() != B.rows() || Cm.rows() != A.rows() || Cm.cols() != B.cols()) return VL_ESHAPE;
    if (k < 0) k = A.cols();
    if (A.cols() != k) return VL_ESHAPE;
    if (A.rows() > VL_MAX_REDUCE || B.cols() > VL_MAX_REDUCE || k > (int64_t(1) << VL_MAX_ROUNDS)) return VL_ESHAPE;
  }
  const int d1 = ceil_log2(k);
  if (proof->K != njobs || proof->k != k || proof->d1 != d1 || proof->status != VL_OK) return VL_REJECT;
  for (int t = 0; t < d1; t++)
    for (int q = 0; q < 3; q++)
      if (!lt_r(fr_from_api(proof->g[t][q]))) return VL_REJECT;
  for (int i = 0; i < njobs; i++)
    if (!lt_r(fr_from_api(claims[i])) || !lt_r(fr_from_api(a[i])) || !lt_r(fr_from_api(b[i]))) return VL_REJECT;
  std::vector<std::vector<Fr>> us(njobs), vs(njobs);
  std::vector<uint8_t> leaves(32 * (size_t)njobs);
  for (int i = 0; i < njobs; i++) {
    const HostMat A{&jobs[i].P}, B{&jobs[i].Q};
    const int64_t m = A.rows(), n = B.cols();
    uint8_t S[32];
    ts_start_member(S, seed, (uint32_t)njobs, (uint32_t)i, (uint32_t)m, (uint32_t)k, (uint32_t)n,
                    (uint32_t)jobs[i].P.trans, (uint32_t)jobs[i].Q.trans, &jobs[i].fs.bind[0][0]);
    const int d0 = ceil_log2(m), d2 = ceil_log2(n);
    for (int t = 0; t < d0; t++) us[i].push_back(to_mont(ts_challenge(S, 'u', t)));
    ts_squeeze_done(S, 'u', d0);
    for (int t = 0; t < d2; t++) vs[i].push_back(to_mont(ts_challenge(S, 'v', t)));
    ts_squeeze_done(S, 'v', d2);
    const Fr c = fr_from_api(claims[i]);
    if (!fr_eq(to_mont(c), mle_eval(HostMat{&C[i]}, us[i], vs[i]))) return VL_REJECT;
    uint8_t cb[32];
    fr_to_le_bytes(c, cb);
    Sha256 h;
    h.init();
    h.byte(0);
    h.update(S, 32);
    h.update(cb, 32);
    h.finish(&leaves[32 * (size_t)i]);
  }
  const std::vector<uint8_t> root = merkle_root_host(leaves, njobs);
  uint8_t S[32];
  ts_start_batch(S, seed, (uint32_t)njobs, root.data());
  const Fr rho = to_mont(ts_challenge(S, 'p', 0));
  ts_squeeze_done(S, 'p', 1);
  std::vector<Fr> w(njobs);
  Fr claim = fr_zero(), pw = fr_r1();
  for (int i = 0; i < njobs; i++) {
    w[i] = pw;
    claim = fr_add(claim, mont_mul(pw, to_mont(fr_from_api(claims[i]))));
    pw = mont_mul(pw, rho);
  }
  std::vector<Fr> r;
  for (int t = 0; t < d1; t++) {
    const Fr g0 = to_mont(fr_from_api(proof->g[t][0])), g1 = to_mont(fr_from_api(proof->g[t][1])),
             g2 = to_mont(fr_from_api(proof->g[t][2]));
    if (!fr_eq(fr_add(g0, g1), claim)) return VL_REJECT;
    const Fr m2[2] = {fr_from_api(proof->g[t][0]), fr_from_api(proof->g[t][2])};
    ts_absorb_fr(S, 'g', m2, 2);
    r.push_back(to_mont(ts_challenge(S, 'r', 0)));
    ts_squeeze_done(S, 'r', 1);
    claim = interp(g0, g1, g2, r.back());
  }
  Fr fin = fr_zero();
  for (int i = 0; i < njobs; i++)
    fin = fr_add(fin, mont_mul(w[i], mont_mul(to_mont(fr_from_api(a[i])), to_mont(fr_from_api(b[i])))));
  if (!fr_eq(fin, claim)) return VL_REJECT;
  for (int i = 0; i < njobs; i++) {
    uint8_t ab[32], bb[32];
    fr_to_le_bytes(fr_from_api(a[i]), ab);
    fr_to_le_bytes(fr_from_api(b[i]), bb);
    Sha256 h;
    h.init();
    h.byte(0);
    h.u32le((uint32_t)i);
    h.update(ab, 32);
    h.update(bb, 32);
    h.finish(&leaves[32 * (size_t)i]);
  }
  const std::vector<uint8_t> root_f = merkle_root_host(leaves, njobs);
  {
    Sha256 h;
    h.init();
    h.update(S, 32);
    h.byte('f');
    h.update(root_f.data(), 32);
    h.finish(S);
  }
  if (std::memcmp(S, proof->state, 32) != 0) return VL_REJECT;
  for (int i = 0; i < njobs; i++) {
    if (!fr_eq(to_mont(fr_from_api(a[i])), mle_eval(HostMat{&jobs[i].P}, us[i], r))) return VL_REJECT;
    if (!fr_eq(to_mont(fr_from_api(b[i])), mle_eval(HostMat{&jobs[i].Q}, r, vs[i]))) return VL_REJECT;
  }
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

// Host verifier of a chained projection proof (Sec. IV, sequential
// composition; the protocol is written out in include/verilora.h): replays
// the chain transcript and every member's rounds, checks the output claims
// against the claimed outputs, each stage-3 claim against the claim the
// rescale relation derives from the claims on H and dH, and opens only X, W,
// A, B, dY and the remainders (evaluated directly from the matrices).
namespace {

int check_host_i16(const vl_mat& M, int64_t rows, int64_t cols) {
  const int e = check_host_mat(&M);
  if (e != VL_OK) return e;
  if (M.dtype == VL_FR_MONT || M.trans != 0) return VL_EINVAL;
  return (M.rows == rows && M.cols == cols) ? VL_OK : VL_ESHAPE;
}

void member_start_host(const uint8_t S[32], uint32_t p, uint8_t out[32]) {
  Sha256 h;
  h.init();
  h.update(S, 32);
  h.byte('M');
  h.u32le(p);
  h.finish(out);
}

// Replay one member's rounds from its start state; returns false on any
// failed check, the challenges in rs (Montgomery).
bool replay_member(const vl_proof& pf, const uint8_t start[32], int64_t m, int64_t k, int64_t n,
                   std::vector<Fr>* rs) {
  const int d0 = ceil_log2(m), d1 = ceil_log2(k), d2 = ceil_log2(n);
  if (pf.m != m || pf.k != k || pf.n != n || pf.d0 != d0 || pf.d1 != d1 || pf.d2 != d2) return false;
  if (pf.status != VL_OK) return false;
  if (!lt_r(fr_from_api(pf.c)) || !lt_r(fr_from_api(pf.a_r)) || !lt_r(fr_from_api(pf.b_r))) return false;
  for (int i = 0; i < d1; i++)
    for (int q = 0; q < 3; q++)
      if (!lt_r(fr_from_api(pf.g[i][q]))) return false;
  uint8_t S[32];
  std::memcpy(S, start, 32);
  const Fr c = fr_from_api(pf.c);
  ts_absorb_fr(S, LBL_C, &c, 1);
  Fr claim = to_mont(c);
  rs->clear();
  for (int i = 0; i < d1; i++) {
    const Fr g[3] = {fr_from_api(pf.g[i][0]), fr_from_api(pf.g[i][1]), fr_from_api(pf.g[i][2])};
    if (!fr_eq(fr_add(g[0], g[1]), from_mont(claim))) return false;
    const Fr g02[2] = {g[0], g[2]};
    ts_absorb_fr(S, LBL_G, g02, 2);
    const Fr r = to_mont(ts_challenge(S, LBL_R, 0));
    ts_squeeze_done(S, LBL_R, 1);
    rs->push_back(r);
    claim = interp(to_mont(g[0]), to_mont(g[1]), to_mont(g[2]), r);
  }
  const Fr ar = fr_from_api(pf.a_r), br = fr_from_api(pf.b_r);
  if (!fr_eq(claim, mont_mul(to_mont(ar), to_mont(br)))) return false;
  const Fr fin[2] = {ar, br};
  ts_absorb_fr(S, LBL_F, fin, 2);
  return std::memcmp(S, pf.state, 32) == 0;
}

// sum_{i < size} eq(x, i) (Montgomery)
Fr eq_sum(const std::vector<Fr>& x, int64_t size) {
  Fr s = fr_zero();
  for (const Fr& e : eq_table(x, size)) s = fr_add(s, e);
  return s;
}

bool opens(const vl_fr& val, const vl_mat& M, const std::vector<Fr>& x, const std::vector<Fr>& y) {
  return fr_eq(to_mont(fr_from_api(val)), mle_eval(HostMat{&M}, x, y));
}

}  // namespace

extern "C" int32_t vl_verify_chain(const vl_chain_job* job, const vl_mat* Y, const vl_mat* dX, const vl_mat* dA,
                                   const vl_mat* dB, const vl_chain_proof* proof) {
  VL_ABI_TRY
  if (!job || !Y || !dX || !dA || !dB || !proof) return VL_EINVAL;
  const vl_chain_job& J = *job;
  const int64_t n = J.X.rows, d = J.X.cols, k = J.W.cols, r = J.A.cols;
  if (n < 1 || d < 1 || k < 1 || r < 1) return VL_ESHAPE;
  if (n > VL_MAX_REDUCE || d > VL_MAX_REDUCE || k > VL_MAX_REDUCE || r > VL_CHAIN_MAX_RANK) return VL_ESHAPE;
  int e;
  if ((e = check_host_i16(J.X, n, d)) || (e = check_host_i16(J.W, d, k)) || (e = check_host_i16(J.A, d, r)) ||
      (e = check_host_i16(J.B, r, k)) || (e = check_host_i16(J.dY, n, k)) || (e = check_host_i16(J.rhoH, n, r)) ||
      (e = check_host_i16(J.rhodH, n, r)))
    return e;
  for (const vl_mat* M : {Y, dX, dA, dB})
    if ((e = check_host_mat(M)) != VL_OK) return e;
  if (Y->rows != n || Y->cols != k || dX->rows != n || dX->cols != d || dA->rows != d || dA->cols != r ||
      dB->rows != r || dB->cols != k || Y->trans || dX->trans || dA->trans || dB->trans)
    return VL_ESHAPE;
  if (proof->n != n || proof->d != d || proof->k != k || proof->r != r || proof->status != VL_OK) return VL_REJECT;
  for (int q = 0; q < 4; q++)
    if (!lt_r(fr_from_api(proof->e[q]))) return VL_REJECT;
  const int ln = ceil_log2(n), ld = ceil_log2(d), lk = ceil_log2(k), lr = ceil_log2(r);

  uint8_t S[32];
  {
    const uint8_t dom[25] = {'v', 'e', 'r', 'i', 'l', 'o', 'r', 'a', '-', 'g', 'b', '3', '0',
                             '0', '/', 'z', 'k', 'c', 'h', 'a', 'i', 'n', '/', 'v', '1'};
    Sha256 h;
    h.init();
    h.update(dom, 25);
    h.u32le((uint32_t)J.seed);
    h.u32le((uint32_t)(J.seed >> 32));
    for (int64_t v : {n, d, k, r}) h.u32le((uint32_t)v);
    h.update(&J.bind[0][0], 7 * 32);
    h.finish(S);
  }
  const int sz[8] = {ln, lk, ln, ld, ld, lr, lr, lk};
  std::vector<Fr> pt[8];
  uint32_t t = 0;
  for (int s = 0; s < 8; s++)
    for (int i = 0; i < sz[s]; i++) pt[s].push_back(to_mont(ts_challenge(S, 'p', t++)));
  ts_squeeze_done(S, 'p', t);
  const std::vector<Fr>&uY = pt[0], &vY = pt[1], &udX = pt[2], &vdX = pt[3], &udA = pt[4], &vdA = pt[5],
                      &udB = pt[6], &vdB = pt[7];
  // members: (m, k, n) of op(P) . op(Q)
  const int64_t shape[VL_CHAIN_MEMBERS][3] = {{n, d, k}, {n, r, k}, {n, k, d}, {n, r, d}, {d, n, r},
                                              {r, n, k}, {n, d, r}, {n, d, r}, {n, k, r}, {n, k, r}};
  std::vector<Fr> rs[VL_CHAIN_MEMBERS];
  uint8_t start[32];
  for (int p = 0; p < 6; p++) {
    member_start_host(S, (uint32_t)p, start);
    if (!replay_member(proof->sub[p], start, shape[p][0], shape[p][1], shape[p][2], &rs[p])) return VL_REJECT;
  }
  const vl_proof* sp = proof->sub;
  // output claims
  if (!fr_eq(to_mont(fr_add(fr_from_api(sp[0].c), fr_from_api(sp[1].c))), mle_eval(HostMat{Y}, uY, vY)))
    return VL_REJECT;
  if (!fr_eq(to_mont(fr_add(fr_from_api(sp[2].c), fr_from_api(sp[3].c))), mle_eval(HostMat{dX}, udX, vdX)))
    return VL_REJECT;
  if (!fr_eq(to_mont(fr_from_api(sp[4].c)), mle_eval(HostMat{dA}, udA, vdA))) return VL_REJECT;
  if (!fr_eq(to_mont(fr_from_api(sp[5].c)), mle_eval(HostMat{dB}, udB, vdB))) return VL_REJECT;
  // openings of the inputs where the stage-1 members end
  if (!opens(sp[0].a_r, J.X, uY, rs[0]) || !opens(sp[0].b_r, J.W, rs[0], vY) || !opens(sp[1].b_r, J.B, rs[1], vY) ||
      !opens(sp[2].a_r, J.dY, udX, rs[2]) || !opens(sp[2].b_r, J.W, vdX, rs[2]) ||
      !opens(sp[3].b_r, J.A, vdX, rs[3]) || !opens(sp[4].a_r, J.X, rs[4], udA) ||
      !opens(sp[5].b_r, J.dY, rs[5], vdB))
    return VL_REJECT;
  {
    Sha256 h;
    h.init();
    h.update(S, 32);
    h.byte('L');
    for (int p = 0; p < 6; p++) h.update(sp[p].state, 32);
    h.finish(S);
  }
  // the claims on H (p1, p2) and dH (q1, q2), and the remainders there
  const std::vector<Fr>* px[4] = {&uY, &rs[5], &udX, &rs[4]};
  const std::vector<Fr>* py[4] = {&rs[1], &udB, &rs[3], &vdA};
  const vl_fr* onH[4] = {&sp[1].a_r, &sp[5].a_r, &sp[3].a_r, &sp[4].b_r};
  Fr ev[4];
  for (int q = 0; q < 4; q++) {
    ev[q] = fr_from_api(proof->e[q]);
    if (!opens(proof->e[q], q < 2 ? J.rhoH : J.rhodH, *px[q], *py[q])) return VL_REJECT;
  }
  ts_absorb_fr(S, 'e', ev, 4);
  const Fr z = to_mont(fr_small(256)), half = to_mont(fr_small(128));
  for (int q = 0; q < 4; q++) {
    // (X.A)~ or (dY.B^T)~ at the point = 2^8 H~ + rho~ - 2^7 J~
    const Fr ones = mont_mul(eq_sum(*px[q], n), eq_sum(*py[q], r));
    const Fr want = fr_sub(fr_add(mont_mul(z, to_mont(fr_from_api(*onH[q]))), to_mont(ev[q])), mont_mul(half, ones));
    const vl_proof& m3 = sp[6 + q];
    if (!fr_eq(to_mont(fr_from_api(m3.c)), want)) return VL_REJECT;
    member_start_host(S, (uint32_t)(6 + q), start);
    if (!replay_member(m3, start, shape[6 + q][0], shape[6 + q][1], shape[6 + q][2], &rs[6 + q])) return VL_REJECT;
    const bool ok = q < 2 ? opens(m3.a_r, J.X, *px[q], rs[6 + q]) && opens(m3.b_r, J.A, rs[6 + q], *py[q])
                          : opens(m3.a_r, J.dY, *px[q], rs[6 + q]) && opens(m3.b_r, J.B, *py[q], rs[6 + q]);
    if (!ok) return VL_REJECT;
  }
  {
    Sha256 h;
    h.init();
    h.update(S, 32);
    h.byte('Z');
    for (int p = 6; p < VL_CHAIN_MEMBERS; p++) h.update(sp[p].state, 32);
    h.finish(S);
  }
  return std::memcmp(S, proof->state, 32) == 0 ? VL_OK : VL_REJECT;
  VL_ABI_CATCH(VL_ENOMEM)
}
