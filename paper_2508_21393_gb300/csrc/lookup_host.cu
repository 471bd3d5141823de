// Host engine and C ABI of the lookup-argument prover (Protocol 1, Eq.
// eq:lookup-sumcheck) for range tables, batched: one plan holds the
// statements, the workspace layout and the work-item tables; a run enqueues
// the host-operand copies, the multiplicity clear and 6 + 3 per round
// launches on the caller's stream (see kernels_lookup.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "common.cuh"
#include "abi_guard.h"

using namespace vl;

namespace {

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

int ceil_log2(int64_t x) {
  int d = 0;
  while ((int64_t(1) << d) < x) d++;
  return d;
}

constexpr int LK_MAX_JOBS = 65535;
constexpr int64_t LK_MAX_T0 = int64_t(1) << 40;

int check_job(const vl_lookup_job& J) {
  const vl_mat& M = J.S;
  if (J.reserved != 0 || J.log2_n < 0 || J.log2_n > VL_LOOKUP_MAX_LOG_N) return VL_EINVAL;
  if (J.t0 < -LK_MAX_T0 || J.t0 > LK_MAX_T0) return VL_EINVAL;
  if (!M.data || M.dtype != VL_I16 || M.trans != 0 || M.reserved != 0) return VL_EINVAL;
  if (M.space != VL_DEVICE && M.space != VL_HOST) return VL_EINVAL;
  if (M.rows < 1 || M.cols < 1) return VL_ESHAPE;
  if (M.ld < M.cols) return VL_EINVAL;
  const int64_t maxd = int64_t(1) << VL_LOOKUP_MAX_LOG_D;
  if (M.rows > maxd || M.cols > maxd || M.rows * M.cols > maxd) return VL_ESHAPE;  // no overflow: each <= 2^24
  return VL_OK;
}

struct LkBufs {
  size_t lop = 0, hip = 0, binv = 0, tb = 0, wb = 0, we = 0, wt = 0, wm = 0, va = 0, vs = 0, counts = 0, stage = 0;
};

int cuda_fail(const char* where, cudaError_t e) {
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", where, cudaGetErrorString(e));
  set_last_error(msg);
  return VL_ECUDA;
}

}  // namespace

struct vl_lookup_plan {
  std::vector<vl_lookup_job> jobs;
  int np = 0, maxL = 0, nslots = 0, nrounds = 0;
  std::vector<LkDev> Ls;  // statements; device pointers filled at bind time
  std::vector<LkBufs> buf;
  std::vector<LkItem> fac, hist, tab, rounds;
  std::vector<int> roff, nhi, nlo;  // round t: items [roff[t], roff[t] + nhi[t] + nlo[t])
  size_t off_L = 0, off_scr = 0, off_fac = 0, off_hist = 0, off_tab = 0, off_rounds = 0, off_part = 0,
         off_out = 0, off_counts = 0, counts_bytes = 0, total = 0;
  uint8_t* bound_ws = nullptr;
  int device = -1;
  cudaEvent_t ev[4] = {};
  bool timed = false;
  ~vl_lookup_plan() {
    for (cudaEvent_t& x : ev)
      if (x) cudaEventDestroy(x);
    ws_release(this);
  }
};

namespace {

int lk_build(vl_lookup_plan* P, const vl_lookup_job* jobs, int32_t njobs) {
  if (!jobs || njobs < 1 || njobs > LK_MAX_JOBS) return VL_EINVAL;
  for (int i = 0; i < njobs; i++) {
    const int e = check_job(jobs[i]);
    if (e != VL_OK) return e;
  }
  P->jobs.assign(jobs, jobs + njobs);
  P->np = njobs;
  P->Ls.assign(njobs, LkDev{});
  P->buf.assign(njobs, LkBufs{});
  const Fr inv2 = to_mont(fr_inv_canonical(fr_small(2))), inv6 = to_mont(fr_inv_canonical(fr_small(6)));
  int slot = 0;
  for (int i = 0; i < njobs; i++) {
    const vl_lookup_job& J = jobs[i];
    LkDev& L = P->Ls[i];
    std::memset(&L, 0, sizeof(L));
    const int64_t n = J.S.rows * J.S.cols;
    L.n = (int)n;
    L.log2_n = J.log2_n;
    L.L = std::max(J.log2_n, ceil_log2(n));
    L.sE = (L.L + 1) >> 1;
    L.t0 = J.t0;
    L.seed = J.seed;
    L.rows = J.S.rows;
    L.cols = J.S.cols;
    L.ld = J.S.space == VL_HOST ? J.S.cols : J.S.ld;  // host operands are staged densely
    std::memcpy(L.bind, J.bind, 32);
    L.inv2 = inv2;
    L.inv6 = inv6;
    L.tail = std::max(1, L.L - LK_TAIL_LOG);  // rounds with h = 2^(L-t) <= 2^LK_TAIL_LOG pairs
    if (L.L == 0) L.tail = 1;
    P->maxL = std::max(P->maxL, L.L);
    const int N = 1 << L.log2_n;
    // suffix eq tables (loP: levels 0..sE; hiP: levels 0..L-sE-1) and eq(u_low, .)
    const int sizes[3] = {(2 << L.sE) - 1, (1 << (L.L - L.sE)) - 1, N};
    for (int w = 0; w < 3; w++)
      for (int k0 = 0; k0 < sizes[w]; k0 += LK_THREADS * 4)
        P->fac.push_back(LkItem{i, k0, std::min(sizes[w], k0 + LK_THREADS * 4), w});
    for (int k0 = 0; k0 < L.n; k0 += LK_HIST) P->hist.push_back(LkItem{i, k0, std::min(L.n, k0 + LK_HIST), 0});
    L.xbeg = slot;
    for (int k0 = 0; k0 < N; k0 += LK_ENTRIES) P->tab.push_back(LkItem{i, k0, std::min(N, k0 + LK_ENTRIES), slot++});
    L.xend = slot;
  }
  // round items: per round, proofs in their high rounds first, then table rounds
  P->roff.assign(P->maxL + 2, 0);
  P->nhi.assign(P->maxL + 2, 0);
  P->nlo.assign(P->maxL + 2, 0);
  for (int t = 1; t <= P->maxL; t++) {
    P->roff[t] = (int)P->rounds.size();
    for (int pass = 0; pass < 2; pass++)
      for (int i = 0; i < njobs; i++) {
        LkDev& L = P->Ls[i];
        if (t >= L.tail) continue;  // the tail kernel runs this proof's later rounds
        const bool jr = t > L.L - L.log2_n;
        if (jr != (pass == 1)) continue;
        const int h = 1 << (L.L - t);
        L.pbeg[t] = slot;
        for (int k0 = 0; k0 < h; k0 += LK_PAIRS) {
          P->rounds.push_back(LkItem{i, k0, std::min(h, k0 + LK_PAIRS), slot++});
          (pass ? P->nlo : P->nhi)[t]++;
        }
        L.pend[t] = slot;
      }
  }
  P->nslots = slot;
  P->nrounds = 0;  // rounds before the tails
  for (const LkDev& L : P->Ls) P->nrounds = std::max(P->nrounds, L.tail - 1);
  // workspace layout
  size_t off = 0;
  auto take = [&off](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  P->off_L = take(sizeof(LkDev) * njobs);
  P->off_scr = take(sizeof(ProofScratch) * njobs);
  P->off_fac = take(sizeof(LkItem) * P->fac.size());
  P->off_hist = take(sizeof(LkItem) * P->hist.size());
  P->off_tab = take(sizeof(LkItem) * P->tab.size());
  P->off_rounds = take(sizeof(LkItem) * P->rounds.size());
  P->off_part = take(sizeof(Fr) * 12 * (size_t)std::max(1, P->nslots));
  P->off_out = take(sizeof(vl_lookup_proof) * njobs);
  // multiplicities of every proof in one region (one clear per run)
  size_t cnt = 0;
  for (int i = 0; i < njobs; i++) {
    P->buf[i].counts = cnt;
    cnt += sizeof(uint32_t) * ((size_t)1 << P->Ls[i].log2_n);
  }
  P->counts_bytes = cnt;
  P->off_counts = take(cnt);
  for (int i = 0; i < njobs; i++) {
    const LkDev& L = P->Ls[i];
    LkBufs& b = P->buf[i];
    const size_t N = (size_t)1 << L.log2_n, half = std::max<size_t>(1, ((size_t)1 << L.L) / 2);
    b.lop = take(sizeof(Fr) * ((2u << L.sE) - 1));
    b.hip = take(sizeof(Fr) * std::max<size_t>(1, (1u << (L.L - L.sE)) - 1));
    b.binv = take(sizeof(Fr) * N);
    b.tb = take(sizeof(Fr) * N);
    b.wb = take(sizeof(Fr) * N);
    b.we = take(sizeof(Fr) * N);
    b.wt = take(sizeof(Fr) * N);
    b.wm = take(sizeof(Fr) * N);
    b.va = take(sizeof(Fr) * half);
    b.vs = take(sizeof(Fr) * half);
    if (jobs[i].S.space == VL_HOST) b.stage = take(sizeof(int16_t) * (size_t)L.n);
  }
  P->total = off;
  return VL_OK;
}

int lk_bind(vl_lookup_plan* P, uint8_t* ws, cudaStream_t st) {
  for (int i = 0; i < P->np; i++) {
    LkDev& L = P->Ls[i];
    const LkBufs& b = P->buf[i];
    const vl_lookup_job& J = P->jobs[i];
    L.S = J.S.space == VL_HOST ? reinterpret_cast<const int16_t*>(ws + b.stage)
                               : static_cast<const int16_t*>(J.S.data);
    L.loP = reinterpret_cast<Fr*>(ws + b.lop);
    L.hiP = reinterpret_cast<Fr*>(ws + b.hip);
    L.Binv = reinterpret_cast<Fr*>(ws + b.binv);
    L.Tb = reinterpret_cast<Fr*>(ws + b.tb);
    L.WB = reinterpret_cast<Fr*>(ws + b.wb);
    L.WE = reinterpret_cast<Fr*>(ws + b.we);
    L.WT = reinterpret_cast<Fr*>(ws + b.wt);
    L.WM = reinterpret_cast<Fr*>(ws + b.wm);
    L.VA = reinterpret_cast<Fr*>(ws + b.va);
    L.VS = reinterpret_cast<Fr*>(ws + b.vs);
    L.counts = reinterpret_cast<uint32_t*>(ws + P->off_counts + b.counts);
    L.part = reinterpret_cast<Fr*>(ws + P->off_part);
    L.scr = reinterpret_cast<ProofScratch*>(ws + P->off_scr) + i;
  }
  cudaError_t ce = cudaSuccess;
  auto up = [&](size_t off, const void* src, size_t bytes) {
    if (ce == cudaSuccess && bytes) ce = cudaMemcpyAsync(ws + off, src, bytes, cudaMemcpyHostToDevice, st);
  };
  up(P->off_L, P->Ls.data(), sizeof(LkDev) * P->np);
  up(P->off_fac, P->fac.data(), sizeof(LkItem) * P->fac.size());
  up(P->off_hist, P->hist.data(), sizeof(LkItem) * P->hist.size());
  up(P->off_tab, P->tab.data(), sizeof(LkItem) * P->tab.size());
  up(P->off_rounds, P->rounds.data(), sizeof(LkItem) * P->rounds.size());
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);  // the host tables must outlive the copies
  if (ce != cudaSuccess) return cuda_fail("lookup proofs: bind", ce);
  P->bound_ws = ws;
  ws_claim(P, ws);
  return VL_OK;
}

cudaError_t lk_events(vl_lookup_plan* P) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev == P->device) return e;
  for (cudaEvent_t& x : P->ev)
    if (x) cudaEventDestroy(x), x = nullptr;
  for (cudaEvent_t& x : P->ev)
    if ((e = cudaEventCreate(&x)) != cudaSuccess) return e;
  P->device = dev;
  return cudaSuccess;
}

}  // namespace

extern "C" size_t vl_lookup_workspace_bytes(const vl_lookup_job* jobs, int32_t njobs) {
  VL_ABI_TRY
  vl_lookup_plan P;
  return lk_build(&P, jobs, njobs) == VL_OK ? P.total : 0;
  VL_ABI_CATCH(0)
}

extern "C" int32_t vl_lookup_plan_create(const vl_lookup_job* jobs, int32_t njobs, vl_lookup_plan** plan) {
  VL_ABI_TRY
  if (!plan) return VL_EINVAL;
  *plan = nullptr;
  std::unique_ptr<vl_lookup_plan> P(new (std::nothrow) vl_lookup_plan);
  if (!P) return VL_ENOMEM;
  const int e = lk_build(P.get(), jobs, njobs);
  if (e != VL_OK) return e;
  *plan = P.release();
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" size_t vl_lookup_plan_workspace_bytes(const vl_lookup_plan* plan) { return plan ? plan->total : 0; }

extern "C" int32_t vl_lookup_plan_run(vl_lookup_plan* P, void* workspace, size_t workspace_bytes,
                                      vl_lookup_proof* out, int32_t out_space, void* stream) {
  VL_ABI_TRY
  if (!P || !workspace || !out || (out_space != VL_DEVICE && out_space != VL_HOST)) return VL_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) & (ALIGN - 1)) return VL_EINVAL;
  if (workspace_bytes < P->total) return VL_ENOMEM;
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  P->timed = false;
  if (P->bound_ws != ws || !ws_owned_by(P, ws)) {  // first run here, or another plan used it
    const int e = lk_bind(P, ws, st);
    if (e != VL_OK) return e;
  }
  cudaError_t ce = lk_events(P);
  for (int i = 0; i < P->np && ce == cudaSuccess; i++) {
    const vl_lookup_job& J = P->jobs[i];
    if (J.S.space == VL_HOST)
      ce = cudaMemcpy2DAsync(ws + P->buf[i].stage, J.S.cols * 2, J.S.data, J.S.ld * 2, J.S.cols * 2, J.S.rows,
                             cudaMemcpyHostToDevice, st);
  }
  if (ce == cudaSuccess) ce = cudaMemsetAsync(ws + P->off_counts, 0, P->counts_bytes, st);
  LkDev* dL = reinterpret_cast<LkDev*>(ws + P->off_L);
  vl_lookup_proof* dout = out_space == VL_DEVICE ? out : reinterpret_cast<vl_lookup_proof*>(ws + P->off_out);
  auto items = [&](size_t off) { return reinterpret_cast<const LkItem*>(ws + off); };
  if (ce == cudaSuccess) ce = cudaEventRecord(P->ev[0], st);
  if (ce == cudaSuccess)
    ce = launch_lookup_setup(dL, P->np, items(P->off_fac), (int)P->fac.size(), items(P->off_hist),
                             (int)P->hist.size(), items(P->off_tab), (int)P->tab.size(), st);
  if (ce == cudaSuccess) ce = cudaEventRecord(P->ev[1], st);
  for (int t = 1; t <= P->nrounds && ce == cudaSuccess; t++)
    ce = launch_lookup_round(dL, P->np, t, items(P->off_rounds) + P->roff[t], P->nhi[t], P->nlo[t], dout, st);
  if (ce == cudaSuccess) ce = cudaEventRecord(P->ev[2], st);
  if (ce == cudaSuccess) ce = launch_lookup_finish(dL, P->np, dout, st);
  if (ce == cudaSuccess) ce = cudaEventRecord(P->ev[3], st);
  if (ce == cudaSuccess && out_space == VL_HOST) {
    ce = cudaMemcpyAsync(out, dout, sizeof(vl_lookup_proof) * P->np, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  }
  if (ce != cudaSuccess) return cuda_fail("vl_lookup_plan_run", ce);
  P->timed = true;
  if (out_space == VL_HOST)
    for (int i = 0; i < P->np; i++)
      if (out[i].status != VL_OK) return out[i].status;
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" int32_t vl_lookup_plan_phase_ms(vl_lookup_plan* P, float ms[3]) {
  if (!P || !ms || !P->timed) return VL_EINVAL;
  cudaError_t ce = cudaEventSynchronize(P->ev[3]);
  for (int i = 0; i < 3 && ce == cudaSuccess; i++) ce = cudaEventElapsedTime(&ms[i], P->ev[i], P->ev[i + 1]);
  return ce == cudaSuccess ? VL_OK : cuda_fail("vl_lookup_plan_phase_ms", ce);
}

extern "C" void vl_lookup_plan_destroy(vl_lookup_plan* plan) { delete plan; }

extern "C" int32_t vl_prove_lookup(const vl_lookup_job* jobs, int32_t njobs, void* workspace, size_t workspace_bytes,
                                   vl_lookup_proof* out, void* stream) {
  vl_lookup_plan* P = nullptr;
  int e = vl_lookup_plan_create(jobs, njobs, &P);
  if (e != VL_OK) return e;
  e = vl_lookup_plan_run(P, workspace, workspace_bytes, out, VL_HOST, stream);
  vl_lookup_plan_destroy(P);
  return e;
}
