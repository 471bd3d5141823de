// Host engine and C ABI of the linear zkMat prover: sum_q c_q op(M_q) = 0
// entrywise, by MLE linearity at a transcript point (Sec. IV: zkMat covers
// matrix additions; the LoRA parameter update of Eq. eq:grad_update_ab is one
// such relation).
//
// One call proves a batch of relations with five launches on a caller-owned
// workspace: the start kernel (per proof: transcript, x and y, eq factors,
// offset correction), the eq-table kernel (chunks of every proof), the
// tensor-core fold of every matrix over its shorter logical dimension, the
// partial dot products against the other dimension's eq table, and the
// finish kernel (per proof: evaluations, absorb, proof); then one copy of the
// proofs to the host.  Reductions of at most LIN_SHORT_MAX entries (the LoRA
// factors' rank dimension) fold on CUDA cores instead of the tensor cores.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <memory>
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

// Fold tiles the segment choice aims for: two per SM of a 152-SM GB300.
constexpr int LIN_TILE_TARGET = 304;
// Shortest reduction segment worth a tile of its own.
constexpr int LIN_MIN_SEG = 1024;
// Longest segment whose digit sums stay exact (256 stages).
constexpr int LIN_MAX_SEG = 32768;
// Proofs per call (the partial-dot launch has one grid z index per proof).
constexpr int LIN_MAX_JOBS = 65535;

// Shape and fold plan of one proof.
struct LinShape {
  int rows = 0, cols = 0, d0 = 0, d1 = 0, q = 0;
  bool red_rows = true;
  bool shortf = false;  // reduction of at most LIN_SHORT_MAX entries: CUDA-core fold
  int red = 0, lines = 0, seg = 0, nsplit = 0, nblk = 0, ntiles = 0, nshort = 0;
};

// Workspace offsets of one proof's buffers.
struct LinBufs {
  size_t fac = 0, w8 = 0, f = 0, part = 0, e2 = 0;
};

struct LinLayout {
  int np = 0, nmats = 0, ntiles = 0, nshort = 0, max_nblk = 1, max_q = 1;
  std::vector<LinShape> shape;
  std::vector<LinBufs> buf;
  std::vector<EqItem> items;
  size_t off_L = 0, off_scr = 0, off_dp = 0, off_tiles = 0, off_short = 0, off_maps = 0, off_items = 0, off_out = 0,
         total = 0;
  std::vector<size_t> off_stage;  // per operand (flattened job by job); unused unless staged
  std::vector<int64_t> stage_ld;
  std::vector<char> staged;
};

int64_t lrows(const vl_mat& M) { return M.trans ? M.cols : M.rows; }
int64_t lcols(const vl_mat& M) { return M.trans ? M.rows : M.cols; }

// The fold reads the stored matrix with TMA: a device operand qualifies with
// a 16-byte aligned base and a leading dimension of a multiple of 8 entries;
// anything else is copied into the workspace first.
bool tma_ready(const vl_mat& M) {
  return M.space == VL_DEVICE && (reinterpret_cast<uintptr_t>(M.data) & 15) == 0 && (M.ld & 7) == 0;
}

int lin_shape(const vl_lin_job& J, LinShape* S) {
  if (!J.mats || !J.coeffs || J.nmats < 1 || J.nmats > VL_LIN_MAX || J.reserved != 0) return VL_EINVAL;
  const vl_mat* mats = J.mats;
  for (int q = 0; q < J.nmats; q++) {
    const vl_mat& M = mats[q];
    if (!M.data || M.dtype != VL_I16 || (M.trans != 0 && M.trans != 1) || M.reserved != 0) return VL_EINVAL;
    if (M.space != VL_DEVICE && M.space != VL_HOST) return VL_EINVAL;
    if (M.rows < 1 || M.cols < 1) return VL_ESHAPE;
    if (M.ld < M.cols) return VL_EINVAL;
    if (lrows(M) != lrows(mats[0]) || lcols(M) != lcols(mats[0])) return VL_ESHAPE;
  }
  const int64_t rows = lrows(mats[0]), cols = lcols(mats[0]);
  if (rows > VL_MAX_REDUCE || cols > VL_MAX_REDUCE) return VL_ESHAPE;
  S->rows = (int)rows;
  S->cols = (int)cols;
  S->d0 = ceil_log2(rows);
  S->d1 = ceil_log2(cols);
  S->q = J.nmats;
  // Reduce over the shorter dimension: the longer one gives the most tiles.
  S->red_rows = rows <= cols;
  S->red = (int)std::min(rows, cols);
  S->lines = (int)std::max(rows, cols);
  const int ntl = (S->lines + TC_M - 1) / TC_M;
  const int want = (LIN_TILE_TARGET + ntl - 1) / ntl;
  const int most = std::max(1, (S->red + LIN_MIN_SEG - 1) / LIN_MIN_SEG);
  const int least = (S->red + LIN_MAX_SEG - 1) / LIN_MAX_SEG;
  const int split = std::max(least, std::min(want, most));
  S->seg = ((S->red + split - 1) / split + TC_KS - 1) / TC_KS * TC_KS;
  S->nsplit = (S->red + S->seg - 1) / S->seg;
  S->ntiles = J.nmats * ntl * S->nsplit;
  // A short reduction would fill few entries of a tensor-core stage: fold it
  // on CUDA cores, one thread per line.
  S->shortf = S->red <= LIN_SHORT_MAX;
  if (S->shortf) {
    S->nsplit = 1;
    S->ntiles = 0;
    S->nshort = J.nmats * ((S->lines + LIN_SHORT_LINES - 1) / LIN_SHORT_LINES);
  }
  // inner sums of the lines side: blocks of 2^s lines, s = ceil(d / 2)
  const int dl = S->red_rows ? S->d1 : S->d0, sl = (dl + 1) >> 1;
  S->nblk = (S->lines + (1 << sl) - 1) >> sl;
  return VL_OK;
}

int lin_layout(const vl_lin_job* jobs, int32_t njobs, LinLayout* L) {
  if (!jobs || njobs < 1 || njobs > LIN_MAX_JOBS) return VL_EINVAL;
  L->np = njobs;
  L->shape.resize(njobs);
  L->buf.resize(njobs);
  for (int i = 0; i < njobs; i++) {
    const int e = lin_shape(jobs[i], &L->shape[i]);
    if (e != VL_OK) return e;
    const LinShape& S = L->shape[i];
    L->nmats += S.q;
    L->ntiles += S.ntiles;
    L->nshort += S.nshort;
    L->max_nblk = std::max(L->max_nblk, S.nblk);
    L->max_q = std::max(L->max_q, S.q);
    // chunks of the reduced side's eq table (padded to whole stages)
    const int rend = (S.red + TC_KS - 1) / TC_KS * TC_KS;
    for (int i0 = 0; i0 < rend; i0 += EQ_CHUNK) L->items.push_back(EqItem{i, 1, i0, std::min(rend, i0 + EQ_CHUNK)});
  }
  size_t off = 0;
  auto take = [&off](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  L->off_L = take(sizeof(LinDev) * njobs);
  L->off_scr = take(sizeof(ProofScratch) * njobs);
  L->off_dp = take(sizeof(DevProof) * njobs);
  L->off_tiles = take(sizeof(TcTile) * (size_t)L->ntiles);
  L->off_short = take(sizeof(LinShort) * (size_t)L->nshort);
  L->off_maps = take(sizeof(CUtensorMap) * (size_t)L->nmats);
  L->off_items = take(sizeof(EqItem) * L->items.size());
  L->off_out = take(sizeof(vl_lin_proof) * njobs);
  for (int i = 0; i < njobs; i++) {
    const LinShape& S = L->shape[i];
    LinBufs& b = L->buf[i];
    b.fac = take(sizeof(Fr) * 4 * EQ_FAC);
    b.w8 = take((size_t)8192 * ((S.red + TC_KS - 1) / TC_KS));
    // f (one segment per tile) or the column-sum accumulators (several)
    b.f = take((S.nsplit == 1 ? sizeof(Fr) : 8 * sizeof(unsigned long long)) * (size_t)S.q * S.lines);
    b.part = take(sizeof(Fr) * (size_t)S.q * S.nblk);
    b.e2 = S.shortf ? take(sizeof(Fr) * (size_t)S.red) : 0;
  }
  L->off_stage.assign(L->nmats, 0);
  L->stage_ld.assign(L->nmats, 0);
  L->staged.assign(L->nmats, 0);
  int g = 0;
  for (int i = 0; i < njobs; i++)
    for (int q = 0; q < jobs[i].nmats; q++, g++) {
      const vl_mat& M = jobs[i].mats[q];
      if (tma_ready(M)) continue;
      L->staged[g] = 1;
      L->stage_ld[g] = (M.cols + 7) & ~int64_t(7);
      L->off_stage[g] = take((size_t)M.rows * L->stage_ld[g] * 2);
    }
  L->total = off;
  return VL_OK;
}

int cuda_fail(const char* where, cudaError_t e) {
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", where, cudaGetErrorString(e));
  set_last_error(msg);
  return VL_ECUDA;
}

}  // namespace

// A batch of linear relations: the statements (copied), the workspace
// layout, and the device tables of the workspace it was last bound to.
struct vl_lin_plan {
  LinLayout lay;
  std::vector<std::vector<vl_mat>> mats;
  std::vector<LinDev> Ls;  // statements; device pointers filled at bind time
  std::vector<DevProof> dps;
  std::vector<CUtensorMap> maps;
  std::vector<TcTile> tiles;
  std::vector<LinShort> shorts;
  uint8_t* bound_ws = nullptr;
  int device = -1;
  cudaEvent_t ev[4] = {};
  bool timed = false;  // the events hold a run
  ~vl_lin_plan() {
    for (cudaEvent_t& x : ev)
      if (x) cudaEventDestroy(x);
    ws_release(this);
  }
};

namespace {

// Device pointers of workspace `ws` into the tables, tensor maps of the
// operands, fold tiles; uploaded on `st` (synchronised: the host tables
// must outlive the copies).
int lin_bind(vl_lin_plan* P, uint8_t* ws, cudaStream_t st) {
  const LinLayout& lay = P->lay;
  const int np = lay.np;
  LinDev* dL = reinterpret_cast<LinDev*>(ws + lay.off_L);
  for (int i = 0; i < np; i++) {
    const LinShape& S = lay.shape[i];
    const LinBufs& b = lay.buf[i];
    LinDev& L = P->Ls[i];
    L.fac = reinterpret_cast<Fr*>(ws + b.fac);
    L.w8 = reinterpret_cast<uint32_t*>(ws + b.w8);
    L.f = S.nsplit == 1 ? reinterpret_cast<Fr*>(ws + b.f) : nullptr;
    L.acc = S.nsplit == 1 ? nullptr : reinterpret_cast<unsigned long long*>(ws + b.f);
    L.part = reinterpret_cast<Fr*>(ws + b.part);
    L.e2 = S.shortf ? reinterpret_cast<Fr*>(ws + b.e2) : nullptr;
    L.scr = reinterpret_cast<ProofScratch*>(ws + lay.off_scr) + i;
    std::memset(&P->dps[i], 0, sizeof(DevProof));
    P->dps[i].scr = L.scr;  // the fold reports a timeout through this proof's status
  }
  P->maps.assign(lay.nmats, CUtensorMap{});
  P->tiles.clear();
  P->tiles.reserve(lay.ntiles);
  P->shorts.clear();
  P->shorts.reserve(lay.nshort);
  int g = 0;
  for (int i = 0; i < np; i++) {
    const LinShape& S = lay.shape[i];
    const LinDev& L = P->Ls[i];
    const int ntl = (S.lines + TC_M - 1) / TC_M;
    for (int q = 0; q < S.q; q++, g++) {
      const vl_mat& M = P->mats[i][q];
      const void* base = lay.staged[g] ? ws + lay.off_stage[g] : M.data;
      const int64_t ld = lay.staged[g] ? lay.stage_ld[g] : M.ld;
      // Column sums reduce over stored rows, row dots over stored columns.
      const int32_t mode = (S.red_rows != (M.trans != 0)) ? MODE_COLSUM : MODE_ROWDOT;
      if (S.shortf) {
        for (int w0 = 0; w0 < S.lines; w0 += LIN_SHORT_LINES) {
          LinShort it{};
          it.base = static_cast<const int16_t*>(base);
          it.ld = ld;
          it.proof = i;
          it.q = q;
          it.w0 = w0;
          it.nw = std::min(LIN_SHORT_LINES, S.lines - w0);
          it.mode = mode;
          it.red = S.red;
          P->shorts.push_back(it);
        }
        continue;
      }
      if (!encode_tc_operand(base, M.rows, M.cols, ld, mode, &P->maps[g])) {
        char msg[128];
        snprintf(msg, sizeof(msg), "linear proofs: tensor map of job %d matrix %d could not be encoded", i, q);
        set_last_error(msg);
        return VL_EINVAL;
      }
      for (int t = 0; t < ntl; t++)
        for (int k = 0; k < S.nsplit; k++) {
          TcTile tt{};
          tt.tmap = ws + lay.off_maps + (size_t)g * sizeof(CUtensorMap);
          tt.w8 = L.w8;
          tt.mode = mode;
          tt.w0 = t * TC_M;
          tt.nw = std::min(TC_M, S.lines - tt.w0);
          tt.k0 = k * S.seg;
          tt.nk = std::min(S.seg, S.red - tt.k0);
          tt.proof = i;
          tt.task = g;
          const size_t line = (size_t)q * S.lines + tt.w0;
          tt.acc = L.acc ? L.acc + line * 8 : nullptr;
          tt.f = L.acc ? nullptr : L.f + line;
          tt.corr = L.acc ? nullptr : &dL[i].corr;
          P->tiles.push_back(tt);
        }
    }
  }
  // Longest tiles first: the fold deals tiles to CTAs round robin.
  std::stable_sort(P->tiles.begin(), P->tiles.end(), [](const TcTile& a, const TcTile& b) { return a.nk > b.nk; });
  cudaError_t ce = cudaSuccess;
  auto up = [&](size_t off, const void* src, size_t bytes) {
    if (ce == cudaSuccess && bytes) ce = cudaMemcpyAsync(ws + off, src, bytes, cudaMemcpyHostToDevice, st);
  };
  up(lay.off_L, P->Ls.data(), sizeof(LinDev) * np);
  up(lay.off_dp, P->dps.data(), sizeof(DevProof) * np);
  up(lay.off_tiles, P->tiles.data(), sizeof(TcTile) * P->tiles.size());
  up(lay.off_short, P->shorts.data(), sizeof(LinShort) * P->shorts.size());
  up(lay.off_maps, P->maps.data(), sizeof(CUtensorMap) * P->maps.size());
  up(lay.off_items, lay.items.data(), sizeof(EqItem) * lay.items.size());
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce == cudaSuccess) ce = fold_tc_prepare();
  if (ce != cudaSuccess) return cuda_fail("linear proofs: bind", ce);
  P->bound_ws = ws;
  ws_claim(P, ws);
  return VL_OK;
}

cudaError_t lin_events(vl_lin_plan* P) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev == P->device) return e;
  for (cudaEvent_t& x : P->ev)
    if (x) cudaEventDestroy(x), x = nullptr;  // events of the previous device
  for (cudaEvent_t& x : P->ev)
    if ((e = cudaEventCreate(&x)) != cudaSuccess) return e;
  P->device = dev;
  return cudaSuccess;
}

}  // namespace

extern "C" size_t vl_linear_workspace_bytes(const vl_lin_job* jobs, int32_t njobs) {
  VL_ABI_TRY
  LinLayout L;
  return lin_layout(jobs, njobs, &L) == VL_OK ? L.total : 0;
  VL_ABI_CATCH(0)
}

extern "C" int32_t vl_lin_plan_create(const vl_lin_job* jobs, int32_t njobs, vl_lin_plan** plan) {
  VL_ABI_TRY
  if (!plan) return VL_EINVAL;
  *plan = nullptr;
  std::unique_ptr<vl_lin_plan> P(new (std::nothrow) vl_lin_plan);
  if (!P) return VL_ENOMEM;
  const int e = lin_layout(jobs, njobs, &P->lay);
  if (e != VL_OK) return e;
  P->mats.resize(njobs);
  P->Ls.assign(njobs, LinDev{});
  P->dps.assign(njobs, DevProof{});
  for (int i = 0; i < njobs; i++) {
    const vl_lin_job& J = jobs[i];
    const LinShape& S = P->lay.shape[i];
    LinDev& L = P->Ls[i];
    std::memset(&L, 0, sizeof(L));
    P->mats[i].assign(J.mats, J.mats + J.nmats);
    for (int q = 0; q < J.nmats; q++) {
      for (int l = 0; l < 8; l++) L.coeffs[q].v[l] = J.coeffs[q].limb[l];
      if (!lt_r(L.coeffs[q])) return VL_EINVAL;  // coefficients are canonical
      if (J.binds) std::memcpy(L.binds[q], J.binds + 32 * q, 32);
    }
    L.rows = S.rows;
    L.cols = S.cols;
    L.d0 = S.d0;
    L.d1 = S.d1;
    L.nmats = S.q;
    L.red_rows = S.red_rows ? 1 : 0;
    L.lines = S.lines;
    L.nblk = S.nblk;
    L.seed = J.seed;
  }
  *plan = P.release();
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" size_t vl_lin_plan_workspace_bytes(const vl_lin_plan* plan) { return plan ? plan->lay.total : 0; }

extern "C" int32_t vl_lin_plan_run(vl_lin_plan* P, void* workspace, size_t workspace_bytes, vl_lin_proof* out,
                                   int32_t out_space, void* stream) {
  VL_ABI_TRY
  if (!P || !workspace || !out || (out_space != VL_DEVICE && out_space != VL_HOST)) return VL_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) & (ALIGN - 1)) return VL_EINVAL;
  const LinLayout& lay = P->lay;
  if (workspace_bytes < lay.total) return VL_ENOMEM;
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  P->timed = false;
  if (P->bound_ws != ws || !ws_owned_by(P, ws)) {  // first run here, or another plan used it
    const int e = lin_bind(P, ws, st);
    if (e != VL_OK) return e;
  }
  cudaError_t ce = lin_events(P);
  // Operands that are not TMA-addressable in place: copied every run.
  int g = 0;
  for (int i = 0; i < lay.np && ce == cudaSuccess; i++)
    for (const vl_mat& M : P->mats[i]) {
      if (lay.staged[g] && ce == cudaSuccess)
        ce = cudaMemcpy2DAsync(ws + lay.off_stage[g], lay.stage_ld[g] * 2, M.data, M.ld * 2, M.cols * 2, M.rows,
                               M.space == VL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
      g++;
    }
  for (int i = 0; i < lay.np && ce == cudaSuccess; i++) {
    const LinDev& L = P->Ls[i];
    if (L.acc) ce = cudaMemsetAsync(L.acc, 0, sizeof(unsigned long long) * 8 * (size_t)L.nmats * L.lines, st);
  }
  LinDev* dL = reinterpret_cast<LinDev*>(ws + lay.off_L);
  vl_lin_proof* dout = out_space == VL_DEVICE ? out : reinterpret_cast<vl_lin_proof*>(ws + lay.off_out);
  cudaEvent_t* ev = P->ev;
  if (ce == cudaSuccess) ce = cudaEventRecord(ev[0], st);
  if (ce == cudaSuccess)
    ce = launch_linear_start(dL, lay.np, reinterpret_cast<const EqItem*>(ws + lay.off_items), (int)lay.items.size(),
                             st);
  if (ce == cudaSuccess) ce = cudaEventRecord(ev[1], st);
  if (ce == cudaSuccess && lay.ntiles > 0)
    ce = launch_fold_tc(reinterpret_cast<const TcTile*>(ws + lay.off_tiles), lay.ntiles,
                        reinterpret_cast<const DevProof*>(ws + lay.off_dp), FOLD_WAIT_NS, st);
  if (ce == cudaSuccess)
    ce = launch_linear_short(dL, reinterpret_cast<const LinShort*>(ws + lay.off_short), lay.nshort, st);
  if (ce == cudaSuccess) ce = cudaEventRecord(ev[2], st);
  if (ce == cudaSuccess) ce = launch_linear_finish(dL, lay.np, lay.max_nblk, lay.max_q, dout, st);
  if (ce == cudaSuccess) ce = cudaEventRecord(ev[3], st);
  if (ce == cudaSuccess && out_space == VL_HOST) {
    ce = cudaMemcpyAsync(out, dout, sizeof(vl_lin_proof) * lay.np, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  }
  if (ce != cudaSuccess) return cuda_fail("vl_lin_plan_run", ce);
  P->timed = true;
  if (out_space == VL_HOST)
    for (int i = 0; i < lay.np; i++)
      if (out[i].status != VL_OK) return out[i].status;
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" int32_t vl_lin_plan_phase_ms(vl_lin_plan* P, float ms[3]) {
  if (!P || !ms || !P->timed) return VL_EINVAL;
  cudaError_t ce = cudaEventSynchronize(P->ev[3]);
  for (int i = 0; i < 3 && ce == cudaSuccess; i++) ce = cudaEventElapsedTime(&ms[i], P->ev[i], P->ev[i + 1]);
  return ce == cudaSuccess ? VL_OK : cuda_fail("vl_lin_plan_phase_ms", ce);
}

extern "C" void vl_lin_plan_destroy(vl_lin_plan* plan) { delete plan; }

extern "C" int32_t vl_prove_linear(const vl_lin_job* jobs, int32_t njobs, void* workspace, size_t workspace_bytes,
                                   vl_lin_proof* out, void* stream) {
  if (!workspace || !out) {
    LinLayout L;  // argument errors of the jobs first, as a plan would report them
    const int e = lin_layout(jobs, njobs, &L);
    return e != VL_OK ? e : VL_EINVAL;
  }
  vl_lin_plan* P = nullptr;
  int e = vl_lin_plan_create(jobs, njobs, &P);
  if (e != VL_OK) return e;
  e = vl_lin_plan_run(P, workspace, workspace_bytes, out, VL_HOST, stream);
  vl_lin_plan_destroy(P);
  return e;
}
