// Host engine and C ABI of the prover (see include/verilora.h).
//
// A plan turns a list of products (jobs) into device descriptor tables:
// one DevProof per job, two fold tasks per job (op(P) against E_u, op(Q)
// against E_v) cut into fold tiles, and a workspace layout.  One proving pass
// is four stream operations: zero the fold accumulators, the prologue kernel
// (transcripts, challenges, eq tables), the fold kernel over all tiles of all
// jobs, and the rounds kernel (claims, sumcheck rounds, proofs).  A plan can
// capture that pass in a CUDA graph and replay it.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
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

size_t esize(int32_t dtype) {
  return dtype == VL_I16 ? 2 : dtype == VL_I64 ? 8 : dtype == VL_FR_MONT ? 32 : 0;
}

int check_mat(const vl_mat* M, bool prover) {
  if (!M || !M->data) return VL_EINVAL;
  if (M->reserved != 0 || (M->trans != 0 && M->trans != 1)) return VL_EINVAL;
  if (M->space != VL_DEVICE && M->space != VL_HOST) return VL_EINVAL;
  if (prover && M->dtype != VL_I16 && M->dtype != VL_FR_MONT) return VL_EINVAL;
  if (!esize(M->dtype)) return VL_EINVAL;
  if (M->rows < 1 || M->cols < 1) return VL_ESHAPE;
  if (M->ld < M->cols) return VL_EINVAL;
  if (M->dtype == VL_FR_MONT && (reinterpret_cast<uintptr_t>(M->data) & 15)) return VL_EINVAL;
  return VL_OK;
}

struct Dims {
  int64_t m, k, n;
};

int job_dims(const vl_job& j, Dims* d) {
  int e;
  if ((e = check_mat(&j.P, true)) != VL_OK) return e;
  if ((e = check_mat(&j.Q, true)) != VL_OK) return e;
  const int64_t m = j.P.trans ? j.P.cols : j.P.rows;
  const int64_t k = j.P.trans ? j.P.rows : j.P.cols;
  const int64_t kq = j.Q.trans ? j.Q.cols : j.Q.rows;
  const int64_t n = j.Q.trans ? j.Q.rows : j.Q.cols;
  if (k != kq) return VL_ESHAPE;
  if (m > VL_MAX_REDUCE || n > VL_MAX_REDUCE || k > (int64_t(1) << VL_MAX_ROUNDS)) return VL_ESHAPE;
  d->m = m;
  d->k = k;
  d->n = n;
  return VL_OK;
}

struct Staged {
  size_t off;
  size_t bytes;
};

// One host-to-device copy of staged operands: host matrices whose ranges
// lie close together keep their relative layout in the workspace and move
// as one range.
struct StageRun {
  const void* host;
  size_t off, bytes;
};

// Where a host operand lives: pinned memory (an allocation of the CUDA
// driver, with its range when the driver reports it) or other (pageable)
// memory.  A copy from pinned memory must stay inside one allocation; a copy
// from pageable memory may only read mapped bytes.
struct HostRange {
  bool pinned = false, known = false;
  uintptr_t base = 0;
  size_t size = 0;
};

HostRange host_range(const void* ptr) {
  using Fn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
  static const Fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<Fn>(f);
    return static_cast<Fn>(nullptr);
  }();
  HostRange r;
  const CUdeviceptr p = reinterpret_cast<CUdeviceptr>(ptr);
  unsigned int type = 0;
  if (!fn) {
    r.pinned = true;  // cannot tell: treat as pinned of unknown extent (never joined)
    return r;
  }
  if (fn(&type, CU_POINTER_ATTRIBUTE_MEMORY_TYPE, p) != CUDA_SUCCESS) return r;  // not the driver's: pageable
  r.pinned = true;
  CUdeviceptr base = 0;
  size_t size = 0;
  if (fn(&base, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, p) == CUDA_SUCCESS &&
      fn(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, p) == CUDA_SUCCESS) {
    r.known = true;
    r.base = (uintptr_t)base;
    r.size = size;
  }
  return r;
}

}  // namespace

struct vl_plan {
  std::vector<vl_job> jobs;
  vl_batch_opts opts{};
  std::vector<DevProof> proofs;
  std::vector<FoldTask> tasks;
  std::vector<FoldTile> tiles;
  std::vector<TcTile> tc_tiles;  // tensor-core fold (phase launches)
  std::vector<DualTile> dual_tiles;  // tensor-core fold of matrices folded both ways
  size_t off_dual_tiles = 0;
  std::vector<EqItem> eq_items;  // eq-table chunks, proof by proof
  std::vector<StepItem> items;  // persistent step: queue order
  // Phase launches: proofs in groups (k descending); the graph folds group g
  // while group g+1's prologue and group g-1's rounds run on other streams.
  struct Group {
    int p0, p1;  // proofs [p0, p1)
    int t0, t1;  // CUDA-core fold tiles [t0, t1)
    int c0, c1;  // tensor-core fold tiles [c0, c1)
    int e0, e1;  // eq-table chunks [e0, e1)
  };
  std::vector<Group> groups;
  std::vector<int> slot_of_job;  // DevProof index of each job
  // Chained proofs (per job, caller order; empty when unused): a given start
  // state and point, and where the rounds store their challenges.
  std::vector<const GivenPoint*> given;
  std::vector<Fr*> rch;
  cudaStream_t side[2] = {nullptr, nullptr};  // rounds stream, prologue stream
  std::vector<cudaEvent_t> gev;               // dependency events (no timing)
  std::vector<CUtensorMap> tmaps;   // one per fold task (TMA operands), built at bind time
  std::vector<CUtensorMap> etmaps;  // limb-major weights of each row-dot task
  size_t off_tmaps = 0, off_etmaps = 0;
  int fold_smem = 0;
  int step_smem = 0;
  int step_grid = 0;            // CTAs of the persistent launch (set at bind time)
  size_t off_ctl = 0, off_items = 0;
  // workspace layout (offsets from the workspace base)
  size_t off_proofs = 0, off_scr = 0, off_tasks = 0, off_tiles = 0, off_tc_tiles = 0, off_eq_items = 0;
  size_t off_acc = 0, acc_bytes = 0, off_out = 0, total = 0;
  // batched rounds (rounds_variant 8): per round t (1-based) its items and
  // the item range of each proof; proofs with d1 >= t are a prefix (k-descending)
  std::vector<RoundItem> ritems;
  std::vector<int> ibase;           // per round: np_t + 1 prefix offsets into that round's items
  std::vector<int> r_item0, r_nitem, r_ib0, r_np;  // per round t (index t): first item, items, ibase start, proofs
  size_t off_ritems = 0, off_ibase = 0, off_partials = 0;
  struct PerProof {
    size_t eqA, eqB, soaA, soaB, w8A, w8B, accA, accB, fA, fB, fac;
  };
  std::vector<PerProof> pp;
  std::map<const void*, Staged> staging;  // host operand -> device copy
  std::vector<StageRun> stage_runs;       // the copies that fill the staging
  // bound state
  void* bound_ws = nullptr;
  vl_proof* bound_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // phase timing: events at the four phase boundaries of every run, taken
  // from a ring of `ring_runs` runs; in a graph the event-record nodes are
  // pointed at the current ring slot before each launch.
  int ring_runs = 64;
  static constexpr int NEV = 4;  // before clear, before fold, after fold, after rounds
  std::vector<cudaEvent_t> ring;
  cudaEvent_t cap_ev[NEV] = {};
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  cudaGraphNode_t ev_node[NEV] = {};
  long runs = 0, timing_base = 0;
};

namespace {

// Phase launches unless the options ask for the persistent single launch.
bool persistent(const vl_plan* p) { return p->opts.persistent == 1; }

// An int16 operand goes to the tensor-core fold when TMA can address it:
// 16-byte aligned base (host operands are staged at 256-byte offsets of a
// workspace aligned to 256 bytes) and rows a multiple of 16 bytes apart.
bool tc_eligible(const vl_plan* p, const vl_mat& M) {
  if (persistent(p) || p->opts.fold_engine == 1 || M.dtype != VL_I16 || (M.ld & 7)) return false;
  return M.space == VL_HOST || (reinterpret_cast<uintptr_t>(M.data) & 15) == 0;
}

void add_fold_task(vl_plan* p, const vl_mat& M, int32_t mode, int proof, int side) {
  FoldTask t{};
  t.mat = nullptr;  // bound at run time
  t.ld = M.ld;
  t.rows = (int32_t)M.rows;
  t.cols = (int32_t)M.cols;
  t.mode = mode;
  t.dtype = M.dtype;
  t.proof = proof;
  t.side = side;
  // TMA box of the stored matrix (used when the operand qualifies at bind time).
  auto round8 = [](int64_t x) { return (int)((x + 7) & ~int64_t(7)); };
  if (mode == MODE_COLSUM) {
    t.box_w = std::min(256, round8(std::min<int64_t>(M.cols, COLSUM_TILE_COLS)));
    const int nsub = (int)((std::min<int64_t>(M.cols, COLSUM_TILE_COLS) + t.box_w - 1) / t.box_w);
    t.box_h = std::max(1, std::min(256, STAGE_BYTES / (nsub * t.box_w * 2)));
  } else {
    t.box_w = std::min(ROWDOT_STAGE_COLS, round8(std::min<int64_t>(M.cols, ROWDOT_TILE_COLS)));
    t.box_h = ROWDOT_BLOCK_ROWS;
  }
  const int task = (int)p->tasks.size();
  int32_t& tabs = side ? p->proofs[proof].tabB : p->proofs[proof].tabA;
  if (tc_eligible(p, M)) {
    // Tensor-core tiles: 128 lines by at most TC_SEG reduced entries.
    t.bulk = 2;
    t.box_w = mode == MODE_ROWDOT ? TC_KP : TC_M;  // row dots: 64 entries x 128 lines (128B-swizzled), two per stage
    t.box_h = mode == MODE_ROWDOT ? TC_M : TC_KS;  // column sums: 128 lines x 128 entries (no swizzle)
    p->tasks.push_back(t);
    tabs |= TAB_BYTES;
    const int lines = mode == MODE_COLSUM ? t.cols : t.rows, red = mode == MODE_COLSUM ? t.rows : t.cols;
    const int seg = p->opts.tc_seg > 0 ? p->opts.tc_seg : TC_SEG;
    // One segment: each tile holds its lines' whole sums and writes f reduced.
    (side ? p->proofs[proof].fdirB : p->proofs[proof].fdirA) = red <= seg ? 1 : 0;
    for (int w0 = 0; w0 < lines; w0 += TC_M)
      for (int k0 = 0; k0 < red; k0 += seg)
      {
        TcTile tt{};
        tt.mode = mode;
        tt.w0 = w0;
        tt.nw = std::min(TC_M, lines - w0);
        tt.k0 = k0;
        tt.nk = std::min(seg, red - k0);
        tt.proof = proof;
        tt.task = task;
        p->tc_tiles.push_back(tt);  // device pointers are filled in at bind time
      }
    return;
  }
  tabs |= TAB_LIMBS;
  p->tasks.push_back(t);
  const size_t tiles_before = p->tiles.size();
  const bool fr = M.dtype == VL_FR_MONT;
  if (mode == MODE_COLSUM) {
    const int tc = fr ? FR_COLSUM_TILE_COLS : COLSUM_TILE_COLS;
    const int tr = p->opts.colsum_rows > 0 ? p->opts.colsum_rows : 256;
    for (int c0 = 0; c0 < t.cols; c0 += tc)
      for (int r0 = 0; r0 < t.rows; r0 += tr) {
        FoldTile ft{};
        ft.task = task;
        ft.r0 = r0;
        ft.r1 = std::min<int>(t.rows, r0 + tr);
        ft.c0 = c0;
        ft.c1 = std::min<int>(t.cols, c0 + tc);
        p->tiles.push_back(ft);
        p->fold_smem = std::max(p->fold_smem, fold_tile_smem(mode, M.dtype, ft.r1 - ft.r0, ft.c1 - ft.c0));
      }
  } else {
    int tcmax = p->opts.rowdot_cols > 0 ? p->opts.rowdot_cols : ROWDOT_TILE_COLS;
    tcmax = (tcmax + 7) & ~7;
    for (int c0 = 0; c0 < t.cols; c0 += tcmax)
      for (int r0 = 0; r0 < t.rows; r0 += ROWDOT_TILE_ROWS) {
        FoldTile ft{};
        ft.task = task;
        ft.r0 = r0;
        ft.r1 = std::min<int>(t.rows, r0 + ROWDOT_TILE_ROWS);
        ft.c0 = c0;
        ft.c1 = std::min<int>(t.cols, c0 + tcmax);
        p->tiles.push_back(ft);
        p->fold_smem = std::max(p->fold_smem, fold_tile_smem(mode, M.dtype, ft.r1 - ft.r0, ft.c1 - ft.c0));
      }
  }
  p->proofs[proof].ntiles += (int32_t)(p->tiles.size() - tiles_before);
}

// Groups of consecutive proofs with about equal fold work (tiles are laid
// out proof by proof, so each group's tiles are contiguous too).
void build_groups(vl_plan* p) {
  const int np = (int)p->proofs.size();
  int ng = p->opts.groups > 0 ? p->opts.groups : 1;
  ng = std::max(1, std::min(std::min(ng, np), STEP_CTL_HEAD_INTS));  // one tile counter per group
  std::vector<int64_t> work(np, 0);
  std::vector<int> first_tile(np + 1, (int)p->tiles.size()), first_tc(np + 1, (int)p->tc_tiles.size()),
      first_eq(np + 1, (int)p->eq_items.size());
  for (int t = (int)p->eq_items.size() - 1; t >= 0; t--) first_eq[p->eq_items[t].proof] = t;
  for (int t = (int)p->tiles.size() - 1; t >= 0; t--) {
    const FoldTile& ft = p->tiles[t];
    const int pi = p->tasks[ft.task].proof;
    work[pi] += (int64_t)(ft.r1 - ft.r0) * (ft.c1 - ft.c0);
    first_tile[pi] = t;
  }
  for (int t = (int)p->tc_tiles.size() - 1; t >= 0; t--) {
    const TcTile& ft = p->tc_tiles[t];
    const int pi = p->tasks[ft.task].proof;
    work[pi] += (int64_t)ft.nw * ft.nk;
    first_tc[pi] = t;
  }
  for (int i = np - 1; i >= 0; i--) {
    first_tile[i] = std::min(first_tile[i], first_tile[i + 1]);
    first_tc[i] = std::min(first_tc[i], first_tc[i + 1]);
    first_eq[i] = std::min(first_eq[i], first_eq[i + 1]);
  }
  int64_t total = 0;
  for (int64_t w : work) total += w;
  p->groups.clear();
  int64_t acc = 0;
  int start = 0;
  for (int i = 0; i < np; i++) {
    acc += work[i];
    const bool cut = (int)p->groups.size() < ng - 1 && acc * ng >= total * (int64_t)(p->groups.size() + 1);
    if (cut || i == np - 1) {
      p->groups.push_back(
          vl_plan::Group{start, i + 1, first_tile[start], first_tile[i + 1], first_tc[start], first_tc[i + 1],
                         first_eq[start], first_eq[i + 1]});
      start = i + 1;
    }
  }
  // Within a group, tensor-core tiles go longest first (the CTAs take them
  // round robin in this order).
  for (const vl_plan::Group& G : p->groups)
    std::stable_sort(p->tc_tiles.begin() + G.c0, p->tc_tiles.begin() + G.c1,
                     [](const TcTile& a, const TcTile& b) { return a.nk > b.nk; });
}

// Queue order of the persistent step: proofs in layout order (k descending);
// each proof's prologue is queued STEP_LOOKAHEAD proofs ahead of its fold
// tiles.
void build_items(vl_plan* p) {
  const int np = (int)p->proofs.size();
  std::vector<int> order(np);
  for (int i = 0; i < np; i++) order[i] = i;  // proofs are already laid out by k descending
  std::vector<std::vector<int>> tiles_of(np);
  for (size_t t = 0; t < p->tiles.size(); t++) tiles_of[p->tasks[p->tiles[t].task].proof].push_back((int)t);
  p->items.clear();
  p->items.reserve(np + p->tiles.size());
  const int look = std::min(np, STEP_LOOKAHEAD);
  for (int i = 0; i < look; i++) p->items.push_back(StepItem{STEP_PROLOGUE, order[i]});
  for (int i = 0; i < np; i++) {
    if (i + look < np) p->items.push_back(StepItem{STEP_PROLOGUE, order[i + look]});
    for (int t : tiles_of[order[i]]) p->items.push_back(StepItem{STEP_FOLD, t});
  }
}

// Pair each tensor-core row-dot task with a tensor-core column-sum task on
// the same stored matrix (rows and columns multiples of 128) into dual tiles
// that stream the matrix once for both; the column-sum side then
// accumulates (each strip adds its rows' partial sums).  One proof group
// and phase launches only.
void build_dual(vl_plan* p) {
  p->dual_tiles.clear();
  if (p->opts.fold_dual != 1 || persistent(p) || p->opts.groups > 1) return;
  const int nt = (int)p->tasks.size();
  std::vector<int> partner(nt, -1);
  auto mat_of = [&](int t) -> const vl_mat& {
    const FoldTask& T = p->tasks[t];
    const vl_job& j = p->jobs[p->proofs[T.proof].job];
    return T.side ? j.Q : j.P;
  };
  for (int r = 0; r < nt; r++) {
    const FoldTask& R = p->tasks[r];
    if (R.bulk != 2 || R.mode != MODE_ROWDOT || R.rows % TC_M || R.cols % TC_KS) continue;
    const vl_mat& MR = mat_of(r);
    for (int c = 0; c < nt; c++) {
      const FoldTask& C = p->tasks[c];
      if (partner[c] >= 0 || C.bulk != 2 || C.mode != MODE_COLSUM) continue;
      const vl_mat& MC = mat_of(c);
      if (MC.data != MR.data || MC.ld != MR.ld || MC.rows != MR.rows || MC.cols != MR.cols || MC.space != MR.space)
        continue;
      partner[c] = r;
      partner[r] = c;
      break;
    }
  }
  const int seg = p->opts.tc_seg > 0 ? p->opts.tc_seg : TC_SEG;
  std::vector<TcTile> keep;
  keep.reserve(p->tc_tiles.size());
  for (const TcTile& tt : p->tc_tiles)
    if (partner[tt.task] < 0) keep.push_back(tt);
  if (keep.size() == p->tc_tiles.size()) return;
  p->tc_tiles.swap(keep);
  for (int r = 0; r < nt; r++) {
    if (partner[r] < 0 || p->tasks[r].mode != MODE_ROWDOT) continue;
    const int c = partner[r];
    const FoldTask& R = p->tasks[r];
    const FoldTask& C = p->tasks[c];
    (C.side ? p->proofs[C.proof].fdirB : p->proofs[C.proof].fdirA) = 0;  // strips add partial column sums
    for (int w0 = 0; w0 < R.rows; w0 += TC_M)
      for (int k0 = 0; k0 < R.cols; k0 += seg) {
        DualTile d{};
        d.w0 = w0;
        d.k0 = k0;
        d.nk = std::min(seg, R.cols - k0);
        d.proofR = R.proof;
        d.proofC = C.proof;
        d.taskR = r;
        d.taskC = c;
        p->dual_tiles.push_back(d);
      }
  }
}

int build_plan(vl_plan* p) {
  const int np = (int)p->jobs.size();
  // u32 digit sums hold at most 512 stages of 64 entries
  if (p->opts.tc_seg < 0 || p->opts.tc_seg % TC_KS || p->opts.tc_seg > 32768) return VL_EINVAL;
  p->proofs.resize(np);
  p->pp.resize(np);
  size_t off = 0;
  p->off_proofs = off;
  off = align_up(off + sizeof(DevProof) * np);
  p->off_scr = off;
  off = align_up(off + sizeof(ProofScratch) * np);
  p->off_out = off;
  off = align_up(off + sizeof(vl_proof) * np);

  // Proofs are laid out by k descending (their rounds take longest, so they
  // should finish first); DevProof.job maps back to the caller's order.
  std::vector<int> order(np);
  std::vector<int64_t> kk(np);
  for (int i = 0; i < np; i++) {
    Dims d;
    int e = job_dims(p->jobs[i], &d);
    if (e != VL_OK) return e;
    order[i] = i;
    kk[i] = d.k;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return kk[a] > kk[b]; });
  p->slot_of_job.assign(np, 0);
  for (int i = 0; i < np; i++) {
    const vl_job& j = p->jobs[order[i]];
    Dims d;
    job_dims(j, &d);
    p->slot_of_job[order[i]] = i;
    DevProof& P = p->proofs[i];
    std::memset(&P, 0, sizeof(P));
    P.m = (int32_t)d.m;
    P.k = (int32_t)d.k;
    P.n = (int32_t)d.n;
    P.d0 = ceil_log2(d.m);
    P.d1 = ceil_log2(d.k);
    P.d2 = ceil_log2(d.n);
    P.tp = j.P.trans;
    P.tq = j.Q.trans;
    P.dtypeA = j.P.dtype;
    P.dtypeB = j.Q.dtype;
    P.seed = j.fs.seed;
    P.job = order[i];
    std::memcpy(P.binds, j.fs.bind, 96);
    // f_A: op(P) over its m rows.  Stored m x k -> column sums; stored k x m -> row dots.
    add_fold_task(p, j.P, j.P.trans ? MODE_ROWDOT : MODE_COLSUM, i, 0);
    // f_B: op(Q) over its n columns.  Stored k x n -> row dots; stored n x k -> column sums.
    add_fold_task(p, j.Q, j.Q.trans ? MODE_COLSUM : MODE_ROWDOT, i, 1);
  }
  build_dual(p);
  // eq-table chunks (tensor-core tables run to a multiple of 128 entries)
  p->eq_items.clear();
  for (int i = 0; i < np; i++) {
    const DevProof& P = p->proofs[i];
    for (int side = 0; side < 2; side++) {
      const int tabs = side ? P.tabB : P.tabA, size = side ? P.n : P.m;
      const int end = (tabs & TAB_BYTES) ? (size + TC_KS - 1) / TC_KS * TC_KS : size;
      for (int c = 0; tabs && c < end; c += EQ_CHUNK) p->eq_items.push_back(EqItem{i, side, c, std::min(end, c + EQ_CHUNK)});
    }
  }
  build_items(p);
  build_groups(p);
  p->off_tasks = off;
  off = align_up(off + sizeof(FoldTask) * p->tasks.size());
  p->off_tiles = off;
  off = align_up(off + sizeof(FoldTile) * p->tiles.size());
  p->off_tc_tiles = off;
  off = align_up(off + sizeof(TcTile) * p->tc_tiles.size());
  p->off_eq_items = off;
  off = align_up(off + sizeof(EqItem) * p->eq_items.size());
  p->off_dual_tiles = off;
  off = align_up(off + sizeof(DualTile) * p->dual_tiles.size());
  p->off_tmaps = off;
  off = align_up(off + sizeof(CUtensorMap) * p->tasks.size());
  p->off_etmaps = off;
  off = align_up(off + sizeof(CUtensorMap) * p->tasks.size());
  p->off_items = off;
  off = align_up(off + sizeof(StepItem) * p->items.size());
  // step control block and accumulators: one contiguous region, zeroed each pass
  p->off_ctl = off;
  off = align_up(off + sizeof(int) * (STEP_CTL_HEAD_INTS + 2 * (size_t)np));
  p->off_acc = off;
  for (int i = 0; i < np; i++) {
    const size_t kb = (size_t)p->proofs[i].k * 8 * sizeof(unsigned long long);
    p->pp[i].accA = p->pp[i].accB = 0;
    if (!p->proofs[i].fdirA) {
      p->pp[i].accA = off;
      off = align_up(off + kb);
    }
    if (!p->proofs[i].fdirB) {
      p->pp[i].accB = off;
      off = align_up(off + kb);
    }
  }
  p->acc_bytes = off - p->off_acc;
  p->step_smem = std::max(p->fold_smem, std::max(PRO_SMEM, RND_SMEM));
  for (int i = 0; i < np; i++) {
    DevProof& P = p->proofs[i];
    P.soa_pitchA = (P.m + 3) & ~3;
    P.soa_pitchB = (P.n + 3) & ~3;
    p->pp[i].eqA = p->pp[i].eqB = p->pp[i].soaA = p->pp[i].soaB = p->pp[i].w8A = p->pp[i].w8B = 0;
    if (P.tabA & TAB_LIMBS) {
      p->pp[i].eqA = off;
      off = align_up(off + sizeof(Fr) * P.m);
      p->pp[i].soaA = off;
      off = align_up(off + 32 * (size_t)P.soa_pitchA);
    }
    if (P.tabB & TAB_LIMBS) {
      p->pp[i].eqB = off;
      off = align_up(off + sizeof(Fr) * P.n);
      p->pp[i].soaB = off;
      off = align_up(off + 32 * (size_t)P.soa_pitchB);
    }
    if (P.tabA & TAB_BYTES) {
      p->pp[i].w8A = off;
      off = align_up(off + 8192 * (size_t)((P.m + TC_KS - 1) / TC_KS));
    }
    if (P.tabB & TAB_BYTES) {
      p->pp[i].w8B = off;
      off = align_up(off + 8192 * (size_t)((P.n + TC_KS - 1) / TC_KS));
    }
    p->pp[i].fA = off;
    off = align_up(off + sizeof(Fr) * ((size_t)1 << P.d1));
    p->pp[i].fB = off;
    off = align_up(off + sizeof(Fr) * ((size_t)1 << P.d1));
    p->pp[i].fac = off;
    off = align_up(off + sizeof(Fr) * 4 * EQ_FAC);
  }
  // batched rounds: items of RB_PAIRS pairs per proof and batched round
  // (proofs with batched rounds are a prefix: k-descending)
  {
    const int maxb = np ? batched_rounds(p->proofs[0].d1) : 0;
    p->ritems.clear();
    p->ibase.clear();
    p->r_item0.assign(maxb + 2, 0);
    p->r_nitem.assign(maxb + 2, 0);
    p->r_ib0.assign(maxb + 2, 0);
    p->r_np.assign(maxb + 2, 0);
    size_t max_items = 1;
    for (int t = 1; t <= maxb; t++) {
      p->r_item0[t] = (int)p->ritems.size();
      p->r_ib0[t] = (int)p->ibase.size();
      int npt = 0;
      for (int i = 0; i < np; i++) {
        const DevProof& P = p->proofs[i];
        if (batched_rounds(P.d1) < t) break;
        npt = i + 1;
        p->ibase.push_back((int)p->ritems.size() - p->r_item0[t]);
        const int pairs = 1 << (P.d1 - t);
        for (int j0 = 0; j0 < pairs; j0 += RB_PAIRS)
          p->ritems.push_back(RoundItem{i, j0, std::min(pairs, j0 + RB_PAIRS), 0});
      }
      p->ibase.push_back((int)p->ritems.size() - p->r_item0[t]);
      p->r_np[t] = npt;
      p->r_nitem[t] = (int)p->ritems.size() - p->r_item0[t];
      max_items = std::max(max_items, (size_t)p->r_nitem[t]);
    }
    p->off_ritems = off;
    off = align_up(off + sizeof(RoundItem) * std::max<size_t>(p->ritems.size(), 1));
    p->off_ibase = off;
    off = align_up(off + sizeof(int) * std::max<size_t>(p->ibase.size(), 1));
    p->off_partials = off;
    off = align_up(off + 3 * sizeof(Fr) * max_items);
  }
  // staging for host operands: one device copy of each distinct host
  // matrix.  Matrices whose host ranges follow each other (both 16-byte
  // aligned; in one pinned allocation with a gap of at most 4 KB, or both in
  // pageable memory and touching) are staged with the same relative layout
  // and copied as one range: a step's many small operands then cost a few
  // large copies instead of one copy each.
  p->staging.clear();
  p->stage_runs.clear();
  for (const vl_job& j : p->jobs) {
    for (const vl_mat* M : {&j.P, &j.Q}) {
      if (M->space != VL_HOST) continue;
      const size_t bytes = ((size_t)(M->rows - 1) * M->ld + M->cols) * esize(M->dtype);
      auto it = p->staging.find(M->data);
      if (it != p->staging.end()) {
        if (it->second.bytes < bytes) return VL_EINVAL;  // same pointer, different extent
        continue;
      }
      p->staging[M->data] = Staged{0, bytes};
    }
  }
  {
    const uint8_t* run_host = nullptr;
    size_t run_off = 0, run_len = 0;
    HostRange run_range;
    for (auto& kv : p->staging) {  // ascending host addresses
      const uint8_t* h = static_cast<const uint8_t*>(kv.first);
      const HostRange hr = host_range(h);
      const bool aligned = reinterpret_cast<uintptr_t>(h) % 16 == 0;
      const size_t gap = run_host && h >= run_host + run_len ? (size_t)(h - (run_host + run_len)) : SIZE_MAX;
      bool fits = false;
      if (run_host && (run_range.pinned || hr.pinned))
        fits = run_range.known && hr.known && run_range.base == hr.base && gap <= 4096 &&
               reinterpret_cast<uintptr_t>(h) + kv.second.bytes <= hr.base + hr.size;
      else if (run_host)
        fits = gap == 0;
      const bool join = fits && aligned && reinterpret_cast<uintptr_t>(run_host) % 16 == 0;
      if (!join) {
        if (run_host) {
          p->stage_runs.push_back(StageRun{run_host, run_off, run_len});
          off = align_up(run_off + run_len);
        }
        run_host = h;
        run_range = hr;
        run_off = off;
        run_len = 0;
      }
      const size_t rel = (size_t)(h - run_host);
      kv.second.off = run_off + rel;
      run_len = std::max(run_len, rel + kv.second.bytes);
    }
    if (run_host) {
      p->stage_runs.push_back(StageRun{run_host, run_off, run_len});
      off = align_up(run_off + run_len);
    }
  }
  p->total = off;
  if (p->fold_smem > 200 * 1024) return VL_ESHAPE;
  return VL_OK;
}

const void* operand_ptr(const vl_plan* p, const vl_mat& M, uint8_t* ws) {
  if (M.space == VL_DEVICE) return M.data;
  return ws + p->staging.at(M.data).off;
}

thread_local char g_last_error[256] = "";

void note_error(const char* where, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
}

// Which plan last wrote its descriptor tables into a workspace (by base
// pointer).  A plan whose workspace was taken over by another plan re-binds
// (re-uploads its tables) before its next run.
std::mutex g_ws_mu;
std::map<const void*, const void*> g_ws_owner;  // workspace -> the plan whose tables it holds

bool owns_workspace(const void* p, const void* ws) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  auto it = g_ws_owner.find(ws);
  return it != g_ws_owner.end() && it->second == p;
}

void claim_workspace(const void* p, const void* ws) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  g_ws_owner[ws] = p;
}

void release_workspaces(const void* p) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  for (auto it = g_ws_owner.begin(); it != g_ws_owner.end();)
    it = it->second == p ? g_ws_owner.erase(it) : std::next(it);
}

int cuda_status(cudaError_t e, const char* where = "cuda") {
  if (e == cudaSuccess) return VL_OK;
  note_error(where, e);
  return VL_ECUDA;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  // Looked up once; the initialisation of a function-local static is
  // thread-safe (plans are built from user threads and the server's worker).
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
  }();
  return fn;
}

// TMA descriptor of an int16 task's stored matrix; false if the operand does
// not qualify (16-byte aligned base, rows a multiple of 16 bytes apart,
// a multiple of 8 columns) or encoding fails.
bool encode_task_map(const FoldTask& t, CUtensorMap* map) {
  if (t.dtype != VL_I16 || (reinterpret_cast<uintptr_t>(t.mat) & 15) || (t.ld & 7) || (t.cols & 7)) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)t.cols, (cuuint64_t)t.rows};
  const cuuint64_t strides[1] = {(cuuint64_t)t.ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)t.box_w, (cuuint32_t)t.box_h};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(t.mat), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA descriptor of a tensor-core task's stored matrix: uint16 boxes of 64
// columns (128 bytes, 128-byte swizzle) by 128 rows for row dots, 128 columns
// by 128 rows (no swizzle: rows of 256 contiguous bytes stream better) for
// column sums; out-of-range entries read as zero.
bool encode_tc_map(const FoldTask& t, CUtensorMap* map) {
  return vl::encode_tc_operand(t.mat, t.rows, t.cols, t.ld, t.mode, map);
}

// TMA descriptor of the limb-major weights a row-dot task reads: 8 rows of
// `pitch` words, boxes of [8 x BW].
bool encode_weight_map(const FoldTask& t, const uint32_t* soa, int pitch, CUtensorMap* map) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)t.cols, 8};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
  const cuuint32_t box[2] = {(cuuint32_t)t.box_w, 8};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t*>(soa), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Fill device pointers for this workspace and upload the descriptor tables.
int bind_workspace(vl_plan* p, uint8_t* ws, cudaStream_t st) {
  const int np = (int)p->jobs.size();
  for (int i = 0; i < np; i++) {
    DevProof& P = p->proofs[i];
    const bool la = P.tabA & TAB_LIMBS, lb = P.tabB & TAB_LIMBS;
    P.eqA = la ? reinterpret_cast<Fr*>(ws + p->pp[i].eqA) : nullptr;
    P.eqB = lb ? reinterpret_cast<Fr*>(ws + p->pp[i].eqB) : nullptr;
    P.eqA_soa = la ? reinterpret_cast<uint32_t*>(ws + p->pp[i].soaA) : nullptr;
    P.eqB_soa = lb ? reinterpret_cast<uint32_t*>(ws + p->pp[i].soaB) : nullptr;
    P.w8A = (P.tabA & TAB_BYTES) ? reinterpret_cast<uint32_t*>(ws + p->pp[i].w8A) : nullptr;
    P.w8B = (P.tabB & TAB_BYTES) ? reinterpret_cast<uint32_t*>(ws + p->pp[i].w8B) : nullptr;
    P.accA = P.fdirA ? nullptr : reinterpret_cast<unsigned long long*>(ws + p->pp[i].accA);
    P.accB = P.fdirB ? nullptr : reinterpret_cast<unsigned long long*>(ws + p->pp[i].accB);
    P.fA = reinterpret_cast<Fr*>(ws + p->pp[i].fA);
    P.fB = reinterpret_cast<Fr*>(ws + p->pp[i].fB);
    P.scr = reinterpret_cast<ProofScratch*>(ws + p->off_scr) + i;
    P.fac = reinterpret_cast<Fr*>(ws + p->pp[i].fac);
    P.given = p->given.empty() ? nullptr : p->given[P.job];
    P.rch = p->rch.empty() ? nullptr : p->rch[P.job];
  }
  p->tmaps.resize(p->tasks.size());
  p->etmaps.resize(p->tasks.size());
  for (size_t i = 0; i < p->tasks.size(); i++) {
    FoldTask& t = p->tasks[i];
    const DevProof& P = p->proofs[t.proof];
    const vl_job& j = p->jobs[P.job];
    t.mat = operand_ptr(p, t.side ? j.Q : j.P, ws);
    std::memset(&p->tmaps[i], 0, sizeof(CUtensorMap));
    std::memset(&p->etmaps[i], 0, sizeof(CUtensorMap));
    t.tmap = ws + p->off_tmaps + i * sizeof(CUtensorMap);
    t.etmap = ws + p->off_etmaps + i * sizeof(CUtensorMap);
    if (t.bulk == 2) {
      if (!encode_tc_map(t, &p->tmaps[i])) {
        snprintf(g_last_error, sizeof(g_last_error), "tensor map of fold task %zu could not be encoded", i);
        return VL_EINVAL;
      }
      continue;
    }
    bool ok = encode_task_map(t, &p->tmaps[i]);
    if (ok && t.mode == MODE_ROWDOT)
      ok = encode_weight_map(t, t.side ? P.eqB_soa : P.eqA_soa, t.side ? P.soa_pitchB : P.soa_pitchA,
                             &p->etmaps[i]);
    t.bulk = ok ? 1 : 0;
  }
  for (TcTile& tt : p->tc_tiles) {
    const FoldTask& t = p->tasks[tt.task];
    const DevProof& P = p->proofs[t.proof];
    tt.tmap = t.tmap;
    tt.w8 = t.side ? P.w8B : P.w8A;
    const bool direct = t.side ? P.fdirB : P.fdirA;
    tt.acc = direct ? nullptr : (t.side ? P.accB : P.accA) + (size_t)tt.w0 * 8;
    tt.f = direct ? (t.side ? P.fB : P.fA) + tt.w0 : nullptr;
    tt.corr = direct ? (t.side ? &P.scr->corrB : &P.scr->corrA) : nullptr;
  }
  for (DualTile& d : p->dual_tiles) {
    const FoldTask& R = p->tasks[d.taskR];
    const FoldTask& C = p->tasks[d.taskC];
    const DevProof& PR = p->proofs[R.proof];
    const DevProof& PC = p->proofs[C.proof];
    d.tmap = R.tmap;
    d.w8R = R.side ? PR.w8B : PR.w8A;
    d.w8C = C.side ? PC.w8B : PC.w8A;
    const bool direct = R.side ? PR.fdirB : PR.fdirA;
    d.accR = direct ? nullptr : (R.side ? PR.accB : PR.accA) + (size_t)d.w0 * 8;
    d.fR = direct ? (R.side ? PR.fB : PR.fA) + d.w0 : nullptr;
    d.corrR = direct ? (R.side ? &PR.scr->corrB : &PR.scr->corrA) : nullptr;
    d.accC = C.side ? PC.accB : PC.accA;
  }
  cudaError_t e = cudaMemcpyAsync(ws + p->off_proofs, p->proofs.data(), sizeof(DevProof) * np,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->dual_tiles.empty())
    e = cudaMemcpyAsync(ws + p->off_dual_tiles, p->dual_tiles.data(), sizeof(DualTile) * p->dual_tiles.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->tasks.empty())
    e = cudaMemcpyAsync(ws + p->off_tasks, p->tasks.data(), sizeof(FoldTask) * p->tasks.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->tiles.empty())
    e = cudaMemcpyAsync(ws + p->off_tiles, p->tiles.data(), sizeof(FoldTile) * p->tiles.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->tc_tiles.empty())
    e = cudaMemcpyAsync(ws + p->off_tc_tiles, p->tc_tiles.data(), sizeof(TcTile) * p->tc_tiles.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->eq_items.empty())
    e = cudaMemcpyAsync(ws + p->off_eq_items, p->eq_items.data(), sizeof(EqItem) * p->eq_items.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->tmaps.empty())
    e = cudaMemcpyAsync(ws + p->off_tmaps, p->tmaps.data(), sizeof(CUtensorMap) * p->tmaps.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->etmaps.empty())
    e = cudaMemcpyAsync(ws + p->off_etmaps, p->etmaps.data(), sizeof(CUtensorMap) * p->etmaps.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->items.empty())
    e = cudaMemcpyAsync(ws + p->off_items, p->items.data(), sizeof(StepItem) * p->items.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->ritems.empty())
    e = cudaMemcpyAsync(ws + p->off_ritems, p->ritems.data(), sizeof(RoundItem) * p->ritems.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->ibase.empty())
    e = cudaMemcpyAsync(ws + p->off_ibase, p->ibase.data(), sizeof(int) * p->ibase.size(), cudaMemcpyHostToDevice,
                        st);
  // The host vectors must outlive the copies: wait for them.
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && p->fold_smem > 0) e = fold_set_smem(p->fold_smem);
  if (e == cudaSuccess && !p->tc_tiles.empty()) e = fold_tc_prepare();
  if (e == cudaSuccess && !p->dual_tiles.empty()) e = fold_dual_prepare();
  if (e == cudaSuccess && persistent(p)) e = step_set_smem(p->step_smem);
  if (e == cudaSuccess && persistent(p) && !p->step_grid) e = step_grid(p->step_smem, &p->step_grid);
  return cuda_status(e, "bind_workspace");
}

// DevProof index of the test hook's proof (given as 1 + job index), or -1.
int never_ready_slot(const vl_plan* p) {
  const int j = p->opts.test_never_ready - 1;
  return (j >= 0 && j < (int)p->slot_of_job.size()) ? p->slot_of_job[j] : -1;
}

unsigned long long wait_ns(const vl_plan* p) {
  return p->opts.wait_limit_us > 0 ? 1000ull * (unsigned long long)p->opts.wait_limit_us : FOLD_WAIT_NS;
}

cudaError_t ensure_events(vl_plan* p) {
  if (p->gev.empty() && !persistent(p) && p->groups.size() > 1) {
    p->gev.resize(2 * p->groups.size() + 2);
    for (cudaEvent_t& ev : p->gev) {
      cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    for (cudaStream_t& s2 : p->side) {
      cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
  }
  if (!p->ring.empty()) return cudaSuccess;
  p->ring.resize((size_t)p->ring_runs * vl_plan::NEV);
  for (cudaEvent_t& ev : p->ring) {
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
  }
  for (cudaEvent_t& ev : p->cap_ev) {
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaEvent_t* slot_events(vl_plan* p, long run) {
  return &p->ring[(size_t)(run % p->ring_runs) * vl_plan::NEV];
}

// Claims and rounds of every proof: one CTA per proof (rounds_kernel), or
// with rounds_variant 8 one launch per round for the round's vector work of
// all proofs and one for its transcript steps.
cudaError_t enqueue_rounds(vl_plan* p, uint8_t* ws, const DevProof* dp, vl_proof* dout, cudaStream_t st) {
  const int np = (int)p->jobs.size();
  if (p->opts.rounds_variant != 8)
    return launch_rounds(dp, np, dout, p->opts.rounds_variant, p->opts.rounds_threads, st);
  const RoundItem* items = reinterpret_cast<const RoundItem*>(ws + p->off_ritems);
  const int* ibase = reinterpret_cast<const int*>(ws + p->off_ibase);
  Fr* partials = reinterpret_cast<Fr*>(ws + p->off_partials);
  cudaError_t e = cudaSuccess;
  for (size_t t = 1; t + 1 < p->r_nitem.size() && e == cudaSuccess; t++) {
    e = launch_rounds_pass(dp, items + p->r_item0[t], p->r_nitem[t], partials, (int)t, st);
    if (e == cudaSuccess) e = launch_rounds_hash(dp, p->r_np[t], ibase + p->r_ib0[t], partials, dout, (int)t, st);
  }
  if (e == cudaSuccess) e = launch_rounds_tail(dp, np, dout, st);
  return e;
}

int rounds_launches(const vl_plan* p) {
  if (p->opts.rounds_variant != 8) return 1;
  int n = 1;  // the tail
  for (size_t t = 1; t + 1 < p->r_nitem.size(); t++) n += (p->r_nitem[t] > 0 ? 1 : 0) + (p->r_np[t] > 0 ? 1 : 0);
  return n;
}

// The device part of one proving pass (graph-capturable).  `ev`: the four
// phase-boundary events to record.
cudaError_t enqueue_pass(vl_plan* p, uint8_t* ws, vl_proof* dout, cudaStream_t st, cudaEvent_t* ev,
                         bool capturing) {
  const DevProof* dp = reinterpret_cast<const DevProof*>(ws + p->off_proofs);
  const FoldTask* dt = reinterpret_cast<const FoldTask*>(ws + p->off_tasks);
  const FoldTile* dl = reinterpret_cast<const FoldTile*>(ws + p->off_tiles);
  const TcTile* dc = reinterpret_cast<const TcTile*>(ws + p->off_tc_tiles);
  const EqItem* de = reinterpret_cast<const EqItem*>(ws + p->off_eq_items);
  const int np = (int)p->jobs.size();
  // Under capture, external records become event-record nodes of the graph
  // (the flag is only valid while capturing).
  const unsigned flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  cudaError_t e = cudaEventRecordWithFlags(ev[0], st, flags);
  if (persistent(p)) {
    // One launch: [0] clear, [1] the persistent step (prologues, folds and
    // rounds interleaved), [2] empty.
    int* ctl = reinterpret_cast<int*>(ws + p->off_ctl);
    const StepItem* di = reinterpret_cast<const StepItem*>(ws + p->off_items);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + p->off_ctl, 0, p->off_acc - p->off_ctl + p->acc_bytes, st);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[1], st, flags);
    if (e == cudaSuccess)
      e = launch_step(di, (int)p->items.size(), dt, dl, dp, np, dout, ctl, p->step_grid, p->step_smem, wait_ns(p),
                      never_ready_slot(p), st);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[2], st, flags);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[3], st, flags);
    return e;
  }
  // Phase launches in groups: stream st folds group g while the rounds stream
  // runs group g-1's rounds and the prologue stream group g+1's prologue.
  // Dependencies are graph edges (events); no kernel waits for another.
  // Phases: [0] clear + first prologue, [1] folds (rounds and prologues of
  // other groups overlap them), [2] rounds left after the last fold.
  const int ng = (int)p->groups.size();
  if (ng == 1) {
    // One group: everything in order on the caller's stream.
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + p->off_ctl, 0, p->off_acc + p->acc_bytes - p->off_ctl, st);
    if (e == cudaSuccess) e = launch_prologue(dp, 0, np, de, (int)p->eq_items.size(), st);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[1], st, flags);
    if (e == cudaSuccess)
      e = launch_fold_dual(reinterpret_cast<const DualTile*>(ws + p->off_dual_tiles), (int)p->dual_tiles.size(), dp,
                           wait_ns(p), st);
    if (e == cudaSuccess) e = launch_fold_tc(dc, (int)p->tc_tiles.size(), dp, wait_ns(p), st);
    if (e == cudaSuccess) e = launch_fold(dt, dl, (int)p->tiles.size(), dp, p->fold_smem, wait_ns(p), st);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[2], st, flags);
    if (e == cudaSuccess) e = enqueue_rounds(p, ws, dp, dout, st);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[3], st, flags);
    return e;
  }
  cudaStream_t rs = p->side[0], ps = p->side[1];
  cudaEvent_t* gev = p->gev.data();  // [0, ng): prologue g done; [ng, 2ng): fold g done; 2ng: start; 2ng+1: rounds done
  // tile counters (one per group) and accumulators: one contiguous region
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + p->off_ctl, 0, p->off_acc + p->acc_bytes - p->off_ctl, st);
  if (e == cudaSuccess) e = cudaEventRecord(gev[2 * ng], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ps, gev[2 * ng], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(rs, gev[2 * ng], 0);
  const vl_plan::Group& g0 = p->groups[0];
  if (e == cudaSuccess) e = launch_prologue(dp, g0.p0, g0.p1, de + g0.e0, g0.e1 - g0.e0, st);
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[1], st, flags);
  for (int g = 1; g < ng && e == cudaSuccess; g++) {
    const vl_plan::Group& G = p->groups[g];
    e = launch_prologue(dp, G.p0, G.p1, de + G.e0, G.e1 - G.e0, ps);
    if (e == cudaSuccess) e = cudaEventRecord(gev[g], ps);
  }
  for (int g = 0; g < ng && e == cudaSuccess; g++) {
    const vl_plan::Group& G = p->groups[g];
    if (g > 0) e = cudaStreamWaitEvent(st, gev[g], 0);
    if (e == cudaSuccess)
      e = launch_fold_tc(dc + G.c0, G.c1 - G.c0, dp, wait_ns(p), st);
    if (e == cudaSuccess) e = launch_fold(dt, dl + G.t0, G.t1 - G.t0, dp, p->fold_smem, wait_ns(p), st);
    if (e == cudaSuccess) e = cudaEventRecord(gev[ng + g], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(rs, gev[ng + g], 0);
    if (e == cudaSuccess) e = launch_rounds(dp + G.p0, G.p1 - G.p0, dout, p->opts.rounds_variant, p->opts.rounds_threads, rs);
  }
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[2], st, flags);
  if (e == cudaSuccess) e = cudaEventRecord(gev[2 * ng + 1], rs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, gev[2 * ng + 1], 0);
  if (e == cudaSuccess) e = cudaEventRecord(gev[0], ps);  // join the prologue stream too
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, gev[0], 0);
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[3], st, flags);
  return e;
}

// After capture: find the event-record node of each phase-boundary event.
cudaError_t find_event_nodes(vl_plan* p) {
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(p->graph, nullptr, &n);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  e = cudaGraphGetNodes(p->graph, nodes.data(), &n);
  if (e != cudaSuccess) return e;
  int found = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev;
    if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
    for (int q = 0; q < vl_plan::NEV; q++)
      if (ev == p->cap_ev[q]) {
        p->ev_node[q] = nd;
        found++;
      }
  }
  return found == vl_plan::NEV ? cudaSuccess : cudaErrorUnknown;
}

void drop_graph(vl_plan* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->gexec = nullptr;
  p->graph = nullptr;
}

int stage_host_operands(vl_plan* p, uint8_t* ws, cudaStream_t st) {
  for (const StageRun& r : p->stage_runs) {
    cudaError_t e = cudaMemcpyAsync(ws + r.off, r.host, r.bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "stage host operand");
  }
  return VL_OK;
}

int run_plan(vl_plan* p, void* workspace, size_t ws_bytes, vl_proof* out, int32_t out_space,
             cudaStream_t st, bool graph) {
  if (!workspace || !out) return VL_EINVAL;
  if (out_space != VL_DEVICE && out_space != VL_HOST) return VL_EINVAL;
  if (ws_bytes < p->total) return VL_ENOMEM;
  if (reinterpret_cast<uintptr_t>(workspace) & (ALIGN - 1)) return VL_EINVAL;
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  vl_proof* dout = out_space == VL_DEVICE ? out : reinterpret_cast<vl_proof*>(ws + p->off_out);
  if (cudaError_t ee = ensure_events(p)) return cuda_status(ee, "cudaEventCreate");
  if (p->bound_ws != workspace || !owns_workspace(p, workspace)) {
    // The graph holds kernel arguments into the workspace; rebuilt on change.
    if (p->bound_ws != workspace) drop_graph(p);
    int e = bind_workspace(p, ws, st);
    if (e != VL_OK) return e;
    p->bound_ws = workspace;
    claim_workspace(p, workspace);
  }
  int e = stage_host_operands(p, ws, st);
  if (e != VL_OK) return e;
  cudaEvent_t* ev = slot_events(p, p->runs);
  cudaError_t ce;
  if (graph) {
    if (p->gexec && p->bound_out != dout) drop_graph(p);
    if (!p->gexec) {
      // Capture on a private stream: the caller's stream may be the legacy
      // default stream, which cannot be captured.  The graph is then launched
      // on the caller's stream.
      if (!p->cap_stream && (ce = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_status(ce, "cudaStreamCreate");
      if ((ce = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_status(ce, "cudaStreamBeginCapture");
      cudaError_t ke = enqueue_pass(p, ws, dout, p->cap_stream, p->cap_ev, true);
      ce = cudaStreamEndCapture(p->cap_stream, &p->graph);
      if (ke != cudaSuccess || ce != cudaSuccess) {
        drop_graph(p);
        return cuda_status(ke != cudaSuccess ? ke : ce, "graph capture");
      }
      if ((ce = find_event_nodes(p)) != cudaSuccess) {
        drop_graph(p);
        return cuda_status(ce, "graph event nodes");
      }
      if ((ce = cudaGraphInstantiate(&p->gexec, p->graph, 0)) != cudaSuccess) {
        p->gexec = nullptr;
        drop_graph(p);
        return cuda_status(ce, "cudaGraphInstantiate");
      }
      p->bound_out = dout;
    }
    for (int q = 0; q < vl_plan::NEV; q++)
      if ((ce = cudaGraphExecEventRecordNodeSetEvent(p->gexec, p->ev_node[q], ev[q])) != cudaSuccess)
        return cuda_status(ce, "cudaGraphExecEventRecordNodeSetEvent");
    if ((ce = cudaGraphLaunch(p->gexec, st)) != cudaSuccess) return cuda_status(ce, "cudaGraphLaunch");
  } else {
    if ((ce = enqueue_pass(p, ws, dout, st, ev, false)) != cudaSuccess) return cuda_status(ce, "enqueue_pass");
  }
  p->runs++;
  if (out_space == VL_HOST) {
    const size_t bytes = sizeof(vl_proof) * p->jobs.size();
    if ((ce = cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_status(ce, "proof copy-out");
    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(ce, "cudaStreamSynchronize");
    for (size_t i = 0; i < p->jobs.size(); i++)
      if (out[i].status != VL_OK) return out[i].status;
  }
  return VL_OK;
}

int make_plan(const vl_job* jobs, int32_t njobs, const vl_batch_opts* opts, vl_plan** out) {
  if (!jobs || njobs < 1 || !out) return VL_EINVAL;
  std::unique_ptr<vl_plan> p(new (std::nothrow) vl_plan());
  if (!p) return VL_ENOMEM;
  p->jobs.assign(jobs, jobs + njobs);
  if (opts) p->opts = *opts;
  if (p->opts.timing_runs > 0) p->ring_runs = p->opts.timing_runs;
  const int e = build_plan(p.get());
  if (e != VL_OK) return e;
  *out = p.release();
  return VL_OK;
}

}  // namespace

namespace vl {
// Plans as building blocks of composite proofs (chained proofs).
int plan_make(const vl_job* jobs, int32_t njobs, const vl_batch_opts* opts, vl_plan** out) {
  return make_plan(jobs, njobs, opts, out);
}
size_t plan_bytes(const vl_plan* p) { return p->total; }
void plan_set_points(vl_plan* p, const std::vector<const GivenPoint*>& given, const std::vector<Fr*>& rch) {
  if (p->given != given || p->rch != rch) {
    p->given = given;
    p->rch = rch;
    drop_graph(p);
    p->bound_ws = nullptr;  // the descriptors change: bind again on the next run
  }
}
// Enqueue one pass (no graph), proofs to device memory in job order.
int plan_enqueue(vl_plan* p, uint8_t* ws, size_t bytes, vl_proof* dout, cudaStream_t st) {
  return run_plan(p, ws, bytes, dout, VL_DEVICE, st, false);
}
}  // namespace vl

extern "C" {

int32_t vl_version(void) { return 100; }

const char* vl_strerror(int32_t s) {
  switch (s) {
    case VL_OK: return "ok";
    case VL_EINVAL: return "invalid argument";
    case VL_ESHAPE: return "invalid shape";
    case VL_ENOMEM: return "workspace too small or host allocation failed";
    case VL_ECUDA: return "CUDA error";
    case VL_ETIMEOUT: return "device wait timed out";
    case VL_REJECT: return "proof rejected";
    case VL_ELOOKUP: return "a lookup value lies outside its table";
    default: return "unknown status";
  }
}

size_t vl_workspace_bytes(const vl_job* jobs, int32_t njobs, const vl_batch_opts* opts) {
  VL_ABI_TRY
  vl_plan* p = nullptr;
  if (make_plan(jobs, njobs, opts, &p) != VL_OK) return 0;
  const size_t t = p->total;
  delete p;
  return t;
  VL_ABI_CATCH(0)
}

int32_t vl_plan_create(const vl_job* jobs, int32_t njobs, const vl_batch_opts* opts, vl_plan** plan) {
  VL_ABI_TRY
  return make_plan(jobs, njobs, opts, plan);
  VL_ABI_CATCH(VL_ENOMEM)
}

size_t vl_plan_workspace_bytes(const vl_plan* plan) { return plan ? plan->total : 0; }

int32_t vl_plan_launches(const vl_plan* plan) {
  if (!plan) return 0;
  if (persistent(plan)) return 1;
  int32_t n = 0;
  for (const vl_plan::Group& G : plan->groups)  // prologue (transcripts, eq chunks), folds, rounds
    n += 1 + (G.e1 > G.e0 ? 1 : 0) + (G.c1 > G.c0 ? 1 : 0) + (G.t1 > G.t0 ? 1 : 0) +
         (plan->groups.size() == 1 ? rounds_launches(plan) + (plan->dual_tiles.empty() ? 0 : 1) : 1);
  return n;
}

int32_t vl_plan_run(vl_plan* plan, void* workspace, size_t workspace_bytes, vl_proof* out, int32_t out_space,
                    void* stream) {
  VL_ABI_TRY
  if (!plan) return VL_EINVAL;
  const bool graph = plan->opts.use_graph != 2;
  return run_plan(plan, workspace, workspace_bytes, out, out_space, static_cast<cudaStream_t>(stream), graph);
  VL_ABI_CATCH(VL_ENOMEM)
}

int32_t vl_plan_phase_ms(vl_plan* plan, float* ms, int32_t max_runs, int32_t reset) {
  if (!plan || (!ms && max_runs > 0) || max_runs < 0) return -VL_EINVAL;
  const long avail = std::min<long>(plan->runs - plan->timing_base, plan->ring_runs);
  const long cnt = std::min<long>(avail, max_runs);
  for (long i = 0; i < cnt; i++) {
    const long run = plan->runs - cnt + i;
    cudaEvent_t* ev = slot_events(plan, run);
    if (cudaEventSynchronize(ev[3]) != cudaSuccess) return -VL_ECUDA;
    for (int q = 0; q < 3; q++)
      if (cudaEventElapsedTime(&ms[i * 3 + q], ev[q], ev[q + 1]) != cudaSuccess) return -VL_ECUDA;
  }
  if (reset) plan->timing_base = plan->runs;
  return (int32_t)cnt;
}

const char* vl_last_error(void) { return g_last_error; }

int32_t vl_workspace_forget(const void* workspace) {
  if (!workspace) return -VL_EINVAL;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  return g_ws_owner.erase(workspace) ? 1 : 0;
}

void vl_plan_destroy(vl_plan* plan) {
  if (!plan) return;
  release_workspaces(plan);
  drop_graph(plan);
  if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
  for (cudaStream_t s2 : plan->side)
    if (s2) cudaStreamDestroy(s2);
  for (cudaEvent_t ev : plan->gev)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : plan->ring) cudaEventDestroy(ev);
  for (cudaEvent_t ev : plan->cap_ev)
    if (ev) cudaEventDestroy(ev);
  delete plan;
}

int32_t vl_prove_batch(const vl_job* jobs, int32_t njobs, void* workspace, size_t workspace_bytes, vl_proof* out,
                       int32_t out_space, void* stream, const vl_batch_opts* opts) {
  VL_ABI_TRY
  vl_plan* p = nullptr;
  int e = make_plan(jobs, njobs, opts, &p);
  if (e != VL_OK) return e;
  // Descriptor tables are uploaded synchronously, so the host plan can go
  // while device work is still queued.
  e = run_plan(p, workspace, workspace_bytes, out, out_space, static_cast<cudaStream_t>(stream), false);
  vl_plan_destroy(p);
  return e;
  VL_ABI_CATCH(VL_ENOMEM)
}

int32_t vl_prove_matmul(const vl_mat* P, const vl_mat* Q, const vl_fs_init* fs, void* workspace,
                        size_t workspace_bytes, vl_proof* out, void* stream) {
  if (!P || !Q || !fs || !out) return VL_EINVAL;
  vl_job j;
  j.P = *P;
  j.Q = *Q;
  j.fs = *fs;
  return vl_prove_batch(&j, 1, workspace, workspace_bytes, out, VL_HOST, stream, nullptr);
}

int32_t vl_encode(const vl_mat* src, void* dst, void* stream) {
  if (!src || !dst) return VL_EINVAL;
  int e = check_mat(src, true);
  if (e != VL_OK) return e;
  if (src->dtype != VL_I16 || src->space != VL_DEVICE) return VL_EINVAL;
  if (reinterpret_cast<uintptr_t>(dst) & 15) return VL_EINVAL;
  return cuda_status(launch_encode(static_cast<const int16_t*>(src->data), src->rows, src->cols, src->ld,
                                   static_cast<Fr*>(dst), static_cast<cudaStream_t>(stream)),
                     "encode_kernel");
}

}  // extern "C"

// ------------------------------------------------- no-allocation variant --
//
// vl_prove_matmul_noalloc: the same proving pass as vl_prove_matmul, with the
// workspace replaced by a file-scope device array, for callers that cannot
// allocate device memory.  Host code must not use the array's name as a
// device address: the address is looked up once per device below.

namespace {

__device__ __align__(256) uint8_t g_noalloc_scratch[VL_NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;  // held for a whole call: calls never overlap on the GPU
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set-up on first use).
int noalloc_scratch_ptr(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return VL_EINVAL;
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(no-allocation scratch)");
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return VL_OK;
}

}  // namespace

extern "C" int32_t vl_prove_matmul_noalloc(const vl_mat* P, const vl_mat* Q, const vl_fs_init* fs, vl_proof* out,
                                           void* stream) {
  VL_ABI_TRY
  if (!P || !Q || !fs || !out) return VL_EINVAL;
  if (P->space != VL_DEVICE || Q->space != VL_DEVICE) return VL_EINVAL;
  vl_job j;
  j.P = *P;
  j.Q = *Q;
  j.fs = *fs;
  vl_plan* p = nullptr;
  vl_batch_opts o{};
  o.persistent = 2;
  o.fold_engine = 1;  // the launches below run the CUDA-core fold
  int e = make_plan(&j, 1, &o, &p);
  if (e != VL_OK) return e;
  if (p->total > VL_NOALLOC_SCRATCH_BYTES) {
    snprintf(g_last_error, sizeof(g_last_error),
             "vl_prove_matmul_noalloc: job needs %zu bytes of scratch, the fixed array holds %u", p->total,
             (unsigned)VL_NOALLOC_SCRATCH_BYTES);
    vl_plan_destroy(p);
    return VL_ENOMEM;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  void* ptr = nullptr;
  e = noalloc_scratch_ptr(&ptr);
  uint8_t* ws = static_cast<uint8_t*>(ptr);
  if (e == VL_OK) e = bind_workspace(p, ws, st);  // descriptor tables into the array (synchronous)
  if (e == VL_OK) {
    const DevProof* dp = reinterpret_cast<const DevProof*>(ws + p->off_proofs);
    const FoldTask* dt = reinterpret_cast<const FoldTask*>(ws + p->off_tasks);
    const FoldTile* dl = reinterpret_cast<const FoldTile*>(ws + p->off_tiles);
    vl_proof* dout = reinterpret_cast<vl_proof*>(ws + p->off_out);
    // The accumulators keep the previous call's sums: clear them first.
    cudaError_t ce = cudaMemsetAsync(ws + p->off_acc, 0, p->acc_bytes, st);
    const EqItem* de = reinterpret_cast<const EqItem*>(ws + p->off_eq_items);
    if (ce == cudaSuccess) ce = launch_prologue(dp, 0, 1, de, (int)p->eq_items.size(), st);
    if (ce == cudaSuccess) ce = launch_fold(dt, dl, (int)p->tiles.size(), dp, p->fold_smem, FOLD_WAIT_NS, st);
    if (ce == cudaSuccess) ce = launch_rounds(dp, 1, dout, 0, 0, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, dout, sizeof(vl_proof), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    // A failed enqueue may leave earlier kernels of this call running on the
    // array: let them finish before the lock lets the next call rebind it.
    if (ce != cudaSuccess) (void)cudaStreamSynchronize(st);
    e = cuda_status(ce, "vl_prove_matmul_noalloc");
    if (e == VL_OK && out->status != VL_OK) e = out->status;
  }
  vl_plan_destroy(p);
  return e;
  VL_ABI_CATCH(VL_ENOMEM)
}

namespace vl {

// TMA descriptor of an int16 operand of the tensor-core fold: uint16 boxes of
// 64 columns (128 bytes, 128-byte swizzle) by 128 rows for row dots, 128
// columns by 128 rows (no swizzle: rows of 256 contiguous bytes stream
// better) for column sums; out-of-range entries read as zero.  False unless
// the base is 16-byte aligned and rows are a multiple of 16 bytes apart.
bool encode_tc_operand(const void* base, int64_t rows, int64_t cols, int64_t ld, int32_t mode, void* out) {
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld & 7)) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)(mode == MODE_ROWDOT ? TC_KP : TC_M),
                             (cuuint32_t)(mode == MODE_ROWDOT ? TC_M : TC_KS)};
  const cuuint32_t estr[2] = {1, 1};
  return enc(static_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base), dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             mode == MODE_ROWDOT ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void set_last_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

bool ws_owned_by(const void* owner, const void* ws) { return owns_workspace(owner, ws); }
void ws_claim(const void* owner, const void* ws) { claim_workspace(owner, ws); }
void ws_release(const void* owner) { release_workspaces(owner); }

}  // namespace vl

// ---------------------------------------------------------------------------
// Batched-claim sumcheck: the products' prologues (member transcripts) and
// folds as in a plan, then the batch kernels (kernels_batch.cu).

namespace {

struct BatchLayout {
  vl_plan* p = nullptr;
  int K = 0, d1 = 0, k = 0, P2 = 1;
  std::vector<LkItem> items;  // round items, round by round
  std::vector<int> roff;      // round t: items [roff[t], roff[t + 1])
  size_t off_state = 0, off_w = 0, off_c = 0, off_tree = 0, off_part = 0, off_items = 0, off_cout = 0,
         off_aout = 0, off_bout = 0, off_proof = 0, total = 0;
};

constexpr int BT_PAIRS = 1024;

int batch_layout(const vl_job* jobs, int32_t njobs, BatchLayout* L) {
  if (!jobs || njobs < 1 || njobs > 65535) return VL_EINVAL;
  vl_batch_opts o{};
  o.persistent = 2;  // phase launches: the batch kernels replace the rounds
  int e = make_plan(jobs, njobs, &o, &L->p);
  if (e != VL_OK) return e;
  vl_plan* p = L->p;
  L->K = njobs;
  L->k = p->proofs[0].k;
  L->d1 = p->proofs[0].d1;
  for (DevProof& P : p->proofs) {
    if (P.k != L->k) return VL_ESHAPE;  // one inner dimension per batch
    P.member1 = P.job + 1;
    P.nmembers = njobs;
  }
  while (L->P2 < njobs) L->P2 <<= 1;
  // round items: each proof's pairs in chunks, round by round (slots = item index)
  L->roff.assign(L->d1 + 2, 0);
  for (int t = 1; t <= L->d1; t++) {
    L->roff[t] = (int)L->items.size();
    const int h = 1 << (L->d1 - t);
    for (int s = 0; s < njobs; s++)
      for (int k0 = 0; k0 < h; k0 += BT_PAIRS)
        L->items.push_back(LkItem{s, k0, std::min(h, k0 + BT_PAIRS), (int)L->items.size()});
  }
  L->roff[L->d1 + 1] = (int)L->items.size();
  size_t off = p->total;
  auto take = [&off](size_t bytes) {
    const size_t o2 = off;
    off = align_up(off + bytes);
    return o2;
  };
  L->off_state = take(sizeof(BtState));
  L->off_w = take(sizeof(Fr) * njobs);
  L->off_c = take(sizeof(Fr) * njobs);
  L->off_tree = take(64 * (size_t)L->P2);
  L->off_part = take(sizeof(Fr) * 2 * std::max<size_t>(1, L->items.size()));
  L->off_items = take(sizeof(LkItem) * std::max<size_t>(1, L->items.size()));
  L->off_cout = take(sizeof(vl_fr) * njobs);
  L->off_aout = take(sizeof(vl_fr) * njobs);
  L->off_bout = take(sizeof(vl_fr) * njobs);
  L->off_proof = take(sizeof(vl_batch_proof));
  L->total = off;
  return VL_OK;
}

}  // namespace

extern "C" size_t vl_batch_workspace_bytes(const vl_job* jobs, int32_t njobs) {
  VL_ABI_TRY
  BatchLayout L;
  const int e = batch_layout(jobs, njobs, &L);
  const size_t total = e == VL_OK ? L.total : 0;
  if (L.p) vl_plan_destroy(L.p);
  return total;
  VL_ABI_CATCH(0)
}

// A batch bound to one workspace at a time: the plan of its products, the
// layout and the batch state template (re-uploaded every run: the kernels
// update it).
struct vl_claims_plan {
  BatchLayout L;
  uint64_t seed = 0;
  uint8_t* bound_ws = nullptr;
  BtState S{};
  ~vl_claims_plan() {
    if (L.p) vl_plan_destroy(L.p);
    vl::ws_release(this);
  }
};

extern "C" int32_t vl_claims_plan_create(const vl_job* jobs, int32_t njobs, uint64_t seed, vl_claims_plan** plan) {
  VL_ABI_TRY
  if (!plan) return VL_EINVAL;
  *plan = nullptr;
  std::unique_ptr<vl_claims_plan> C(new (std::nothrow) vl_claims_plan);
  if (!C) return VL_ENOMEM;
  const int e = batch_layout(jobs, njobs, &C->L);
  if (e != VL_OK) return e;
  C->seed = seed;
  for (DevProof& P : C->L.p->proofs) P.seed = seed;  // member transcripts use the batch seed
  BtState& S = C->S;
  S.K = C->L.K;
  S.d1 = C->L.d1;
  S.status = VL_OK;
  S.P2 = C->L.P2;
  S.seed = seed;
  S.inv2 = to_mont(fr_inv_canonical(fr_small(2)));
  for (int t = 1; t <= C->L.d1; t++) {
    S.pbeg[t] = C->L.roff[t];
    S.pend[t] = C->L.roff[t + 1];
  }
  *plan = C.release();
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" size_t vl_claims_plan_workspace_bytes(const vl_claims_plan* plan) { return plan ? plan->L.total : 0; }

extern "C" void vl_claims_plan_destroy(vl_claims_plan* plan) { delete plan; }

extern "C" int32_t vl_claims_plan_run(vl_claims_plan* C, void* workspace, size_t workspace_bytes, vl_batch_proof* out,
                                      vl_fr* claims, vl_fr* a, vl_fr* b, int32_t out_space, void* stream) {
  VL_ABI_TRY
  if (!C || !workspace || !out || !claims || !a || !b || (out_space != VL_DEVICE && out_space != VL_HOST))
    return VL_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) & (ALIGN - 1)) return VL_EINVAL;
  BatchLayout& L = C->L;
  if (workspace_bytes < L.total) return VL_ENOMEM;
  vl_plan* p = L.p;
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int e = VL_OK;
  cudaError_t ce = cudaSuccess;
  if (C->bound_ws != ws || !owns_workspace(C, ws)) {  // first run here, or another plan's tables replaced ours
    BtState& S = C->S;
    S.w = reinterpret_cast<Fr*>(ws + L.off_w);
    S.c = reinterpret_cast<Fr*>(ws + L.off_c);
    S.tree = ws + L.off_tree;
    S.part = reinterpret_cast<Fr*>(ws + L.off_part);
    S.c_out = reinterpret_cast<vl_fr*>(ws + L.off_cout);
    S.a_out = reinterpret_cast<vl_fr*>(ws + L.off_aout);
    S.b_out = reinterpret_cast<vl_fr*>(ws + L.off_bout);
    S.out = reinterpret_cast<vl_batch_proof*>(ws + L.off_proof);
    e = bind_workspace(p, ws, st);  // descriptor tables, member fields included (synchronous)
    if (e == VL_OK && !L.items.empty())
      ce = cudaMemcpyAsync(ws + L.off_items, L.items.data(), sizeof(LkItem) * L.items.size(), cudaMemcpyHostToDevice,
                           st);
    if (e == VL_OK && ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (e != VL_OK) return e;
    if (ce != cudaSuccess) return cuda_status(ce, "vl_claims_plan_run: bind");
    C->bound_ws = ws;
    claim_workspace(C, ws);
  }
  e = stage_host_operands(p, ws, st);
  if (e != VL_OK) return e;
  BtState* dS = reinterpret_cast<BtState*>(ws + L.off_state);
  const DevProof* dp = reinterpret_cast<const DevProof*>(ws + p->off_proofs);
  const FoldTask* dt = reinterpret_cast<const FoldTask*>(ws + p->off_tasks);
  const FoldTile* dl = reinterpret_cast<const FoldTile*>(ws + p->off_tiles);
  const TcTile* dc = reinterpret_cast<const TcTile*>(ws + p->off_tc_tiles);
  const EqItem* de = reinterpret_cast<const EqItem*>(ws + p->off_eq_items);
  const LkItem* di = reinterpret_cast<const LkItem*>(ws + L.off_items);
  const int np = (int)p->jobs.size();
  const int K = L.K;
  ce = cudaMemcpyAsync(dS, &C->S, sizeof(BtState), cudaMemcpyHostToDevice, st);  // status, pointers (the plan keeps the source)
  if (ce == cudaSuccess) ce = cudaMemsetAsync(ws + p->off_ctl, 0, p->off_acc + p->acc_bytes - p->off_ctl, st);
  if (ce == cudaSuccess) ce = launch_prologue(dp, 0, np, de, (int)p->eq_items.size(), st);
  if (ce == cudaSuccess)
    ce = launch_fold_dual(reinterpret_cast<const DualTile*>(ws + p->off_dual_tiles), (int)p->dual_tiles.size(), dp,
                          wait_ns(p), st);
  if (ce == cudaSuccess) ce = launch_fold_tc(dc, (int)p->tc_tiles.size(), dp, wait_ns(p), st);
  if (ce == cudaSuccess) ce = launch_fold(dt, dl, (int)p->tiles.size(), dp, p->fold_smem, wait_ns(p), st);
  if (ce == cudaSuccess) ce = launch_batch_claims(dp, np, dS, st);
  for (int t = 1; t <= L.d1 && ce == cudaSuccess; t++)
    ce = launch_batch_round(dp, dS, t, di + L.roff[t], L.roff[t + 1] - L.roff[t], st);
  if (ce == cudaSuccess) ce = launch_batch_finish(dp, np, dS, L.k, st);
  const cudaMemcpyKind kind = out_space == VL_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, ws + L.off_proof, sizeof(vl_batch_proof), kind, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(claims, ws + L.off_cout, sizeof(vl_fr) * K, kind, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(a, ws + L.off_aout, sizeof(vl_fr) * K, kind, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(b, ws + L.off_bout, sizeof(vl_fr) * K, kind, st);
  if (ce == cudaSuccess && out_space == VL_HOST) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_status(ce, "vl_claims_plan_run");
  if (out_space == VL_HOST && out->status != VL_OK) return out->status;
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" int32_t vl_prove_matmul_batched(const vl_job* jobs, int32_t njobs, uint64_t seed, void* workspace,
                                           size_t workspace_bytes, vl_batch_proof* out, vl_fr* claims, vl_fr* a,
                                           vl_fr* b, void* stream) {
  vl_claims_plan* C = nullptr;
  int e = vl_claims_plan_create(jobs, njobs, seed, &C);
  if (e != VL_OK) return e;
  e = vl_claims_plan_run(C, workspace, workspace_bytes, out, claims, a, b, VL_HOST, stream);
  vl_claims_plan_destroy(C);
  return e;
}
