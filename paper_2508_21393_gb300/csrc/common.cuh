// Device-side descriptors shared by the prover kernels and the host engine.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fr.cuh"
#include "verilora.h"

namespace vl {

// How a fold task reduces its stored matrix.
//   COLSUM: out[c] = sum_r W[r] . M[r, c]   (reduce over stored rows)
//   ROWDOT: out[r] = sum_c M[r, c] . W[c]   (reduce over stored columns)
// f_A comes from op(P) folded against E_u over its m rows: COLSUM when P is
// stored m x k, ROWDOT when stored k x m (trans).  f_B comes from op(Q)
// folded against E_v over its n columns: ROWDOT when Q is stored k x n,
// COLSUM when stored n x k (trans).
enum : int32_t { MODE_COLSUM = 0, MODE_ROWDOT = 1 };

// Per-proof mutable state (device, in the workspace).
struct ProofScratch {
  uint8_t state[32];  // transcript state after the u, v squeezes (then after each round)
  Fr corrA;           // 2^15 . sum E_u  (Montgomery), int16 offset correction
  Fr corrB;           // 2^15 . sum E_v
  int32_t status;
  int32_t pad[7];
  Fr r;               // batched rounds: the latest challenge (Montgomery)
};

// Batched rounds (one launch per round over all proofs): the pairs of one
// proof's round evaluated by one CTA.
struct RoundItem {
  int32_t proof;  // DevProof index
  int32_t j0, j1; // pairs [j0, j1) of the round
  int32_t pad;
};
static constexpr int RB_PAIRS = 256;    // pairs per item
static constexpr int RB_THREADS = 128;  // threads of a pass CTA
static constexpr int RB_WARPS = 4;      // proofs per transcript CTA (one warp each)
static constexpr int RB_TAIL_LOG = 9;   // rounds with at most 2^9 pairs run in the per-proof tail
// Rounds of a proof with d1 variables that run batched: those with more than
// 2^RB_TAIL_LOG pairs (round t has 2^(d1 - t) pairs).
__host__ __device__ __forceinline__ int batched_rounds(int d1) {
  return d1 - RB_TAIL_LOG - 1 > 0 ? d1 - RB_TAIL_LOG - 1 : 0;
}

// Per-proof read-only descriptor (device copy of the plan).
struct DevProof {
  int32_t m, k, n, d0, d1, d2;
  int32_t tp, tq;
  int32_t dtypeA, dtypeB;  // VL_I16 or VL_FR_MONT
  int32_t member1;         // batched proofs: 1 + the product's index in the batch (0: a proof of its own)
  int32_t nmembers;        // batched proofs: products in the batch
  uint64_t seed;
  uint8_t binds[96];
  Fr* eqA;                 // m entries, E_u in double-Montgomery form (x.R^2)
  Fr* eqB;                 // n entries, E_v
  uint32_t* eqA_soa;       // the same tables limb-major: [8][pitch] words (row-dot
  uint32_t* eqB_soa;       //   weights are fetched as [8 x box] tensor boxes)
  int32_t soa_pitchA, soa_pitchB;  // words per limb row, multiples of 4
  unsigned long long* accA;  // k x 8 column sums (f_A numerators)
  unsigned long long* accB;  // k x 8
  Fr* fA;                  // 2^d1 working vector for the rounds (Montgomery)
  Fr* fB;
  ProofScratch* scr;
  int32_t ntiles;          // fold tiles of this proof (both tasks)
  int32_t job;             // index of the proof in the caller's job list (output slot)
  int32_t tabA, tabB;      // weight tables each side needs: TAB_LIMBS and/or TAB_BYTES
  int32_t fdirA, fdirB;    // 1: the fold writes f_A (f_B) itself, reduced (no accumulators)
  Fr* fac;                 // eq factor tables: [lo_u 256 | hi_u 256 | lo_v 256 | hi_v 256]
  uint32_t* w8A;           // tensor-core weights: E_u bytes as fp16, [ceil(m / 128) x 2 chunks] x 4 KB
  uint32_t* w8B;           // E_v bytes
  const struct GivenPoint* given;  // non-null: start state and (u, v) given (chained proofs), no squeeze
  Fr* rch;                 // non-null: the rounds store their challenges r_1..r_d1 here (Montgomery)
};

// Start of a proof whose point is fixed by an earlier proof (a member of a
// chained proof): the transcript state the proof starts from, and u (d0
// entries), v (d2 entries) in Montgomery form.
static constexpr int GIVEN_VARS = 16;  // log2 of VL_MAX_REDUCE
struct GivenPoint {
  uint8_t state[32];
  Fr u[GIVEN_VARS];
  Fr v[GIVEN_VARS];
};

// Weight tables of one side of a proof.
//   TAB_LIMBS: E in Montgomery limbs, entry-major (eqA) and limb-major (soa)
//   TAB_BYTES: the 32 bytes of each E entry as fp16 values, in the shared-
//              memory operand layout of the tensor-core fold (per 64-entry
//              chunk: [8 entry groups][4 byte groups][8 entries][8 bytes]),
//              zero past the last entry up to a multiple of 128 entries
enum : int32_t { TAB_LIMBS = 1, TAB_BYTES = 2 };

// Eq-table expansion: entries [i0, i1) of one side's table.
struct EqItem {
  int32_t proof, side;
  int32_t i0, i1;
};
static constexpr int EQ_CHUNK = 1024;
static constexpr int EQ_FAC = 256;  // entries of each factor table

// Persistent step: work items in queue order.
enum : int32_t { STEP_PROLOGUE = 0, STEP_FOLD = 1 };
struct StepItem {
  int32_t kind;
  int32_t idx;  // proof (prologue) or fold tile
};
// Dynamic shared memory of the prologue and rounds block functions.
static constexpr int PRO_SMEM = 18816;
static constexpr int RND_SMEM = 1792;
// Prologue items run this many proofs ahead of their fold tiles in the queue.
static constexpr int STEP_LOOKAHEAD = 256;

// Control block of a persistent step (zeroed every pass): the queue head
// padded to its own 128 bytes, then ready[nproofs], done[nproofs].
static constexpr int STEP_CTL_HEAD_INTS = 32;

struct FoldTask {
  const void* mat;  // stored matrix (device)
  int64_t ld;       // elements between stored rows
  int32_t rows, cols;
  int32_t mode, dtype;
  int32_t proof, side;  // side 0: weights E_u, output accA; side 1: E_v, accB
  int32_t bulk;         // 1: int16 tiles staged by TMA tensor copies (alignment checked on the host)
  int32_t box_w;        // TMA box: columns (a multiple of 8)
  int32_t box_h;        //          rows
  int32_t pad;
  const void* tmap;     // TMA tensor map of the stored matrix (device, 64-byte aligned)
  const void* etmap;    // TMA tensor map of the limb-major weights (row dots)
};

// Tensor-core fold tile: stored lines [w0, w0 + nw) (columns for COLSUM,
// rows for ROWDOT; nw <= 128), reduced over [k0, k0 + nk) (k0 a multiple of
// 128, nk <= 32768).  Everything a CTA needs to stream the tile is resolved
// at bind time, so taking a tile is one 64-byte load.
struct TcTile {
  const void* tmap;         // TMA tensor map of the stored matrix (device)
  const uint32_t* w8;       // fp16 weight-byte table of the task's side
  unsigned long long* acc;  // accumulator rows of lines w0.. (8 per line), or
  Fr* f;                    //   when the tile covers the whole reduction: f[w0..] written reduced
  const Fr* corr;           //   minus this offset correction (Montgomery)
  int32_t mode;
  int32_t w0, nw;
  int32_t k0, nk;
  int32_t proof;            // for status reports
  int32_t task;             // host bookkeeping
  int32_t pad;
};
static_assert(sizeof(TcTile) == 72, "tile descriptor");

// Dual tensor-core fold tile: one 128-row strip of a stored int16 matrix W
// (rows and columns multiples of 128) that one proof folds as row dots (its
// lines are W's rows) and another as column sums (lines are W's columns),
// streamed once in stages of 128 columns [k0, k0 + nk).  The row dots of the
// strip's rows run across the tile (written reduced to fR when the tile
// covers every column, else added to accR); each stage's column sums cover
// only the strip's rows and are added to accC.
struct DualTile {
  const void* tmap;          // TMA map of W with row-dot boxes (64 columns x 128 rows, 128B swizzle)
  const uint32_t* w8R;       // fp16 weight bytes of the row-dot side (over W's columns)
  const uint32_t* w8C;       // fp16 weight bytes of the column-sum side (over W's rows)
  unsigned long long* accR;  // row-dot accumulators of the strip's first row, or
  Fr* fR;                    //   its f entries (whole-reduction tiles)
  const Fr* corrR;           //   minus this offset correction (Montgomery)
  unsigned long long* accC;  // column-sum accumulators of W's column 0 (8 per column)
  int32_t w0;                // first row of the strip
  int32_t k0, nk;            // columns [k0, k0 + nk), nk a multiple of 128
  int32_t proofR, proofC;    // for status reports
  int32_t taskR, taskC;      // host bookkeeping
  int32_t pad[3];
};
static_assert(sizeof(DualTile) == 96, "dual tile descriptor");
static constexpr int TC_M = 128;        // lines per tile (MMA M)
static constexpr int TC_KS = 128;       // reduction entries per pipeline stage
static constexpr int TC_KP = 64;        // entries per weight-table chunk and per row-dot TMA box (two per stage)
static constexpr int TC_SEG = 16384;    // reduction entries per tile (default; a multiple of TC_KS, at most 32768)
static constexpr int TC_CONV_WARPS = 8;   // int16 -> fp16 byte operands
static constexpr int TC_DRAIN_WARPS = 8;  // TMEM -> digit sums (two groups of four lane quarters)
static constexpr int TC_ISSUERS = 4;      // MMA issuing threads (one per warp): two (lo, hi) pairs
// warp 0 producer, warp 1 first MMA issuer (TMEM owner), then converters,
// drainers, and the other MMA issuers last
static constexpr int TC_THREADS = 32 * (1 + TC_ISSUERS + TC_CONV_WARPS + TC_DRAIN_WARPS);
// Ring depths.
#ifndef TC_NR
#define TC_NR 4  // operand (TMA) stages, 32 KB of shared memory each
#endif
static constexpr int TC_NW = 4;   // weight stages, 8 KB each
static constexpr int TC_NC = 2;   // converted-operand stages (TMEM, 128 columns each: lo 64, hi 64)
static constexpr int TC_NA = 4;   // accumulator buffers (TMEM, 64 columns each: lo 32, hi 32)
static constexpr int TC_HR = 32;  // stage-header ring (> TC_NR + TC_NC + TC_NA)
static_assert(TC_HR > TC_NR + TC_NC + TC_NA, "header ring");
static constexpr int TC_SMEM = 1024 + TC_NR * 32768 + TC_NW * 8192 + 5120 + 4096 + 3072;

struct FoldTile {
  int32_t task;
  int32_t r0, r1;  // stored rows [r0, r1)
  int32_t c0, c1;  // stored columns [c0, c1)
  int32_t pad[3];
};

// Fold tile geometry (threads per CTA and per-thread vector widths).
static constexpr int FOLD_THREADS = 256;
static constexpr int COLSUM_VEC = 4;                              // int16 columns per thread
static constexpr int COLSUM_TILE_COLS = FOLD_THREADS * COLSUM_VEC;  // 1024
// Register-load and Montgomery row-dot paths: 4 rows per warp, 32-row blocks.
static constexpr int ROWDOT_ROWS_PER_WARP = 4;
static constexpr int FB_BLOCK_ROWS = (FOLD_THREADS / 32) * ROWDOT_ROWS_PER_WARP;  // 32
// Bulk row-dot path: 8 rows per warp, 64-row blocks; a tile is 2 blocks
// sharing its staged weights.
static constexpr int BULK_ROWS_PER_WARP = 8;
static constexpr int ROWDOT_BLOCK_ROWS = (FOLD_THREADS / 32) * BULK_ROWS_PER_WARP;  // 64
static constexpr int ROWDOT_TILE_ROWS = 2 * ROWDOT_BLOCK_ROWS;                      // 128
static constexpr int ROWDOT_TILE_COLS = 1024;
static constexpr int FR_COLSUM_TILE_COLS = FOLD_THREADS;          // Montgomery operands: 1 col/thread
// TMA pipeline: NSTAGE shared-memory slots of SLOT_BYTES; a slot holds up to
// STAGE_BYTES of operand entries followed by the weights those entries need
// (column sums: the stage's rows, 32 bytes each; row dots: 8 limb rows of the
// stage's columns).
static constexpr int NSTAGE = 4;
static constexpr int STAGE_BYTES = 16384;
static constexpr int SLOT_BYTES = 24576;
static constexpr int ROWDOT_STAGE_COLS = STAGE_BYTES / (ROWDOT_BLOCK_ROWS * 2);  // 128
static constexpr int FOLD_SMEM_HEAD = 128;  // mbarriers
// Default bound on any single wait for a bulk copy (ns of %globaltimer).
static constexpr unsigned long long FOLD_WAIT_NS = 2000000000ull;

// Dynamic shared memory a fold tile needs (bytes): the TMA pipeline for
// int16 operands, or the staged weights of the register-load and Montgomery
// paths, whichever is larger.
inline int fold_tile_smem(int mode, int dtype, int tile_rows, int tile_cols) {
  const int staged = mode == MODE_COLSUM ? tile_rows * 32 : ((tile_cols + 3) & ~3) * 32;
  const int pipe = dtype == VL_I16 ? NSTAGE * SLOT_BYTES : 0;
  return FOLD_SMEM_HEAD + (staged > pipe ? staged : pipe);
}

// Prologue in two launches: per proof the transcript start, squeezes, eq
// factor tables and offset corrections; then the eq tables chunk by chunk.
// proofs: the plan's proof table; [p0, p1) the proofs whose transcripts run;
// items: their eq chunks (proof indices into `proofs`).
cudaError_t launch_prologue(const DevProof* proofs, int p0, int p1, const EqItem* items, int nitems,
                            cudaStream_t st);
// Raise the fold kernel's dynamic shared-memory limit (call before capture).
cudaError_t fold_set_smem(int smem_bytes);
cudaError_t launch_fold(const FoldTask* tasks, const FoldTile* tiles, int ntiles,
                        const DevProof* proofs, int smem_bytes, unsigned long long wait_ns, cudaStream_t st);
// Tensor-core fold of int16 operands (kernels_fold_tc.cu): CTA b of the
// grid takes tiles b, b + grid, b + 2 grid, ... (tiles sorted longest first).
cudaError_t fold_tc_prepare();
cudaError_t launch_fold_tc(const TcTile* tiles, int ntiles, const DevProof* proofs, unsigned long long wait_ns,
                           cudaStream_t st);
// Dual tiles (kernels_fold_tc.cu): CTA b takes tiles b, b + grid, ...
cudaError_t fold_dual_prepare();
cudaError_t launch_fold_dual(const DualTile* tiles, int ntiles, const DevProof* proofs, unsigned long long wait_ns,
                             cudaStream_t st);
// Linear zkMat (kernels_linear.cu): the statement and the device buffers of
// one proof, in the workspace.  The tensor-core fold reduces every matrix
// over one logical dimension (rows when red_rows, else columns) with that
// dimension's eq weights, leaving a vector over the other ("lines").
struct LinDev {
  int32_t rows, cols, d0, d1, nmats;
  int32_t red_rows;                // 1: reduce over rows (weights E_x); 0: over columns (E_y)
  int32_t lines;                   // entries of each folded vector
  int32_t nblk;                    // inner sums per matrix: ceil(lines / 2^s), s = ceil(d_lines / 2)
  uint64_t seed;
  Fr coeffs[VL_LIN_MAX];           // canonical
  uint8_t binds[VL_LIN_MAX][32];
  uint32_t S[8];                   // transcript state after the squeezes (big-endian words)
  Fr corr;                         // 2^15 . sum of the reduced side's eq table (Montgomery)
  Fr* fac;                         // eq factors: [lo_x 256 | hi_x 256 | lo_y 256 | hi_y 256]; lo of the
                                   //   reduced side double-Montgomery, all others Montgomery
  uint32_t* w8;                    // reduced side's eq table as fp16 bytes (fold weights)
  Fr* f;                           // one segment per tile: nmats x lines, M_q~ folded (Montgomery)
  unsigned long long* acc;         // several segments: nmats x lines x 8 column sums
  Fr* part;                        // nmats x nblk inner sums (Montgomery)
  ProofScratch* scr;               // status (the fold's DevProof points here)
  Fr* e2;                          // short reductions: the reduced side's eq table, double-Montgomery
};
// Linear zkMat, short reductions (at most LIN_SHORT_MAX entries): the fold on
// CUDA cores, one thread per line (a tensor-core stage would be mostly
// padding).  One item per block of LIN_SHORT_LINES lines of one matrix.
static constexpr int LIN_SHORT_MAX = 128;
static constexpr int LIN_SHORT_LINES = 256;
struct LinShort {
  const int16_t* base;  // stored matrix (device)
  int64_t ld;           // elements between stored rows
  int32_t proof, q;     // proof, matrix of the proof
  int32_t w0, nw;       // lines [w0, w0 + nw): stored rows (ROWDOT) or columns (COLSUM)
  int32_t mode, red;    // MODE_ROWDOT / MODE_COLSUM, reduced entries per line
};
static_assert(sizeof(LinShort) == 40, "short item");
// Lookup argument (kernels_lookup.cu): one LkDev per proof, in the workspace.
static constexpr int LK_MAX_L = VL_LOOKUP_MAX_LOG_D;
struct LkDev {
  int32_t n, L, log2_n, sE;        // entries, log2 D, log2 N, variables of the low eq block
  int64_t t0;
  uint64_t seed;
  int64_t rows, cols, ld;          // S as stored (row-major, k = row . cols + col)
  const int16_t* S;
  uint8_t bind[32];
  Fr beta, alpha, c_nd, Cb;        // Montgomery; c_nd = N / D; Cb = alpha^2 X1 - X2 (table side's cube sum)
  Fr claim, half_t;                // running claim; 2^-t during the high rounds
  Fr ct;                           // prod_{v < t} eqf(u_v, r_v): eq(u, .) folded by the bound variables
  Fr ctj;                          // the same product over the bound table variables (eq(u_low, .))
  Fr inv2, inv6;                   // 1/2, 1/6 (Montgomery)
  Fr u[LK_MAX_L], r[LK_MAX_L];     // challenges (Montgomery)
  uint32_t St[8];                  // transcript state (big-endian words)
  int32_t pbeg[LK_MAX_L + 1], pend[LK_MAX_L + 1];  // partial-sum slots of each round (1-based)
  int32_t xbeg, xend;              // slots of the table-side sums X1, X2
  int32_t tail, pad_tail;          // first round run by the per-proof tail kernel
  Fr* loP;                         // eq over the last m variables of u, levels m = 0..sE at offset 2^m - 1
  Fr* hiP;                         // eq over the last m variables of u_1..u_{L-sE}, levels m = 0..L-sE-1
  Fr* Binv;                        // 1 / (beta + t0 + j), N (gather source, never folded)
  Fr* Tb;                          // beta + t0 + j, N (gather source)
  Fr* WB; Fr* WE; Fr* WT; Fr* WM;  // table side: B, eq(u_low, .) (for Cb only), T + beta, m (folded in place)
  Fr* VA; Fr* VS;                  // folded A and S + beta, D/2 each
  uint32_t* counts;                // N multiplicities
  Fr* part;                        // partial sums (12 per slot)
  ProofScratch* scr;               // status
};
// A block of work of one proof: entries or pairs [k0, k1), partial slot.
struct LkItem {
  int32_t proof, k0, k1, slot;
};
static constexpr int LK_THREADS = 256;
static constexpr int LK_PPT_LOG = 2;
static constexpr int LK_PPT = 1 << LK_PPT_LOG;  // pairs per thread in a round pass
static constexpr int LK_PAIRS = LK_THREADS * LK_PPT;  // pairs per round item
static constexpr int LK_ENTRIES = 1024;   // table entries per table item (one batch inversion)
static constexpr int LK_HIST = 8192;      // S entries per histogram item
#ifndef LK_TAIL_LOG
#define LK_TAIL_LOG 11  // rounds of at most 2^LK_TAIL_LOG pairs run in one block per proof
#endif
cudaError_t launch_lookup_setup(LkDev* Ls, int np, const LkItem* fac_items, int nfac, const LkItem* hist_items,
                                int nhist, const LkItem* tab_items, int ntab, cudaStream_t st);
// Round t: nhi items of proofs in their high rounds, then nlo items of
// proofs in their table rounds.
cudaError_t launch_lookup_round(LkDev* Ls, int np, int t, const LkItem* items, int nhi, int nlo,
                                vl_lookup_proof* out, cudaStream_t st);
cudaError_t launch_lookup_finish(LkDev* Ls, int np, vl_lookup_proof* out, cudaStream_t st);
cudaError_t launch_lookup_passes(LkDev* Ls, int t, const LkItem* items, int nhi, int nlo, cudaStream_t st);

// Batched-claim sumcheck (kernels_batch.cu): the batch transcript and
// buffers, in the workspace.
struct BtState {
  int32_t K, d1, status, P2;       // products, rounds, status, leaves of the Merkle trees (2^t >= K)
  uint64_t seed;
  Fr rho, claim, inv2;             // Montgomery
  Fr r[VL_MAX_ROUNDS];
  uint32_t St[8];                  // batch transcript state (big-endian words)
  int32_t pbeg[VL_MAX_ROUNDS + 1], pend[VL_MAX_ROUNDS + 1];  // partial-sum slots of each round
  Fr* w;                           // rho^i
  Fr* c;                           // claims (Montgomery)
  uint8_t* tree;                   // 2 P2 nodes of 32 bytes (leaves at [P2, 2 P2), root at 1)
  Fr* part;                        // partial sums, 2 per slot (g(0), g(2))
  vl_fr* c_out;                    // canonical outputs: claims, a_i, b_i
  vl_fr* a_out;
  vl_fr* b_out;
  vl_batch_proof* out;
};
cudaError_t launch_batch_claims(const DevProof* dp, int np, BtState* B, cudaStream_t st);
cudaError_t launch_batch_round(const DevProof* dp, BtState* B, int t, const LkItem* items, int nitems,
                               cudaStream_t st);
cudaError_t launch_batch_finish(const DevProof* dp, int np, BtState* B, int k, cudaStream_t st);

// Host helpers of the engine shared with the linear prover.
bool encode_tc_operand(const void* base, int64_t rows, int64_t cols, int64_t ld, int32_t mode, void* map);
void set_last_error(const char* msg);
// Which plan's tables a workspace holds (every plan type registers here, so
// a plan re-binds when another plan has used its workspace since).
bool ws_owned_by(const void* owner, const void* ws);
void ws_claim(const void* owner, const void* ws);
void ws_release(const void* owner);
// Batches: one LinDev per proof; chunks of the reduced side's eq table as
// EqItem {proof, side (unused), i0, i1}.
// Short-reduction folds (kernels_linear.cu): f_q of every item's lines.
cudaError_t launch_linear_short(const LinDev* Ls, const LinShort* items, int nitems, cudaStream_t st);
cudaError_t launch_linear_start(LinDev* Ls, int nproofs, const EqItem* items, int nitems, cudaStream_t st);
cudaError_t launch_linear_finish(LinDev* Ls, int nproofs, int max_nblk, int max_nmats, vl_lin_proof* out,
                                 cudaStream_t st);
cudaError_t step_set_smem(int smem_bytes);
cudaError_t step_grid(int smem_bytes, int* grid);
cudaError_t launch_step(const StepItem* items, int nitems, const FoldTask* tasks, const FoldTile* tiles,
                        const DevProof* proofs, int nproofs, vl_proof* out, int* ctl, int grid, int smem_bytes,
                        unsigned long long wait_ns, int never_ready, cudaStream_t st);
// Batched rounds: round t (1-based, t <= batched_rounds(d1)) of every such
// proof.  Pass: fold with r_(t-1) (for t = 1 the fold's output is reduced)
// and evaluate the round over `nitems` items, one canonical partial triple
// per item; transcript: one warp per proof of [0, nproofs) sums its items'
// partials (items ibase[p] .. ibase[p + 1]), writes and absorbs the round
// message and squeezes r_t.  Tail: one CTA per proof runs its remaining
// rounds and writes the proof.
cudaError_t launch_rounds_pass(const DevProof* proofs, const RoundItem* items, int nitems, Fr* partials, int t,
                               cudaStream_t st);
cudaError_t launch_rounds_hash(const DevProof* proofs, int nproofs, const int* ibase, const Fr* partials,
                               vl_proof* out, int t, cudaStream_t st);
cudaError_t launch_rounds_tail(const DevProof* proofs, int nproofs, vl_proof* out, cudaStream_t st);
cudaError_t launch_rounds(const DevProof* proofs, int nproofs, vl_proof* out, int variant, int threads,
                          cudaStream_t st);
cudaError_t launch_encode(const int16_t* src, int64_t rows, int64_t cols, int64_t ld, Fr* dst,
                          cudaStream_t st);

}  // namespace vl
