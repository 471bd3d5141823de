/*
 * verilora.h - C ABI of the GB300 (sm_103a) matmul-sumcheck prover.
 *
 * What is proved.  zkMat (Sec. IV-B) proves each matrix product of a LoRA
 * step with the sumcheck protocol over multilinear extensions (Sec. II-B,
 * Eq. eq:MLE; Sec. II-C, Eq. eq:matmul and eq:zk-mle-matmul).  For
 * A = op(P) (m x k) and B = op(Q) (k x n), dimensions zero-padded to powers
 * of two D0 = 2^d0, D1 = 2^d1, D2 = 2^d2, the prover draws u in F^d0 and
 * v in F^d2 from the transcript and runs d1 rounds of sumcheck on
 *     sum_{w in {0,1}^d1} A~(u, w) . B~(w, v) = c   (c = C~(u, v) when C = A.B)
 * over the BLS12-381 scalar field (Sec. V), with SHA-256 Fiat-Shamir
 * challenges (Sec. IV-A footnote).  Commitments are outside this library:
 * every verifier evaluates the MLEs it needs directly from the matrices.
 *
 * Also proved (sections below): linear relations sum_q c_q op(M_q) = 0, the
 * parameter updates and matrix additions of Sec. IV (vl_prove_linear);
 * range lookups of int16 values in a table of consecutive integers
 * (Protocol 1, Eq. eq:lookup-sumcheck; vl_prove_lookup); and K products of
 * one inner dimension under one transcript with one random-combination
 * sumcheck (Sec. IV, putting everything together; vl_prove_matmul_batched);
 * and the chained proof of one LoRA projection, whose intermediate tensors
 * are never opened (Sec. IV, sequential composition; vl_prove_chain).
 *
 * Conventions.
 *  - Field elements (vl_fr) are canonical, 8 x 32-bit limbs, little endian.
 *  - Matrices are row-major with a leading dimension `ld` (elements between
 *    row starts, ld >= cols).  `trans` = 1 means the operand is the transpose
 *    of the stored matrix; no transpose is ever materialised.
 *  - Row bits are the high MLE variables; variable 1 is the most significant
 *    bit of an index, and sumcheck binds it first.
 *  - int16 entries are fixed-point values embedded as x mod r (x < 0 maps to
 *    r - |x|); the prover folds them without converting them to field form.
 *  - The transcript format (start state, absorb, counter-mode squeeze) is
 *    this library's own; it is written out in the transcript source header.
 *
 * Ownership.  The caller owns every buffer: operand matrices, the device
 * workspace (size from vl_workspace_bytes / vl_plan_workspace_bytes, any
 * alignment >= 256 bytes), the proof outputs and the CUDA stream.  The
 * library never calls cudaMalloc: its only device memory of its own is the
 * fixed scratch array of vl_prove_matmul_noalloc, part of the loaded
 * module.  (The proving server stages proofs in pinned host buffers it
 * allocates and frees itself.)  Operands must stay unchanged until the
 * call's stream work has finished.
 *
 * Process-wide state (each guarded for calls from several host threads):
 * the autotuner's cache (vl_autotune_clear), the per-workspace record of
 * which plan's tables a workspace holds (vl_workspace_forget), the scratch
 * array and lock of vl_prove_matmul_noalloc, and one-time kernel attribute
 * settings.  vl_last_error() is per thread.
 *
 * Errors.  Every call returns VL_OK (0) or one of the codes below; no C++
 * exception crosses this interface (a failed host allocation inside the
 * library returns VL_ENOMEM, or 0 from a *_workspace_bytes call, with a
 * message in vl_last_error()).  vl_strerror() names a code.  A failed call
 * leaves outputs unspecified.
 */
#ifndef VERILORA_H
#define VERILORA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define VL_OK 0
#define VL_EINVAL 1   /* null pointer, bad enum, bad leading dimension       */
#define VL_ESHAPE 2   /* inner dimensions differ, empty or oversized dims    */
#define VL_ENOMEM 3   /* workspace smaller than required, or host allocation */
#define VL_ECUDA 4    /* a CUDA runtime call failed                          */
#define VL_ETIMEOUT 5 /* a bounded device-side wait gave up                  */
#define VL_REJECT 6   /* vl_verify_matmul: the proof does not verify         */
#define VL_ELOOKUP 7  /* vl_prove_lookup: a value lies outside its table     */

/* Element types of a vl_mat. */
#define VL_I16 1     /* int16 fixed-point, 2 bytes                            */
#define VL_I64 2     /* int64, 8 bytes (claimed products for the verifier)    */
#define VL_FR_MONT 3 /* field element in Montgomery form (x.2^256 mod r), 32 B */

/* Memory spaces. */
#define VL_DEVICE 0
#define VL_HOST 1

/* Limits: reduced dimensions (m and n) <= 2^16 (exactness of the 64-bit column
 * sums of the int16 fold), k <= 2^VL_MAX_ROUNDS. */
#define VL_MAX_ROUNDS 24
#define VL_MAX_REDUCE (1 << 16)

typedef struct vl_fr {
  uint32_t limb[8];
} vl_fr;

typedef struct vl_mat {
  const void* data; /* device or host pointer, per `space`; caller-owned   */
  int64_t rows;     /* stored rows                                         */
  int64_t cols;     /* stored columns                                      */
  int64_t ld;       /* elements between consecutive stored rows (>= cols)  */
  int32_t dtype;    /* VL_I16, VL_I64 or VL_FR_MONT                        */
  int32_t trans;    /* 1: the operand is the stored matrix transposed      */
  int32_t space;    /* VL_DEVICE or VL_HOST                                */
  int32_t reserved; /* must be 0                                           */
} vl_mat;

/* Public transcript inputs of one proof: a 64-bit seed and three 32-byte
 * commitment stand-ins (bindings to P, Q, C; zeros when unused). */
typedef struct vl_fs_init {
  uint64_t seed;
  uint8_t bind[3][32];
} vl_fs_init;

/* One proof.  g[i] = (g_i(0), g_i(1), g_i(2)) for rounds i < d1; entries at
 * i >= d1 are zero.  `state` is the transcript state after the last absorb.
 * `status` is VL_OK for a finished proof. */
typedef struct vl_proof {
  int32_t m, k, n, d0, d1, d2;
  int32_t status;
  int32_t reserved;
  vl_fr c;
  vl_fr g[VL_MAX_ROUNDS][3];
  vl_fr a_r;
  vl_fr b_r;
  uint8_t state[32];
} vl_proof;

/* One product to prove: C = op(P) . op(Q). */
typedef struct vl_job {
  vl_mat P;
  vl_mat Q;
  vl_fs_init fs;
} vl_job;

/* Batch options; 0 in any field selects the default or the autotuned value. */
typedef struct vl_batch_opts {
  int32_t colsum_rows;   /* stored rows per column-sum fold tile              */
  int32_t rowdot_cols;   /* stored columns per row-dot fold tile              */
  int32_t persistent;    /* 1: one persistent launch (CUDA-core fold);
                            0 or 2: phase launches (prologue, fold, rounds)  */
  int32_t groups;        /* phase launches: proof groups pipelined across
                            three streams (0: 1, no overlap)                 */
  int32_t fold_engine;   /* phase launches: 0 tensor cores for every int16
                            operand that TMA can address (16-byte aligned
                            base, rows and columns multiples of 8 entries),
                            CUDA cores for the rest; 1 CUDA cores only      */
  int32_t use_graph;     /* 1: capture vl_plan_run in a CUDA graph; 2: never   */
  int32_t timing_runs;   /* runs kept by vl_plan_phase_ms (0: 64)             */
  int32_t wait_limit_us; /* bound on any single device-side wait, in us (0: 2 s);
                            a wait that runs out sets the proof's status to
                            VL_ETIMEOUT and its CTA returns                  */
  int32_t rounds_variant; /* rounds kernel: CTAs per SM, 7, 6, 5, 4, 3 or 2
                            (0: 7); 7 to 4 set the register budget, 3 and 2 also
                            cap residency (fewer proofs share an SM); 8:
                            batched rounds, one launch per round for the
                            vector work of all proofs and one for their
                            transcript steps (one-group phase launches) */
  int32_t rounds_threads; /* rounds kernel threads per proof: 128, 192 or 256
                            (0: 128)                                         */
  int32_t tc_seg;        /* tensor-core fold: reduced entries per tile, a
                            multiple of 128 up to 32768 (0: 16384); shorter
                            segments spread narrow operands over more SMs */
  int32_t test_never_ready; /* fault injection for tests: 1 + index of a job
                            whose prologue never signals ready, so that its
                            fold tiles exhaust their bounded wait and report
                            VL_ETIMEOUT (persistent mode); 0: off            */
  int32_t fold_dual;     /* tensor-core fold, one proof group: a matrix that
                            one job folds as row dots and another as column
                            sums (the frozen W of X.W and dY.W^T), with rows
                            and columns multiples of 128, is streamed once for
                            both (one conversion, two MMA sets): 1: on, 0: off
                            (default: on the LoRA steps it is slower than two
                            passes, the second one hitting L2)               */
} vl_batch_opts;

typedef struct vl_plan vl_plan; /* opaque batched-step plan */

/* Version of this ABI (major * 100 + minor). */
int32_t vl_version(void);

/* Name of a status code (static string). */
const char* vl_strerror(int32_t status);

/* Detail of the last VL_ECUDA failure on the calling thread (the failing
 * step and the CUDA error string), or of a host-side failure reported as
 * VL_ENOMEM; "" if none.  Valid until the next call. */
const char* vl_last_error(void);

/*
 * Device workspace needed to prove `njobs` products in one batch, in bytes.
 * Host-space operands add staging room for one device copy of each distinct
 * host matrix.  Returns 0 on invalid input.
 */
size_t vl_workspace_bytes(const vl_job* jobs, int32_t njobs, const vl_batch_opts* opts);

/*
 * Prove one product (Sec. II-C via zkMat, Sec. IV-B).  P, Q: device or host
 * int16 / Montgomery matrices; fs: transcript inputs; workspace: caller's
 * device buffer of at least vl_workspace_bytes() for this single job; out:
 * host proof.  Runs on `stream` (a cudaStream_t, NULL for the legacy
 * stream) and synchronises it before returning.
 */
int32_t vl_prove_matmul(const vl_mat* P, const vl_mat* Q, const vl_fs_init* fs,
                        void* workspace, size_t workspace_bytes, vl_proof* out, void* stream);

/*
 * Prove all jobs of a batch (the products of a LoRA step, Protocol 2 phases 1
 * and 2) in one pass of the device pipeline.  out: njobs proofs in
 * `out_space` memory; for VL_HOST the call synchronises the stream, for
 * VL_DEVICE it returns with the work enqueued.  Each proof is byte-identical
 * to the same job proved alone.
 */
int32_t vl_prove_batch(const vl_job* jobs, int32_t njobs, void* workspace, size_t workspace_bytes,
                       vl_proof* out, int32_t out_space, void* stream, const vl_batch_opts* opts);

/*
 * Reusable plan for a fixed batch (same shapes, same operand pointers): the
 * descriptor tables are built once, and vl_plan_run replays a CUDA graph of
 * the whole step after its first call.  The plan copies `jobs`.
 */
int32_t vl_plan_create(const vl_job* jobs, int32_t njobs, const vl_batch_opts* opts, vl_plan** plan);
size_t vl_plan_workspace_bytes(const vl_plan* plan);
/* Enqueue one proving pass; out: njobs proofs in `out_space` memory (VL_HOST
 * synchronises, and returns the first non-OK proof status, e.g. VL_ETIMEOUT).  Host-space operands are copied in on every run.  The first
 * run on a workspace uploads the plan's descriptor tables into it (a
 * synchronous copy); later runs reuse them.  Several plans may take turns on
 * one workspace (same base pointer): a plan re-uploads its tables when
 * another plan used the workspace since its last run.  Anything else that
 * writes to the workspace between runs must be followed by
 * vl_workspace_forget.  Runs that overlap in time on the GPU must use
 * disjoint workspaces. */
int32_t vl_plan_run(vl_plan* plan, void* workspace, size_t workspace_bytes, vl_proof* out,
                    int32_t out_space, void* stream);
/* Workspace bookkeeping (the paper has no counterpart: plans are this
 * library's way of replaying one step's proofs).  The library records, per
 * workspace base pointer, which plan's tables the workspace holds (for plans
 * of every kind: matmul, linear, lookup, claims).
 * Call this after anything other than a plan run wrote to a workspace, and
 * before a buffer freed and reallocated at the same address is given to a
 * plan again: it forgets the record, so the next plan run there re-uploads
 * its tables.  Host only; no CUDA call.  Returns 1 if a record was dropped,
 * 0 if there was none, -VL_EINVAL for a null pointer. */
int32_t vl_workspace_forget(const void* workspace);
/* Number of kernel launches one vl_plan_run enqueues (graph nodes included). */
int32_t vl_plan_launches(const vl_plan* plan);
/*
 * Device time of the most recent proving passes of a plan, from CUDA events
 * the plan records on its stream at the phase boundaries of every run
 * (inside the graph when one is used).  ms: max_runs x 3 floats per run:
 * [0] accumulator clear + prologue (transcripts, challenges, eq tables),
 * [1] fold, [2] claims + sumcheck rounds.  Fills the last min(max_runs, runs
 * since the previous reset, opts.timing_runs) runs, oldest first, waiting for the last
 * one to finish.  reset != 0 restarts the count.  Returns the number of runs
 * filled, or -status on error.
 */
int32_t vl_plan_phase_ms(vl_plan* plan, float* ms, int32_t max_runs, int32_t reset);
void vl_plan_destroy(vl_plan* plan);

/*
 * Verify a proof on the host (Def. def:ip verifier; Sec. V-B completeness).
 * P, Q, C are HOST matrices (C: the claimed m x n product, VL_I64 or VL_I16).
 * Replays the transcript, checks g_i(0) + g_i(1) against the running claim,
 * the final claim against a_r . b_r, and evaluates A~(u, r), B~(r, v) and
 * C~(u, v) directly (the stand-in for commitment openings).
 * Returns VL_OK (accept), VL_REJECT, or an input error.
 */
int32_t vl_verify_matmul(const vl_mat* P, const vl_mat* Q, const vl_mat* C, const vl_fs_init* fs,
                         const vl_proof* proof);

/*
 * Prove one product without allocating device memory and without a
 * caller-provided workspace.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- for example a plug-in
 * running inside a host application that owns all device memory through its
 * own pool and forbids allocations outside it, or a latency-critical loop
 * that cannot take the implicit device synchronisation of cudaMalloc/cudaFree.
 *
 * Scratch: one file-scope device array of VL_NOALLOC_SCRATCH_BYTES inside the
 * library.  Every GPU on which the library is used holds it until the process
 * exits.  A job whose scratch does not fit is refused with VL_ENOMEM and a
 * message in vl_last_error() (a single 7B- or 13B-shaped projection product
 * fits; the scratch grows with k and the row/column counts).
 * Set-up: the first call on each device, with that device current, looks up
 * the array's device address; make that first call before any stream capture
 * on the device.  The address is kept for the life of the process, so this
 * entry point must not be called on a device after cudaDeviceReset there.
 * Sharing: all calls use the same array, which keeps the previous call's
 * contents (the call clears what must start at zero).  Two calls running on
 * the GPU at the same time would race on it; within one process the entry
 * point prevents that by holding a lock for the whole call, which ends only
 * after its stream has finished.
 * P, Q: DEVICE matrices (VL_I16 or VL_FR_MONT); fs: transcript inputs; out:
 * host proof.  The result is byte-identical to vl_prove_matmul's.  Calls no
 * cudaMalloc, cudaFree or other allocating routine.
 */
#define VL_NOALLOC_SCRATCH_BYTES (8u << 20)
int32_t vl_prove_matmul_noalloc(const vl_mat* P, const vl_mat* Q, const vl_fs_init* fs, vl_proof* out,
                                void* stream);

/*
 * Encode int16 fixed-point values into field elements in Montgomery form
 * (Sec. II-C embeds integer tensors into F; x < 0 maps to r - |x|):
 * dst[i * cols + j] = (src[i, j] mod r) . 2^256 mod r, 32 bytes each, dense
 * row-major.  src and dst are device pointers; runs asynchronously on
 * `stream`.  The output can be proved with dtype VL_FR_MONT.
 */
int32_t vl_encode(const vl_mat* src, void* dst, void* stream);

/* ---------------------------------------------------------------------------
 * Linear zkMat (Sec. IV: zkMat proves matrix additions as well as products):
 * a proof that sum_q coeffs[q] * op(mats[q]) = 0 entrywise over F, by MLE
 * linearity and no sumcheck.  The transcript (domain "verilora-gb300/zklin/v1",
 * seed u64le, rows, cols, q u32le, the coefficients, one 32-byte bind per
 * matrix) gives a point (x, y), x in F^d0 over the row bits and y in F^d1 over
 * the column bits (d0 = ceil log2 rows, d1 = ceil log2 cols); the proof
 * carries e_q = M_q~(x, y) of Eq. eq:MLE (absorbed under label 'e') and the
 * final transcript state.  The verifier checks sum_q c_q e_q = 0 and
 * evaluates each M_q~(x, y) from the matrices.  The LoRA parameter update of
 * Eq. eq:grad_update_ab, A' = A - eta dA, is one such relation.
 * ------------------------------------------------------------------------- */
#define VL_LIN_MAX 16

typedef struct vl_lin_job {
  const vl_mat* mats;    /* nmats operands of one logical shape (after transposes) */
  const vl_fr* coeffs;   /* nmats canonical coefficients                           */
  const uint8_t* binds;  /* nmats x 32 bytes, or NULL for zeros                    */
  uint64_t seed;
  int32_t nmats;         /* 1 .. VL_LIN_MAX                                        */
  int32_t reserved;      /* must be 0                                              */
} vl_lin_job;

typedef struct vl_lin_proof {
  int32_t rows, cols, d0, d1, nmats;
  int32_t status;
  vl_fr evals[VL_LIN_MAX]; /* canonical; the first nmats are used              */
  uint8_t state[32];
} vl_lin_proof;

/* Device workspace vl_prove_linear needs for this batch (0 on invalid
 * arguments: see vl_prove_linear). */
size_t vl_linear_workspace_bytes(const vl_lin_job* jobs, int32_t njobs);
/* Prove a batch of 1 .. 65535 linear relations on the GPU, one independent
 * transcript each.  Operands: int16 (VL_EINVAL otherwise), logical rows and columns at
 * most VL_MAX_REDUCE (VL_ESHAPE), on the device or the host; device operands
 * with a 16-byte aligned base and a leading dimension of a multiple of 8
 * entries are read in place, all others are first copied into the
 * workspace.  workspace: device memory, 256-byte aligned, at least
 * vl_linear_workspace_bytes (VL_ENOMEM).  out: host memory for njobs proofs.
 * Synchronises `stream`.  Returns VL_OK, or the first proof's non-OK status
 * (VL_ETIMEOUT from a bounded device wait).  The prover does not check the
 * relation: a false one yields a proof that the verifier rejects. */
int32_t vl_prove_linear(const vl_lin_job* jobs, int32_t njobs, void* workspace, size_t workspace_bytes,
                        vl_lin_proof* out, void* stream);
/* Plans: the same batch proved repeatedly (a training loop's updates).  A
 * plan copies the statements (the operand descriptors, not their data: the
 * matrices are read at every run) and, on its first run with a workspace,
 * uploads its tables there (synchronising `stream`); later runs with that
 * workspace only enqueue the host-operand copies and five kernels.  The
 * workspace must not be used by anything else between runs (else call
 * vl_workspace_forget before the next run).  out_space
 * VL_DEVICE: `out` is device memory and the run is asynchronous (each
 * proof's status field reports its outcome); VL_HOST: as vl_prove_linear. */
typedef struct vl_lin_plan vl_lin_plan;
int32_t vl_lin_plan_create(const vl_lin_job* jobs, int32_t njobs, vl_lin_plan** plan);
size_t vl_lin_plan_workspace_bytes(const vl_lin_plan* plan);
int32_t vl_lin_plan_run(vl_lin_plan* plan, void* workspace, size_t workspace_bytes, vl_lin_proof* out,
                        int32_t out_space, void* stream);
/* Device times (ms) of the plan's last run (waits for it): ms[0] start and eq
 * tables, ms[1] the tensor-core fold, ms[2] partial dot products and proofs. */
int32_t vl_lin_plan_phase_ms(vl_lin_plan* plan, float ms[3]);
void vl_lin_plan_destroy(vl_lin_plan* plan);
/* Verify one proof on the host against host operands (int16, int64 or
 * Montgomery): VL_OK (accept), VL_REJECT, or an argument error. */
int32_t vl_verify_linear(const vl_lin_job* job, const vl_lin_proof* proof);

/* ---------------------------------------------------------------------------
 * Lookup argument (Sec. II, lookup arguments; Protocol 1; Eq.
 * eq:lookup-sumcheck): a proof that every entry of S lies in the table
 * T = [t0, t0 + N), N = 2^log2_n (a range check, e.g. of rescale
 * remainders).  S (n entries, row-major) is padded with t0 to
 * D = max(N, 2^ceil(log2 n)) entries; with A_k = 1/(beta + S_k),
 * B_j = 1/(beta + T_j) and multiplicities m_j, a degree-3 sumcheck over the
 * log2 D variables shows that
 *   P(k) = alpha A(k) eq(u,k) (S(k) + beta) + A(k)
 *          + (N/D) (alpha^2 B(j) eq(u_low,j) (T(j) + beta) - B(j) m(j))
 * (j = k mod N, u_low the last log2 N coordinates of u) sums to
 * alpha + alpha^2.  Transcript: domain "verilora-gb300/zklookup/v1", seed
 * u64le, n, log2 D, log2 N u32le, t0 i64le, bind; squeeze beta ('b'),
 * alpha ('a'), u ('u', log2 D); per round absorb g(0), g(2), g(3) ('g') and
 * squeeze r ('r'); absorb a_r, s_r, b_r, m_r ('f').  The verifier
 * recomputes A, B, m from S and T in place of commitment openings.
 * ------------------------------------------------------------------------- */
#define VL_LOOKUP_MAX_LOG_D 24
#define VL_LOOKUP_MAX_LOG_N 16

typedef struct vl_lookup_job {
  vl_mat S;          /* int16 values, trans 0, read in row-major order      */
  int64_t t0;        /* first table value                                    */
  int32_t log2_n;    /* table size 2^log2_n, 0 .. VL_LOOKUP_MAX_LOG_N        */
  int32_t reserved;  /* must be 0                                            */
  uint64_t seed;
  uint8_t bind[32];  /* commitment stand-in for S (zeros when unused)        */
} vl_lookup_job;

typedef struct vl_lookup_proof {
  int32_t n, log2_d, log2_n, status;
  int64_t t0;
  vl_fr g[VL_LOOKUP_MAX_LOG_D][4]; /* g_t(0), g_t(1), g_t(2), g_t(3), canonical */
  vl_fr a_r, s_r, b_r, m_r;        /* A~(r), S~(r), B~(r_low), m~(r_low)        */
  uint8_t state[32];
} vl_lookup_proof;

typedef struct vl_lookup_plan vl_lookup_plan;
/* Device workspace a batch of 1 .. 65535 lookups needs (0 on invalid
 * arguments: S not int16, transposed or empty; n > 2^VL_LOOKUP_MAX_LOG_D;
 * log2_n out of range; |t0| > 2^40; reserved != 0). */
size_t vl_lookup_workspace_bytes(const vl_lookup_job* jobs, int32_t njobs);
/* Plans, as for linear proofs: the statements are copied (S's data is read
 * at every run; host S is copied into the workspace at every run), tables
 * are bound once per workspace; out_space VL_DEVICE runs asynchronously
 * (each proof's status field reports VL_OK or VL_ELOOKUP), VL_HOST
 * synchronises `stream` and returns the first non-OK status. */
int32_t vl_lookup_plan_create(const vl_lookup_job* jobs, int32_t njobs, vl_lookup_plan** plan);
size_t vl_lookup_plan_workspace_bytes(const vl_lookup_plan* plan);
int32_t vl_lookup_plan_run(vl_lookup_plan* plan, void* workspace, size_t workspace_bytes, vl_lookup_proof* out,
                           int32_t out_space, void* stream);
/* Device times (ms) of the last run: ms[0] setup (transcript start, tables,
 * multiplicities, inverses), ms[1] the sumcheck rounds run as batched passes,
 * ms[2] every proof's last rounds (at most 2^11 pairs) in one block per proof
 * and the proofs. */
int32_t vl_lookup_plan_phase_ms(vl_lookup_plan* plan, float ms[3]);
void vl_lookup_plan_destroy(vl_lookup_plan* plan);
/* One-shot: plan, run with host output, destroy. */
int32_t vl_prove_lookup(const vl_lookup_job* jobs, int32_t njobs, void* workspace, size_t workspace_bytes,
                        vl_lookup_proof* out, void* stream);
/* Host verifier against host S (int16 or int64): VL_OK, VL_REJECT or an
 * argument error (VL_EINVAL as for the prover, VL_ESHAPE when S has more
 * than 2^VL_LOOKUP_MAX_LOG_D entries). */
int32_t vl_verify_lookup(const vl_lookup_job* job, const vl_lookup_proof* proof);

/* ---------------------------------------------------------------------------
 * Batched-claim sumcheck (Sec. IV, putting everything together: claims of
 * many proving steps aggregated at random points under one Fiat-Shamir
 * transcript).  K products C_i = op(P_i) op(Q_i) with a common inner
 * dimension k are proved by ONE sumcheck over w in {0,1}^d1:
 *   member transcripts  M_i = SHA256("verilora-gb300/zkbatch/v1/member" ||
 *     seed || K, i || m_i, k, n_i || transP, transQ || three binds) give
 *     u_i, v_i (as in a single proof); c_i = sum_w A_i~(u_i,w) B_i~(w,v_i);
 *   the claims are bound by a Merkle root over SHA256(0x00 || S_i || c_i)
 *     (S_i the member state, node = SHA256(0x01 || l || r)), the batch
 *     transcript starts at SHA256("verilora-gb300/zkbatch/v1" || seed || K ||
 *     root) and squeezes rho ('p');
 *   rounds prove sum_w sum_i rho^i A_i~ B_i~ = sum_i rho^i c_i (g(0), g(2)
 *     absorbed as 'g', r squeezed); finally a_i = A_i~(u_i, r),
 *     b_i = B_i~(r, v_i), bound by a Merkle root over
 *     SHA256(0x00 || i u32le || a_i || b_i) absorbed as 'f'.
 * Each job's own fs.seed is not used (the batch seed is); its binds are.
 * ------------------------------------------------------------------------- */
typedef struct vl_batch_proof {
  int32_t K, k, d1, status;
  vl_fr g[VL_MAX_ROUNDS][3];       /* g_t(0), g_t(1), g_t(2), canonical        */
  uint8_t state[32];
} vl_batch_proof;

/* Device workspace for a batch (0 on invalid arguments or inner dimensions
 * that differ). */
size_t vl_batch_workspace_bytes(const vl_job* jobs, int32_t njobs);
/* Prove a batch on the GPU.  Operands as for vl_prove_batch; njobs <= 65535,
 * all with the same inner dimension (VL_ESHAPE otherwise).  out, claims, a,
 * b: host memory (claims, a, b hold njobs canonical elements each, in job
 * order).  Synchronises `stream`. */
int32_t vl_prove_matmul_batched(const vl_job* jobs, int32_t njobs, uint64_t seed, void* workspace,
                                size_t workspace_bytes, vl_batch_proof* out, vl_fr* claims, vl_fr* a, vl_fr* b,
                                void* stream);
/* Plans, as for single proofs: the batch (operand descriptors) is copied at
 * creation, its tables are bound to a workspace on the first run there
 * (synchronising `stream`); a run stages host operands, enqueues the
 * launches and copies the proof, claims, a and b to the given buffers in
 * out_space: VL_DEVICE asynchronously (status in out->status), VL_HOST
 * synchronously.  The workspace must not be used by anything else between
 * runs of the plan. */
typedef struct vl_claims_plan vl_claims_plan;
int32_t vl_claims_plan_create(const vl_job* jobs, int32_t njobs, uint64_t seed, vl_claims_plan** plan);
size_t vl_claims_plan_workspace_bytes(const vl_claims_plan* plan);
int32_t vl_claims_plan_run(vl_claims_plan* plan, void* workspace, size_t workspace_bytes, vl_batch_proof* out,
                           vl_fr* claims, vl_fr* a, vl_fr* b, int32_t out_space, void* stream);
void vl_claims_plan_destroy(vl_claims_plan* plan);
/* Host verifier: C[i] are the claimed products (host), checked through the
 * claims; the final values are checked against the operands. */
int32_t vl_verify_matmul_batched(const vl_job* jobs, const vl_mat* C, int32_t njobs, uint64_t seed,
                                 const vl_batch_proof* proof, const vl_fr* claims, const vl_fr* a, const vl_fr* b);

/* Autotuner (the paper has no counterpart): picks the launch and tile
 * options for `jobs` by timing candidate plans on the caller's workspace and
 * stream — coordinate descent from `base` (NULL: defaults) over the fold
 * engine, the dual tiles (fold_dual), tc_seg, rounds_variant (including the
 * batched rounds, 8),
 * rounds_threads and, where CUDA-core fold tiles run, colsum_rows /
 * rowdot_cols (the persistent launch is not a candidate: its CUDA-core fold
 * is slower than phase launches); each candidate is run once untimed
 * and `runs` times timed (0: 3), its time the median.  Candidates needing more
 * workspace than workspace_bytes (which must also hold njobs proofs at its
 * end) are skipped.  The result is cached per shape signature (dimensions,
 * transposes, dtypes, memory spaces, TMA addressability of every operand) for
 * the process: a later call with the same shapes returns the cached options
 * without running.  *best receives the options, *best_ms (optional) the time
 * of one run.  Synchronises `stream`.  Proofs do not depend on the options. */
int32_t vl_autotune(const vl_job* jobs, int32_t njobs, const vl_batch_opts* base, void* workspace,
                    size_t workspace_bytes, void* stream, int32_t runs, vl_batch_opts* best, float* best_ms);
/* Forget every cached autotuning result. */
void vl_autotune_clear(void);

/* ---------------------------------------------------------------------------
 * Proving server: continuous batching under a device-memory budget.  The
 * paper proves one step at a time and has no counterpart; this is the
 * serving pattern around its prover.
 *
 * The caller gives the server a device arena (its admission budget, any
 * alignment; the server sub-allocates plan workspaces and proof outputs from
 * it and allocates no device memory).  Requests are submitted as job lists
 * (e.g. one projection's products) and proved in arrival order: a worker
 * thread merges the queued requests that fit the largest free arena block
 * (at most max_batch_requests) into one batch whenever one of max_inflight
 * streams is free, runs it as one plan on that stream (batches overlap on
 * the device), and when it completes copies each request's proofs to its
 * `out` (host memory, njobs proofs) and reports the request as done with its
 * submit-to-completion latency.  Operands may be device matrices (resident,
 * e.g. frozen weights) or host matrices (staged into the batch's arena block;
 * pinned host memory keeps the copies asynchronous); they must stay unchanged
 * until the request is done.  A request that cannot fit even an empty arena
 * is done with VL_ENOMEM; one the library rejects is done with that status.
 * Proofs are identical to proving the same jobs alone.
 * ------------------------------------------------------------------------- */
typedef struct vl_server vl_server;

typedef struct vl_server_opts {
  void* arena;                /* device buffer owned by the caller          */
  size_t arena_bytes;         /* admission budget                            */
  int32_t max_inflight;       /* batches on the device at once (0: 4)        */
  int32_t max_batch_requests; /* requests merged into one batch (0: 64)     */
  int32_t wait_limit_us;      /* as vl_batch_opts.wait_limit_us              */
  int32_t reserved[4];        /* must be 0                                   */
} vl_server_opts;

typedef struct vl_server_done {
  uint64_t ticket;
  int32_t status;     /* VL_OK, or the first non-OK proof / launch status   */
  int32_t batch;      /* batch the request ran in (-1: never admitted)      */
  double latency_ms;  /* submit to completion seen by the server            */
  double dev_start_ms; /* the batch's device interval, in ms of the GPU's   */
  double dev_end_ms;   /*   clock since the server started (CUDA events on  */
                       /*   the batch's stream around its work; 0 if never  */
                       /*   admitted)                                       */
} vl_server_done;

typedef struct vl_server_stats {
  int64_t submitted, completed, failed, batches, proofs, queued;
  int64_t launched;   /* batches put on the device so far                   */
} vl_server_stats;

/* Start a server (and its worker thread) on the current device. */
int32_t vl_server_create(const vl_server_opts* opts, vl_server** out);
/* Queue one request; *ticket identifies it in vl_server_poll. */
int32_t vl_server_submit(vl_server* server, const vl_job* jobs, int32_t njobs, vl_proof* out,
                         uint64_t* ticket);
/* Move up to `max` completed requests into done[]; *ndone = how many.
 * Non-blocking. */
int32_t vl_server_poll(vl_server* server, vl_server_done* done, int32_t max, int32_t* ndone);
/* Counters (queued = requests waiting for admission). */
int32_t vl_server_stats_get(vl_server* server, vl_server_stats* out);
/* Finish the batches on the device, stop the worker, free host resources.
 * Queued requests that were never admitted are dropped. */
int32_t vl_server_destroy(vl_server* server);

/* ---------------------------------------------------------------------------
 * Chained proof of one LoRA projection (Sec. IV, putting everything together:
 * sequential composition, where the claim a sub-proof leaves on an
 * intermediate tensor is reduced to claims on the tensors that made it
 * instead of being opened).  In the X.A.B convention the projection has
 * outputs Y = X.W + H.B, dX = dY.W^T + dH.A^T, dA = X^T.dH, dB = H^T.dY and
 * the fixed-point rescales (Sec. IV-A, quantisation z = zeta z' + r with
 * zeta = 2^8) X.A + 2^7 = 2^8 H + rhoH and dY.B^T + 2^7 = 2^8 dH + rhodH,
 * whose remainders rhoH, rhodH are witnesses (their range is a lookup,
 * vl_prove_lookup).  Ten matmul sumchecks (Eq. eq:zk-mle-matmul) run under
 * one transcript:
 *   S0 = SHA256("verilora-gb300/zkchain/v1" || seed u64le || n, d, k, r u32le
 *               || the seven binds);  squeeze 'p': u_Y, v_Y, u_dX, v_dX,
 *               u_dA, v_dA, u_dB, v_dB (log2 of n, k, n, d, d, r, r, k
 *               entries) -> S1;
 *   stage 1, member p starting at SHA256(S1 || 'M' || p u32le), each at its
 *     given point (no u, v squeeze; then absorb c, rounds, absorb a_r, b_r):
 *     0 X.W and 1 H.B at (u_Y, v_Y), 2 dY.W^T and 3 dH.A^T at (u_dX, v_dX),
 *     4 X^T.dH at (u_dA, v_dA), 5 H^T.dY at (u_dB, v_dB);
 *   S2 = SHA256(S1 || 'L' || the six final member states); the claims left
 *     on H and dH sit at p1 = (u_Y, r^1), p2 = (r^5, u_dB), q1 = (u_dX, r^3),
 *     q2 = (r^4, v_dA) (r^p: member p's round challenges);
 *     e = (rhoH~(p1), rhoH~(p2), rhodH~(q1), rhodH~(q2)) absorbed as 'e' -> S3;
 *   stage 3, members from SHA256(S3 || 'M' || p): 6, 7 X.A at p1, p2;
 *     8, 9 dY.B^T at q1, q2 (their claims must equal 2^8 H~ + rho~ - 2^7 J~
 *     at the point, J the all-ones n x r matrix);
 *   final state SHA256(S3 || 'Z' || the four stage-3 final member states).
 * H, dH, X.A and dY.B^T are never opened; the verifier opens X, W, A, B, dY,
 * rhoH, rhodH and checks the four output claims against the claimed outputs.
 * ------------------------------------------------------------------------- */
#define VL_CHAIN_MEMBERS 10
#define VL_CHAIN_MAX_RANK 256
typedef struct vl_chain_job {
  /* int16 matrices, stored as named (trans = 0): X n x d, W d x k, A d x r,
   * B r x k, dY n x k, H, dH, rhoH, rhodH n x r.  Device matrices for the
   * prover, host matrices for the verifier.  n, d, k <= VL_MAX_REDUCE,
   * r <= VL_CHAIN_MAX_RANK. */
  vl_mat X, W, A, B, dY, H, dH, rhoH, rhodH;
  uint64_t seed;
  uint8_t bind[7][32]; /* X, W, A, B, dY, rhoH, rhodH: commitment stand-ins */
} vl_chain_job;

typedef struct vl_chain_proof {
  int32_t n, d, k, r;
  int32_t status;   /* VL_OK, or the first non-OK member status */
  int32_t reserved;
  vl_proof sub[VL_CHAIN_MEMBERS]; /* members 0..9 as above; their `state` is
                                     the member's final transcript state */
  vl_fr e[4];                     /* the remainder evaluations, canonical */
  uint8_t state[32];              /* final chain state */
} vl_chain_proof;

/* Device workspace for a batch of chained proofs (0 on invalid input). */
size_t vl_chain_workspace_bytes(const vl_chain_job* jobs, int32_t njobs);
/* Prove `njobs` projections (independent chains, one batch of launches).
 * out: host, njobs proofs.  Synchronises `stream`; returns the first
 * non-OK member status. */
int32_t vl_prove_chain(const vl_chain_job* jobs, int32_t njobs, void* workspace, size_t workspace_bytes,
                       vl_chain_proof* out, void* stream);
/* The same batch proved repeatedly: the member plans are built once
 * (vl_chain_plan_create copies the jobs) and bound to a workspace on its
 * first run there; each run synchronises `stream`. */
typedef struct vl_chain_plan vl_chain_plan;
int32_t vl_chain_plan_create(const vl_chain_job* jobs, int32_t njobs, vl_chain_plan** plan);
size_t vl_chain_plan_workspace_bytes(const vl_chain_plan* plan);
int32_t vl_chain_plan_run(vl_chain_plan* plan, void* workspace, size_t workspace_bytes, vl_chain_proof* out,
                          void* stream);
void vl_chain_plan_destroy(vl_chain_plan* plan);
/* Host verifier of one chained proof: job holds HOST matrices (H and dH are
 * not read); Y (n x k), dX (n x d), dA (d x r), dB (r x k) are the claimed
 * outputs (VL_I64 or VL_I16 host matrices).  Returns VL_OK, VL_REJECT or an
 * input error. */
int32_t vl_verify_chain(const vl_chain_job* job, const vl_mat* Y, const vl_mat* dX, const vl_mat* dA,
                        const vl_mat* dB, const vl_chain_proof* proof);

#ifdef __cplusplus
}
#endif

#endif /* VERILORA_H */
