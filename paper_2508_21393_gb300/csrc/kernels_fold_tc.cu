// Tensor-core fold of int16 operands (tcgen05.mma with TMEM operands and
// accumulators, TMA tensor copies, mbarrier pipelines).
//
// The fold f[w] = sum_i E_i . x[i, w] (Sec. II-C: A~(u, w) is the eq-weighted
// sum of column w; row dots likewise) is an integer matrix-vector product with
// 255-bit weights.  Write each weight as 32 bytes, E_i = sum_b 2^(8b) e[i, b],
// and each offset entry p = x + 2^15 (in [0, 2^16)) as two bytes,
// p = lo + 2^8 hi.  Then
//     D_lo[w, b] = sum_i lo[w, i] e[i, b],   D_hi[w, b] = sum_i hi[w, i] e[i, b]
// are two dense products (M = 128 lines w, N = 32 bytes b, K = the reduced
// index i), and
//     sum_i E_i p[w, i] = sum_{t=0}^{32} 2^(8t) s_t,  s_t = D_lo[w, t] + D_hi[w, t-1].
// All operands are integers in [0, 255] (exact in fp16); a product is at most
// 255^2, so over one 128-entry pipeline stage each of D_lo and D_hi is below
// 255^2 . 128 < 2^23 and fp32 accumulation is exact.  Both accumulators of a
// stage start at 2^23 (one MMA of constants each), which puts them in
// [2^23, 2^24), where the fp32 bit pattern is 0x4B000000 + D: the drainers
// add bit patterns as 32-bit integers, s_t += bits(D_lo[t]) +
// bits(D_hi[t-1]) in one three-input add, and remove the offsets once per
// tile.  At the end of a tile the 33
// digit sums become the eight 64-bit column sums sum_j 2^(32j) col_j of the
// CUDA-core fold (col_7 also takes s_32 . 2^32), added with red.add, so the
// rounds reduce them unchanged (Montgomery reduction, minus 2^15 . sum E).
//
// Roles in a CTA (one CTA per SM; CTA b takes tiles b, b + grid, ... of a
// list sorted longest first), each running at its own pace and linked only by
// mbarriers:
// A pipeline stage is 128 lines x 128 entries: one accumulation period.
//   warp 0       producer: per stage the operand (row dots: two boxes of 64
//                entries x 128 lines, 128B-swizzled; column sums: one box of
//                128 lines x 128 entries) into one of TC_NR shared-memory
//                slots, and the stage's 8 KB of fp16 weight bytes into one of
//                TC_NW slots
//   warps 1, 18-20  MMA issuers (warp 1 also owns TMEM, 512 columns): a
//                pair per stage parity, in each pair one thread for the lo
//                and one for the hi products.  One thread issues an MMA only
//                every ~140 cycles, whatever N, while the SM runs several
//                issuers' MMAs at once; so per stage each thread issues the
//                MMA of constants (accumulator := 2^23) before the operand is
//                converted, then 8 MMAs (K = 16) with A read from TMEM and B
//                (weights) from shared memory
//   warps 2-9    converters: one thread per (line, half of the stage's 128
//                entries) reads its entries from the box, forms the fp16
//                lo/hi operand rows and stores them to TMEM (one of TC_NC
//                operand buffers) with tcgen05.st
//   warps 10-17  drainers: accumulator buffer -> per-line digit sums (two
//                groups of four warps, one warp per TMEM lane quarter, one
//                group digits 0-15, the other 16-32); tile epilogue
// TMEM columns: accumulator buffer a at 64a ([lo 32 | hi 32]), operand
// buffer c at 64 TC_NA + 128c ([lo 64 | hi 64], two fp16 per column).
// Stage headers (tile, stage) sit in a ring of TC_HR entries, longer than
// the stages any role can be ahead of another.  Every wait is bounded; a
// wait that runs out marks the proof VL_ETIMEOUT, and the CTA drains its
// copies and MMAs before it frees TMEM and returns.
#include <atomic>
#include <mutex>

#include "fold_dev.cuh"
#include "fr_dev.cuh"

namespace vl {
namespace {

constexpr int SM_RAW = 0;                          // TC_NR x 32 KB of int16 operand
constexpr int SM_W = SM_RAW + TC_NR * 32768;       // TC_NW x 8 KB of fp16 weight bytes
constexpr int SM_ACONST = SM_W + TC_NW * 8192;    // 128 x 16 fp16, K-major: column 0 = 256
constexpr int SM_BCONST = SM_ACONST + 4096;        // 16 x 32 fp16, MN-major: row 0 = 32768
constexpr int SM_XCH = SM_BCONST + 1024;           // 128 lines x 4 u64: drainer groups' column exchange
constexpr int SM_HDR = SM_XCH + 4096;              // TC_HR stage headers
constexpr int SM_BAR = SM_HDR + TC_HR * 48;
// Completion of stage s's MMAs (both issuers of its pair) is one barrier of
// a ring of TC_ND: the converters (TMEM operand reuse), the producer (weight
// slot reuse) and the drainers (accumulator ready) all wait on it.  TC_ND
// exceeds the lead any waiter can have, so no phase is lapped.
constexpr int TC_ND = 16;
constexpr int TC_PAIRS = TC_ISSUERS / 2;
// Pair g takes the stages s = g (mod TC_PAIRS): every operand, weight and
// accumulator barrier (s mod TC_NC, TC_NW, TC_NA) belongs to one pair.
static_assert(TC_NC % TC_PAIRS == 0 && TC_NW % TC_PAIRS == 0 && TC_NA % TC_PAIRS == 0, "rings per pair");
static_assert(TC_ND > TC_NW && TC_ND > TC_NC && TC_ND >= TC_NA, "stage-done ring");
constexpr int NBAR = 2 * TC_NR + TC_NC + TC_NA + TC_NW + TC_ND + 3;
constexpr int SM_TMEM = SM_BAR + NBAR * 8;
static_assert(SM_TMEM + 16 <= TC_SMEM - 1024, "shared-memory layout");
constexpr uint32_t TMEM_COLS = 512;

constexpr uint32_t ACONV_COL = 64 * TC_NA;
static_assert(ACONV_COL + 128 * TC_NC <= TMEM_COLS, "TMEM columns");

// Instruction descriptor of kind::f16: fp32 accumulator, fp16 A and B,
// A K-major (from TMEM), B MN-major, N = 32, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 16) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle: core matrices of 8 x 16 bytes
// stored contiguously, `lbo` bytes apart along K and `sbo` bytes apart along
// M or N.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | (1ull << 46);
}

// D (TMEM) (+)= A (shared memory) . B (shared memory).
__device__ __forceinline__ void umma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// D (TMEM) (+)= A (TMEM, 128 lanes x 8 columns) . B (shared memory).
__device__ __forceinline__ void umma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Arrive on `bar` once every MMA this thread issued so far has completed.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define TC_R8(b) "=r"(r[b + 0]), "=r"(r[b + 1]), "=r"(r[b + 2]), "=r"(r[b + 3]), "=r"(r[b + 4]), "=r"(r[b + 5]), \
                 "=r"(r[b + 6]), "=r"(r[b + 7])

// 16 columns into r[OFF .. OFF + 15].
template <int OFF>
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : TC_R8(OFF), TC_R8(OFF + 8)
      : "r"(taddr));
}
// 32 columns into r[0 .. 31].
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : TC_R8(0), TC_R8(8), TC_R8(16), TC_R8(24)
      : "r"(taddr));
}
// 8 columns into r[OFF .. OFF + 7].
template <int OFF>
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : TC_R8(OFF)
               : "r"(taddr));
}
#undef TC_R8
// 1 column into r[OFF].
template <int OFF>
__device__ __forceinline__ void tmem_ld1(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[OFF]) : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 consecutive columns of this warp's lane quarter from r[0..15].
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Two fp16 values from bytes of t selected by `sel` (bytes 0x64 fill the
// high halves): 0x64bb is 1024 + bb exactly, minus 1024 leaves bb.
__device__ __forceinline__ uint32_t bytes_f16x2(uint32_t t, uint32_t sel) {
  const uint32_t v = __byte_perm(t, 0x64646464u, sel);
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(0x64006400u));
  return r;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete is
// suspended in hardware (woken when the phase completes, or after ~1 us)
// instead of polling, which would take issue slots from the working warps.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(1000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: a non-blocking test first (most phases are complete when
// asked), then suspending waits; gives up after wait_ns of %globaltimer
// (read only when the first suspending wait fails).
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, unsigned long long wait_ns) {
  if (mbar_test_wait(bar, parity)) return true;
  if (mbar_try_wait_sleep(bar, parity)) return true;
  const uint64_t deadline = global_ns() + wait_ns;
  while (!mbar_try_wait_sleep(bar, parity))
    if (global_ns() > deadline) return false;
  return true;
}

// A bounded wait taken by a whole warp: it succeeds only if every lane's did,
// so the warp never splits before a .sync.aligned instruction.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, unsigned long long wait_ns) {
  return __all_sync(0xffffffffu, tc_wait(bar, parity, wait_ns));
}

__device__ __forceinline__ uint32_t fbits_add(uint32_t a, uint32_t b) {
  return __float_as_uint(__fadd_rn(__uint_as_float(a), __uint_as_float(b)));
}

// One pipeline stage as every role sees it (written by the producer).
struct StageHdr {
  int32_t tile;   // -1: end marker
  int32_t stage;  // stage within the tile
  int32_t nst;    // stages of the tile
  int32_t mode;
  int32_t nw;     // lines of the tile
  int32_t pad;
  unsigned long long* acc;  // accumulator rows of the tile's first line, or
  Fr* f;                    //   f entries of the tile's first line (whole-reduction tiles)
  const Fr* corr;
};
static_assert(sizeof(StageHdr) == 48, "stage header");

struct TcBars {
  uint32_t b;
  __device__ uint32_t raw_full(int s) const { return b + 8 * s; }
  __device__ uint32_t raw_empty(int s) const { return b + 8 * (TC_NR + s); }
  __device__ uint32_t conv_full(int c) const { return b + 8 * (2 * TC_NR + c); }
  __device__ uint32_t acc_empty(int a) const { return b + 8 * (2 * TC_NR + TC_NC + a); }
  __device__ uint32_t w_full(int w) const { return b + 8 * (2 * TC_NR + TC_NC + TC_NA + w); }
  __device__ uint32_t done(int s) const { return b + 8 * (2 * TC_NR + TC_NC + TC_NA + TC_NW + s % TC_ND); }
  __device__ uint32_t fin() const { return b + 8 * (2 * TC_NR + TC_NC + TC_NA + TC_NW + TC_ND); }
  // drainer groups' column exchange for whole-reduction tiles
  __device__ uint32_t xch_full() const { return b + 8 * (2 * TC_NR + TC_NC + TC_NA + TC_NW + TC_ND + 1); }
  __device__ uint32_t xch_empty() const { return b + 8 * (2 * TC_NR + TC_NC + TC_NA + TC_NW + TC_ND + 2); }
};
// parity of stage s's phase on its done barrier
__device__ __forceinline__ uint32_t done_parity(int s) { return (uint32_t)(s / TC_ND) & 1; }

__device__ __forceinline__ void mark_timeout(const DevProof* proofs, const TcTile* tiles, int tile) {
  atomicExch(&proofs[tiles[tile < 0 ? 0 : tile].proof].scr->status, VL_ETIMEOUT);
}

// Add one (lo, hi) accumulator pair (lo at ta, hi at ta + 32, both started
// at 2^23: bit patterns 0x4B000000 + D) to the digit sums s_t, t in [T0, T1]:
// dg[t - T0] += bits(D_lo[t]) + bits(D_hi[t - 1]) (D_lo[32] and D_hi[-1] are
// absent).  The two digit groups read disjoint columns: [0, 15] reads lo
// 0..15 and hi 0..14, [16, 32] reads lo 16..31 and hi 15..31.
template <int T0, int T1>
__device__ __forceinline__ void drain_pair(uint32_t ta, uint32_t (&dg)[17]) {
  static_assert((T0 == 0 && T1 == 15) || (T0 == 16 && T1 == 32), "digit groups");
  uint32_t L[32], H[32];
  if (T0 == 0) {
    tmem_ld16<0>(ta, L);         // lo 0..15
    tmem_ld16<0>(ta + 32, H);    // hi 0..15 (0..14 used)
  } else {
    tmem_ld16<16>(ta + 16, L);   // lo 16..31
    tmem_ld1<15>(ta + 47, H);    // hi 15
    tmem_ld16<16>(ta + 48, H);   // hi 16..31
  }
  tmem_wait_ld();
#pragma unroll
  for (int t = T0; t <= T1; t++) {
    if (t == 0) dg[0] += L[0];
    else if (t == 32) dg[t - T0] += H[31];
    else dg[t - T0] += L[t] + H[t - 1];
  }
}

// This warp's reads of an accumulator buffer are done: free it.
__device__ __forceinline__ void release_acc(uint32_t acc_empty) {
  tc_fence_before();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(acc_empty);
}

// The offsets in a digit sum after nst stages of PAIRS accumulator pairs
// each: 0x4B000000 per accumulator drained into it (digits 0 and 32 take one
// accumulator of a pair, the others two).
template <int PAIRS>
__device__ __forceinline__ uint32_t digit_offset(int t, int nst) {
  return (uint32_t)(nst * PAIRS * ((t == 0 || t == 32) ? 1 : 2)) * 0x4B000000u;
}

// Column sums col_j = sum_q 2^(8q) s_{4j+q} of the digits s_t, t in [T0, T1]
// (s_32 into col_7 as s_32 . 2^32); columns outside the range are 0.
template <int T0, int T1, int PAIRS>
__device__ __forceinline__ void digit_columns(const uint32_t (&dg)[17], int nst, uint64_t (&col)[8]) {
#pragma unroll
  for (int j = 0; j < 8; j++) col[j] = 0;
#pragma unroll
  for (int t = T0; t <= T1; t++) {
    const int c = t < 32 ? t >> 2 : 7, sh = t < 32 ? 8 * (t & 3) : 32;
    col[c] += (uint64_t)(dg[t - T0] - digit_offset<PAIRS>(t, nst)) << sh;
  }
}

// Combine a tile's digit sums s_t, t in [T0, T1], into the column sums
// col_j = sum_q 2^(8q) s_{4j+q} and add them to the proof's accumulators;
// s_32 goes to col_7 as s_32 . 2^32 (2^256 = 2^32 . 2^224).
template <int T0, int T1, int PAIRS>
__device__ __forceinline__ void tc_epilogue(uint32_t (&dg)[17], int nst, unsigned long long* acc) {
#pragma unroll
  for (int j = 0; j < 8; j++) {
    uint64_t c = 0;
    bool any = false;
#pragma unroll
    for (int t = T0; t <= T1; t++) {
      const int col = t < 32 ? t >> 2 : 7, sh = t < 32 ? 8 * (t & 3) : 32;
      if (col == j) {
        c += (uint64_t)(dg[t - T0] - digit_offset<PAIRS>(t, nst)) << sh;
        any = true;
      }
    }
    if (any) red_add_u64(acc + j, c);
  }
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS, 1)
    fold_tc_kernel(const TcTile* __restrict__ tiles, int ntiles, const DevProof* __restrict__ proofs,
                   unsigned long long wait_ns) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  const uint32_t raw_addr = smem_addr(tc_smem_raw);
  const uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
  uint8_t* sm = tc_smem_raw + pad;
  const uint32_t base = raw_addr + pad;
  const TcBars bars{base + SM_BAR};
  StageHdr* hdr = reinterpret_cast<StageHdr*>(sm + SM_HDR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < TC_NR; s++) {
      mbar_init(bars.raw_full(s), 1);
      mbar_init(bars.raw_empty(s), TC_CONV_WARPS);
    }
    for (int c = 0; c < TC_NC; c++) mbar_init(bars.conv_full(c), TC_CONV_WARPS);
    for (int a = 0; a < TC_NA; a++) mbar_init(bars.acc_empty(a), TC_DRAIN_WARPS);
    for (int w = 0; w < TC_NW; w++) mbar_init(bars.w_full(w), 1);
    for (int d = 0; d < TC_ND; d++) mbar_init(bars.done(d), 2);  // the lo and hi issuers of the stage commit
    mbar_init(bars.fin(), TC_ISSUERS);
    mbar_init(bars.xch_full(), TC_DRAIN_WARPS / 2);
    mbar_init(bars.xch_empty(), TC_DRAIN_WARPS / 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + SM_TMEM),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (warp >= 2 && warp < 2 + TC_CONV_WARPS) {
    // Constant operands of the init MMA: A[m][0] = 256, B[0][n] = 32768, so
    // an accumulator starts at 2^23; every other entry 0.
    const int wi = tid - 64, nw = 32 * TC_CONV_WARPS;
    uint32_t* ac = reinterpret_cast<uint32_t*>(sm + SM_ACONST);
    // A K-major: entry (m, k = 0) at byte m * 16 of the first 2 KB (k < 8).
    for (int i = wi; i < 1024; i += nw) ac[i] = (i < 512 && (i & 3) == 0) ? 0x5C00u : 0u;
    // B MN-major: row k = 0 is bytes [0, 16) of each 128-byte core matrix of
    // the first 512 bytes (k < 8).
    uint32_t* bc = reinterpret_cast<uint32_t*>(sm + SM_BCONST);
    for (int i = wi; i < 256; i += nw) bc[i] = (i < 128 && (i & 31) < 4) ? 0x78007800u : 0u;
    fence_proxy_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + SM_TMEM);
  bool ok = true;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int last_use[TC_NR], last_wuse[TC_NW];
#pragma unroll
      for (int i = 0; i < TC_NR; i++) last_use[i] = -1;
#pragma unroll
      for (int i = 0; i < TC_NW; i++) last_wuse[i] = -1;
      int s = 0;
      const int G = gridDim.x;
      int tile = blockIdx.x;
      // descriptors of this tile and the next are in registers; the one after
      // is loaded while this tile streams
      TcTile T = tile < ntiles ? tiles[tile] : TcTile{};
      TcTile Tn = tile + G < ntiles ? tiles[tile + G] : TcTile{};
      for (bool done = false; !done && ok;) {
        done = tile >= ntiles;
        TcTile Tnn{};
        if (!done && tile + 2 * G < ntiles) Tnn = tiles[tile + 2 * G];
        // after the last tile, two end markers: one for each issuer pair
        const int nst = done ? 2 : (T.nk + TC_KS - 1) / TC_KS;
        for (int st = 0; st < nst; st++, s++) {
          const int slot = s % TC_NR, use = s / TC_NR, ws = s % TC_NW, wuse = s / TC_NW;
          if (use > 0 && !tc_wait(bars.raw_empty(slot), (use - 1) & 1, wait_ns)) {
            ok = false;
            break;
          }
          hdr[s % TC_HR] = StageHdr{done ? -1 : tile, st, nst, T.mode, T.nw, 0, T.acc, T.f, T.corr};
          last_use[slot] = use;
          const uint32_t raw = base + SM_RAW + slot * 32768;
          const int kk = T.k0 + st * TC_KS;
          if (done) {
            mbar_arrive(bars.raw_full(slot));
          } else {
            // the block first (HBM latency, TC_NR stages of lookahead)
            mbar_arrive_expect_tx(bars.raw_full(slot), 32768);
            if (T.mode == MODE_ROWDOT) {
              tma_load_2d(raw, T.tmap, kk, T.w0, bars.raw_full(slot));
              tma_load_2d(raw + 16384, T.tmap, kk + TC_KP, T.w0, bars.raw_full(slot));
            } else {
              tma_load_2d(raw, T.tmap, T.w0, kk, bars.raw_full(slot));
            }
          }
          // the stage's weights once their slot is free (stage s - TC_NW's
          // MMAs completed); the barrier also publishes the header to the
          // issuers (end markers too)
          if (wuse > 0 && !tc_wait(bars.done(s - TC_NW), done_parity(s - TC_NW), wait_ns)) {
            ok = false;
            break;
          }
          last_wuse[ws] = wuse;
          if (done) {
            mbar_arrive(bars.w_full(ws));  // completes at once: no copy
            continue;
          }
          mbar_arrive_expect_tx(bars.w_full(ws), 8192);
          bulk_g2s(base + SM_W + ws * 8192, reinterpret_cast<const uint8_t*>(T.w8) + (size_t)(kk / TC_KP) * 4096,
                   8192, bars.w_full(ws));
        }
        if (!done) {
          tile += G;
          T = Tn;
          Tn = Tnn;
        }
      }
      if (!ok) mark_timeout(proofs, tiles, tile < ntiles ? tile : -1);
      // Copies still in flight must land before the CTA leaves.
      for (int i = 0; i < TC_NR; i++)
        if (last_use[i] >= 0) tc_wait(bars.raw_full(i), last_use[i] & 1, wait_ns);
      for (int i = 0; i < TC_NW; i++)
        if (last_wuse[i] >= 0) tc_wait(bars.w_full(i), last_wuse[i] & 1, wait_ns);
    }
  } else if (warp == 1 || warp >= TC_THREADS / 32 - (TC_ISSUERS - 1)) {
    // ---------------------------------------------------------------- MMA issuers
    // Pair g takes stages g, g + TC_PAIRS, ...; in a pair one thread for the
    // lo and one for the hi products.  The waits for the weights and the
    // accumulator buffer and the constant MMA (accumulator := 2^23) go ahead
    // of the wait for the converted operand; only the stage's 8 operand MMAs
    // follow it.
    if (lane == 0) {
      const int j = warp == 1 ? 0 : warp - (TC_THREADS / 32 - (TC_ISSUERS - 1)) + 1;  // 0..3
      const uint32_t plane = j & 1;
      for (int s = j >> 1;; s += TC_PAIRS) {
        const int c = s % TC_NC, a = s % TC_NA, ws = s % TC_NW;
        if (!tc_wait(bars.w_full(ws), (s / TC_NW) & 1, wait_ns)) {
          ok = false;
          break;
        }
        const int tile = hdr[s % TC_HR].tile;
        if (tile < 0) {
          umma_commit(bars.done(s));  // end marker: the drainers stop at the first one
          break;
        }
        if (s >= TC_NA && !tc_wait(bars.acc_empty(a), ((s / TC_NA) - 1) & 1, wait_ns)) {
          ok = false;
          mark_timeout(proofs, tiles, tile);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + 64 * a + 32 * plane;  // lo at +0, hi at +32
        umma_ss(d, sdesc(base + SM_ACONST, 2048, 128), sdesc(base + SM_BCONST, 512, 128), IDESC, 0);
        if (!tc_wait(bars.conv_full(c), (s / TC_NC) & 1, wait_ns)) {
          ok = false;
          mark_timeout(proofs, tiles, tile);
          break;
        }
        tc_fence_after();
        const uint32_t av = tmem + ACONV_COL + 128 * c + 64 * plane;  // lo at +0, hi at +64
        const uint32_t wts = base + SM_W + ws * 8192;
#pragma unroll
        for (int ks = 0; ks < 8; ks++) umma_ts(d, av + 8 * ks, sdesc(wts + ks * 1024, 512, 128), IDESC, 1);
        umma_commit(bars.done(s));
      }
      // every MMA this thread issued has completed before TMEM is freed
      umma_commit(bars.fin());
      tc_wait(bars.fin(), 0, wait_ns);
    }
  } else if (warp < 2 + TC_CONV_WARPS) {
    // ---------------------------------------------------------------- converters
    // Thread = line m (its TMEM lane) x half kh of the stage's 128 entries.
    const int quarter = warp & 3, kh = (warp - 2) >> 2;  // entries [64 kh, 64 kh + 64) of each stage
    const int m = 32 * quarter + lane;
    const uint32_t tq = tmem + ((uint32_t)(32 * quarter) << 16) + ACONV_COL + 32 * kh;
    int ends = 0;
    for (int s = 0;; s++) {
      const int slot = s % TC_NR, c = s % TC_NC;
      if (!warp_wait(bars.raw_full(slot), (s / TC_NR) & 1, wait_ns)) {
        ok = false;
        break;
      }
      const StageHdr& h = hdr[s % TC_HR];
      if (s >= TC_NC && !warp_wait(bars.done(s - TC_NC), done_parity(s - TC_NC), wait_ns)) {
        ok = false;
        mark_timeout(proofs, tiles, h.tile);
        break;
      }
      const int tl = h.tile;
      if (tl >= 0) {
        const uint8_t* raw = sm + SM_RAW + slot * 32768;
#pragma unroll
        for (int j2 = 0; j2 < 2; j2++) {  // 32 entries at a time: e0 = 64 kh + 32 j2
          uint32_t w[16];  // entry pairs (e0 + 2i, e0 + 2i + 1) of line m
          if (h.mode == MODE_ROWDOT) {
            // box kh [128 lines][64 entries]: chunk j of line m at 16 (j ^ (m % 8))
#pragma unroll
            for (int j = 0; j < 4; j++) {
              const uint4 v = *reinterpret_cast<const uint4*>(raw + 16384 * kh + m * 128 +
                                                              (((4 * j2 + j) ^ (m & 7)) << 4));
              w[4 * j] = v.x; w[4 * j + 1] = v.y; w[4 * j + 2] = v.z; w[4 * j + 3] = v.w;
            }
          } else {
            // box [128 entries][128 lines], no swizzle: line m of entry k at 256 k + 2 m
            const uint8_t* col = raw + 2 * m + (64 * kh + 32 * j2) * 256;
#pragma unroll
            for (int i = 0; i < 16; i++) {
              const uint32_t a = *reinterpret_cast<const uint16_t*>(col + (2 * i) * 256);
              const uint32_t b = *reinterpret_cast<const uint16_t*>(col + (2 * i + 1) * 256);
              w[i] = __byte_perm(a, b, 0x5410);
            }
          }
          uint32_t lo[16], hi[16];
#pragma unroll
          for (int i = 0; i < 16; i++) {
            const uint32_t t = w[i] ^ 0x80008000u;  // p = x + 2^15, per entry
            lo[i] = bytes_f16x2(t, 0x4240);
            hi[i] = bytes_f16x2(t, 0x4341);
          }
          tmem_st16(tq + 128 * c + 16 * j2, lo);
          tmem_st16(tq + 128 * c + 64 + 16 * j2, hi);
        }
        tmem_wait_st();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bars.conv_full(c));
        if (tl >= 0) mbar_arrive(bars.raw_empty(slot));
      }
      if (tl < 0 && ++ends == 2) break;
    }
  } else {
    // ---------------------------------------------------------------- drainers
    const int grp = (warp - 2 - TC_CONV_WARPS) >> 2, quarter = warp & 3;
    const int line = 32 * quarter + lane;
    const uint32_t tq = tmem + ((uint32_t)(32 * quarter) << 16);
    uint32_t dg[17];
#pragma unroll
    for (int t = 0; t < 17; t++) dg[t] = 0;
    int nx = 0;  // whole-reduction epilogues done (exchange barrier phases)
    for (int s = 0;; s++) {
      const int a = s % TC_NA;
      if (!warp_wait(bars.done(s), done_parity(s), wait_ns)) {
        ok = false;
        break;
      }
      const StageHdr& h = hdr[s % TC_HR];
      if (h.tile < 0) break;
      tc_fence_after();
      const uint32_t ta = tq + 64 * a;
      if (grp == 0) drain_pair<0, 15>(ta, dg);
      else drain_pair<16, 32>(ta, dg);
      release_acc(bars.acc_empty(a));
      if (h.stage == h.nst - 1) {
        if (h.f) {
          // Whole-reduction tile: group 1 hands its columns (4..7) to group 0
          // through shared memory; group 0 reduces the line's sum and stores
          // f = REDC(sum) - 2^15 . sum E (Montgomery).  The hand-over is an
          // mbarrier pair with bounded waits.
          uint64_t* xch = reinterpret_cast<uint64_t*>(sm + SM_XCH) + line * 4;
          uint64_t col[8];
          if (grp == 1) {
            if (nx > 0 && !warp_wait(bars.xch_empty(), (nx - 1) & 1, wait_ns)) {
              ok = false;
              break;
            }
            digit_columns<16, 32, 1>(dg, h.nst, col);
#pragma unroll
            for (int j = 0; j < 4; j++) xch[j] = col[4 + j];
            __syncwarp();
            if (lane == 0) mbar_arrive(bars.xch_full());
          } else {
            if (!warp_wait(bars.xch_full(), nx & 1, wait_ns)) {
              ok = false;
              break;
            }
            digit_columns<0, 15, 1>(dg, h.nst, col);
            if (line < h.nw) {
              U64x8 acc;
#pragma unroll
              for (int j = 0; j < 8; j++) acc.v[j] = col[j] + (j >= 4 ? xch[j - 4] : 0ull);
              h.f[line] = fr_sub(redc_columns_ni(acc), *h.corr);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bars.xch_empty());
          }
          nx++;
        } else if (line < h.nw) {
          unsigned long long* acc = h.acc + (size_t)line * 8;
          if (grp == 0) tc_epilogue<0, 15, 1>(dg, h.nst, acc);
          else tc_epilogue<16, 32, 1>(dg, h.nst, acc);
        }
#pragma unroll
        for (int t = 0; t < 17; t++) dg[t] = 0;
      }
    }
    if (!ok) mark_timeout(proofs, tiles, -1);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
  if (tid == 0) {
    for (int i = 0; i < NBAR; i++) mbar_inval(bars.b + 8 * i);
  }
}

// ------------------------------------------------------------------ dual tiles
//
// One stored matrix W folded both ways in one pass (DualTile): a strip of 128
// rows streamed in stages of 128 columns.  Each stage's 128 x 128 block is
// loaded once (two row-dot TMA boxes), converted once into fp16 lo and hi
// byte planes in shared memory, and read by two MMA sets as their A operand:
// K-major for the row dots (M = the strip's rows, K = the stage's columns),
// MN-major for the column sums (M = the stage's columns, K = the strip's
// rows).  The planes are 16 x 16 core matrices of 8 rows x 8 columns
// (16 bytes per row along the columns), core (rb, cb) at (16 rb + cb) x 128
// bytes: along the columns the core stride is 128 bytes, along the rows
// 2048.  The exactness of the byte-limb products is as in fold_tc_kernel
// (one accumulation period per stage, accumulators preloaded with 2^23);
// the row-dot digit sums run across the strip, the column-sum digits of a
// stage are turned into column sums and added with red.add at once.
// Roles: warp 0 producer; warps 1, 18, 19, 20 MMA issuers (row-dot lo, hi,
// column-sum lo, hi; warp 1 owns TMEM); warps 2-9 converters; warps 10-17
// drainers (both accumulator sets).  TMEM: row-dot buffers at 0 and 64,
// column-sum buffers at 128 and 192 (each [lo 32 | hi 32]).
namespace {

constexpr int DU_THREADS = 32 * (5 + TC_CONV_WARPS + TC_DRAIN_WARPS);
constexpr int DU_NR = 3;                           // raw block slots, 32 KB each
constexpr int DU_NW = 4;                           // row-dot weight slots, 8 KB each
constexpr int DS_RAW = 0;
constexpr int DS_CONV = DS_RAW + DU_NR * 32768;    // lo plane 32 KB, hi plane 32 KB
constexpr int DS_WR = DS_CONV + 65536;
constexpr int DS_WC = DS_WR + DU_NW * 8192;        // column-sum weights, two tile slots
constexpr int DS_ACONST = DS_WC + 2 * 8192;
constexpr int DS_BCONST = DS_ACONST + 4096;
constexpr int DS_XCH = DS_BCONST + 1024;
constexpr int DS_HDR = DS_XCH + 4096;
constexpr int DU_HR = 16;                          // stage-header ring (> DU_NR + 2)
constexpr int DU_ND = 16;                          // stage-done ring
constexpr int DU_NBAR = 2 * DU_NR + 1 + 4 + DU_NW + 2 + DU_ND + 3 + 2;
constexpr int DS_BAR = DS_HDR + DU_HR * 64;
constexpr int DS_TMEM = DS_BAR + DU_NBAR * 8;
constexpr int DU_SMEM = 1024 + DS_TMEM + 16;
static_assert(DU_SMEM <= 227 * 1024, "dual tile shared memory");

// Row dots: A K-major (default); column sums: A MN-major (bit 15).
constexpr uint32_t IDESC_MN_A = IDESC | (1u << 15);

struct DualHdr {
  int32_t tile;   // -1: end marker
  int32_t stage;  // stage within the tile
  int32_t nst;    // stages of the tile
  int32_t tcnt;   // tiles this CTA took before this one (column-sum weight slot and phase)
  unsigned long long* accR;
  Fr* fR;
  const Fr* corrR;
  unsigned long long* accC;  // accumulators of the stage's first column
  int64_t pad[2];
};
static_assert(sizeof(DualHdr) == 64, "dual stage header");

struct DuBars {
  uint32_t b;
  __device__ uint32_t raw_full(int s) const { return b + 8 * s; }
  __device__ uint32_t raw_empty(int s) const { return b + 8 * (DU_NR + s); }
  __device__ uint32_t conv_full() const { return b + 8 * (2 * DU_NR); }
  __device__ uint32_t acc_empty(int side, int a) const { return b + 8 * (2 * DU_NR + 1 + 2 * side + a); }
  __device__ uint32_t wr_full(int w) const { return b + 8 * (2 * DU_NR + 5 + w); }
  __device__ uint32_t wc_full(int w) const { return b + 8 * (2 * DU_NR + 5 + DU_NW + w); }
  __device__ uint32_t done(int s) const { return b + 8 * (2 * DU_NR + 7 + DU_NW + s % DU_ND); }
  __device__ uint32_t fin() const { return b + 8 * (2 * DU_NR + 7 + DU_NW + DU_ND); }
  __device__ uint32_t xch_full() const { return b + 8 * (2 * DU_NR + 8 + DU_NW + DU_ND); }
  __device__ uint32_t xch_empty() const { return b + 8 * (2 * DU_NR + 9 + DU_NW + DU_ND); }
  // a tile's column-sum weight slot is free once the MMAs of its last stage completed
  __device__ uint32_t wc_empty(int w) const { return b + 8 * (2 * DU_NR + 10 + DU_NW + DU_ND + w); }
};
__device__ __forceinline__ uint32_t du_parity(int s) { return (uint32_t)(s / DU_ND) & 1; }

__device__ __forceinline__ void du_mark_timeout(const DevProof* proofs, const DualTile* tiles, int tile) {
  const DualTile& t = tiles[tile < 0 ? 0 : tile];
  atomicExch(&proofs[t.proofR].scr->status, VL_ETIMEOUT);
  atomicExch(&proofs[t.proofC].scr->status, VL_ETIMEOUT);
}

}  // namespace

__global__ void __launch_bounds__(DU_THREADS, 1)
    fold_dual_kernel(const DualTile* __restrict__ tiles, int ntiles, const DevProof* __restrict__ proofs,
                     unsigned long long wait_ns) {
  extern __shared__ __align__(1024) uint8_t du_smem_raw[];
  const uint32_t raw_addr = smem_addr(du_smem_raw);
  const uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
  uint8_t* sm = du_smem_raw + pad;
  const uint32_t base = raw_addr + pad;
  const DuBars bars{base + DS_BAR};
  DualHdr* hdr = reinterpret_cast<DualHdr*>(sm + DS_HDR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < DU_NR; s++) {
      mbar_init(bars.raw_full(s), 1);
      mbar_init(bars.raw_empty(s), TC_CONV_WARPS);
    }
    mbar_init(bars.conv_full(), TC_CONV_WARPS);
    for (int side = 0; side < 2; side++)
      for (int a = 0; a < 2; a++) mbar_init(bars.acc_empty(side, a), TC_DRAIN_WARPS);
    for (int w = 0; w < DU_NW; w++) mbar_init(bars.wr_full(w), 1);
    for (int w = 0; w < 2; w++) mbar_init(bars.wc_full(w), 1);
    for (int d = 0; d < DU_ND; d++) mbar_init(bars.done(d), 4);  // the four issuers commit each stage
    mbar_init(bars.fin(), 4);
    mbar_init(bars.xch_full(), TC_DRAIN_WARPS / 2);
    mbar_init(bars.xch_empty(), TC_DRAIN_WARPS / 2);
    for (int w = 0; w < 2; w++) mbar_init(bars.wc_empty(w), 2);  // the two column-sum issuers commit
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + DS_TMEM),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (warp >= 2 && warp < 2 + TC_CONV_WARPS) {
    // constant operands of the 2^23 preload, as in fold_tc_kernel
    const int wi = tid - 64, nw = 32 * TC_CONV_WARPS;
    uint32_t* ac = reinterpret_cast<uint32_t*>(sm + DS_ACONST);
    for (int i = wi; i < 1024; i += nw) ac[i] = (i < 512 && (i & 3) == 0) ? 0x5C00u : 0u;
    uint32_t* bc = reinterpret_cast<uint32_t*>(sm + DS_BCONST);
    for (int i = wi; i < 256; i += nw) bc[i] = (i < 128 && (i & 31) < 4) ? 0x78007800u : 0u;
    fence_proxy_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + DS_TMEM);
  bool ok = true;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int last_use[DU_NR], last_wuse[DU_NW], last_cuse[2];
#pragma unroll
      for (int i = 0; i < DU_NR; i++) last_use[i] = -1;
#pragma unroll
      for (int i = 0; i < DU_NW; i++) last_wuse[i] = -1;
      last_cuse[0] = last_cuse[1] = -1;
      int s = 0, tcnt = 0;
      for (int tile = blockIdx.x; ok; tile += gridDim.x, tcnt++) {
        const bool done = tile >= ntiles;
        DualTile T{};
        if (!done) T = tiles[tile];
        const int nst = done ? 1 : T.nk / TC_KS;
        if (!done) {
          // the strip's column-sum weights into slot tcnt & 1, once the
          // stages of the tile that used it before have completed
          const int cs = tcnt & 1, cuse = tcnt >> 1;
          if (cuse > 0 && !tc_wait(bars.wc_empty(cs), (cuse - 1) & 1, wait_ns)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(bars.wc_full(cs), 8192);
          bulk_g2s(base + DS_WC + cs * 8192, reinterpret_cast<const uint8_t*>(T.w8C) + (size_t)(T.w0 / TC_KP) * 4096,
                   8192, bars.wc_full(cs));
          last_cuse[cs] = cuse;
        }
        for (int st = 0; st < nst; st++, s++) {
          const int slot = s % DU_NR, use = s / DU_NR, ws = s % DU_NW, wuse = s / DU_NW;
          if (use > 0 && !tc_wait(bars.raw_empty(slot), (use - 1) & 1, wait_ns)) {
            ok = false;
            break;
          }
          DualHdr H{};
          H.tile = done ? -1 : tile;
          H.stage = st;
          H.nst = nst;
          H.tcnt = tcnt;
          H.accR = T.accR;
          H.fR = T.fR;
          H.corrR = T.corrR;
          H.accC = done ? nullptr : T.accC + (size_t)(T.k0 + st * TC_KS) * 8;
          hdr[s % DU_HR] = H;
          last_use[slot] = use;
          const uint32_t raw = base + DS_RAW + slot * 32768;
          if (done) {
            mbar_arrive(bars.raw_full(slot));
            continue;
          }
          // the block first (HBM latency, DU_NR stages of lookahead), then the
          // stage's weights once their slot is free
          const int kk = T.k0 + st * TC_KS;
          mbar_arrive_expect_tx(bars.raw_full(slot), 32768);
          tma_load_2d(raw, T.tmap, kk, T.w0, bars.raw_full(slot));
          tma_load_2d(raw + 16384, T.tmap, kk + TC_KP, T.w0, bars.raw_full(slot));
          if (wuse > 0 && !tc_wait(bars.done(s - DU_NW), du_parity(s - DU_NW), wait_ns)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(bars.wr_full(ws), 8192);
          bulk_g2s(base + DS_WR + ws * 8192, reinterpret_cast<const uint8_t*>(T.w8R) + (size_t)(kk / TC_KP) * 4096,
                   8192, bars.wr_full(ws));
          last_wuse[ws] = wuse;
        }
        if (done) break;
      }
      if (!ok) du_mark_timeout(proofs, tiles, -1);
      for (int i = 0; i < DU_NR; i++)
        if (last_use[i] >= 0) tc_wait(bars.raw_full(i), last_use[i] & 1, wait_ns);
      for (int i = 0; i < DU_NW; i++)
        if (last_wuse[i] >= 0) tc_wait(bars.wr_full(i), last_wuse[i] & 1, wait_ns);
      for (int i = 0; i < 2; i++)
        if (last_cuse[i] >= 0) tc_wait(bars.wc_full(i), last_cuse[i] & 1, wait_ns);
    }
  } else if (warp == 1 || warp >= DU_THREADS / 32 - 3) {
    // ---------------------------------------------------------------- MMA issuers
    if (lane == 0) {
      const int j = warp == 1 ? 0 : warp - (DU_THREADS / 32 - 3) + 1;  // 0..3
      const int side = j >> 1;                  // 0 row dots, 1 column sums
      const uint32_t half = (j & 1) ? 32 : 0;   // lo or hi
      const uint32_t plane = base + DS_CONV + ((j & 1) ? 32768u : 0u);
      for (int s = 0;; s++) {
        const int a = s & 1;
        if (!tc_wait(bars.conv_full(), (uint32_t)s & 1, wait_ns)) {
          ok = false;
          break;
        }
        const DualHdr h = hdr[s % DU_HR];
        if (h.tile < 0) {
          umma_commit(bars.done(s));  // end marker
          break;
        }
        if (s >= 2 && !tc_wait(bars.acc_empty(side, a), ((s >> 1) - 1) & 1, wait_ns)) {
          ok = false;
          du_mark_timeout(proofs, tiles, h.tile);
          break;
        }
        uint32_t wts;
        bool wok;
        if (side == 0) {
          wts = base + DS_WR + (s % DU_NW) * 8192;
          wok = tc_wait(bars.wr_full(s % DU_NW), (uint32_t)(s / DU_NW) & 1, wait_ns);
        } else {
          wts = base + DS_WC + (h.tcnt & 1) * 8192;
          wok = tc_wait(bars.wc_full(h.tcnt & 1), (uint32_t)(h.tcnt >> 1) & 1, wait_ns);
        }
        if (!wok) {
          ok = false;
          du_mark_timeout(proofs, tiles, h.tile);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + 128 * side + 64 * a + half;
        umma_ss(d, sdesc(base + DS_ACONST, 2048, 128), sdesc(base + DS_BCONST, 512, 128), IDESC, 0);  // := 2^23
#pragma unroll
        for (int ks = 0; ks < 8; ks++) {
          // K-major rows (row dots): cores 2ks, 2ks + 1 of the columns;
          // MN-major columns (column sums): cores 2ks, 2ks + 1 of the rows
          const uint64_t ad = side == 0 ? sdesc(plane + 2 * ks * 128, 128, 2048) : sdesc(plane + 2 * ks * 2048, 2048, 128);
          umma_ss(d, ad, sdesc(wts + ks * 1024, 512, 128), side == 0 ? IDESC : IDESC_MN_A, 1);
        }
        umma_commit(bars.done(s));
        if (side == 1 && h.stage == h.nst - 1) umma_commit(bars.wc_empty(h.tcnt & 1));
      }
      umma_commit(bars.fin());
      tc_wait(bars.fin(), 0, wait_ns);
    }
  } else if (warp < 2 + TC_CONV_WARPS) {
    // ---------------------------------------------------------------- converters
    // Thread = row m of the strip x half kh of the stage's 128 columns.
    const int quarter = warp & 3, kh = (warp - 2) >> 2;
    const int m = 32 * quarter + lane;
    uint8_t* lo_plane = sm + DS_CONV;
    uint8_t* hi_plane = sm + DS_CONV + 32768;
    const int rowoff = (m >> 3) * 16 * 128 + (m & 7) * 16;
    for (int s = 0;; s++) {
      const int slot = s % DU_NR;
      if (!warp_wait(bars.raw_full(slot), (s / DU_NR) & 1, wait_ns)) {
        ok = false;
        break;
      }
      const DualHdr h = hdr[s % DU_HR];
      // The planes are free once the previous stage's MMAs completed; the
      // wait also keeps conv_full from completing a phase before the issuers
      // have seen the previous one (the end marker included).
      if (s > 0 && !warp_wait(bars.done(s - 1), du_parity(s - 1), wait_ns)) {
        ok = false;
        du_mark_timeout(proofs, tiles, h.tile);
        break;
      }
      if (h.tile < 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bars.conv_full());  // the issuers see the end marker
        break;
      }
      const uint8_t* raw = sm + DS_RAW + slot * 32768;
#pragma unroll
      for (int j2 = 0; j2 < 2; j2++) {  // 32 columns at a time: c0 = 64 kh + 32 j2
        uint32_t w[16];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const uint4 v = *reinterpret_cast<const uint4*>(raw + 16384 * kh + m * 128 + (((4 * j2 + j) ^ (m & 7)) << 4));
          w[4 * j] = v.x; w[4 * j + 1] = v.y; w[4 * j + 2] = v.z; w[4 * j + 3] = v.w;
        }
        uint32_t lo[16], hi[16];
#pragma unroll
        for (int i = 0; i < 16; i++) {
          const uint32_t t = w[i] ^ 0x80008000u;  // p = x + 2^15
          lo[i] = bytes_f16x2(t, 0x4240);
          hi[i] = bytes_f16x2(t, 0x4341);
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {  // core columns 8 kh + 4 j2 + c: 8 columns, 16 bytes per plane
          const int off = rowoff + (8 * kh + 4 * j2 + c) * 128;
          *reinterpret_cast<uint4*>(lo_plane + off) = make_uint4(lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
          *reinterpret_cast<uint4*>(hi_plane + off) = make_uint4(hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
        }
      }
      fence_proxy_async_smem();  // the planes are read by the MMAs (async proxy)
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bars.conv_full());
        mbar_arrive(bars.raw_empty(slot));
      }
    }
  } else {
    // ---------------------------------------------------------------- drainers
    const int grp = (warp - 2 - TC_CONV_WARPS) >> 2, quarter = warp & 3;
    const int line = 32 * quarter + lane;
    const uint32_t tq = tmem + ((uint32_t)(32 * quarter) << 16);
    uint32_t dg[17];
#pragma unroll
    for (int t = 0; t < 17; t++) dg[t] = 0;
    int nx = 0;
    for (int s = 0;; s++) {
      const int a = s & 1;
      if (!warp_wait(bars.done(s), du_parity(s), wait_ns)) {
        ok = false;
        break;
      }
      const DualHdr& h = hdr[s % DU_HR];
      if (h.tile < 0) break;
      tc_fence_after();
      // row dots: digits run across the strip
      const uint32_t taR = tq + 64 * a, taC = tq + 128 + 64 * a;
      if (grp == 0) drain_pair<0, 15>(taR, dg);
      else drain_pair<16, 32>(taR, dg);
      release_acc(bars.acc_empty(0, a));
      // column sums of this stage's 128 columns over the strip's rows
      {
        uint32_t dc[17];
#pragma unroll
        for (int t = 0; t < 17; t++) dc[t] = 0;
        if (grp == 0) {
          drain_pair<0, 15>(taC, dc);
          release_acc(bars.acc_empty(1, a));
          tc_epilogue<0, 15, 1>(dc, 1, h.accC + (size_t)line * 8);
        } else {
          drain_pair<16, 32>(taC, dc);
          release_acc(bars.acc_empty(1, a));
          tc_epilogue<16, 32, 1>(dc, 1, h.accC + (size_t)line * 8);
        }
      }
      if (h.stage == h.nst - 1) {
        if (h.fR) {
          // whole row: group 1 hands its columns (4..7) to group 0, which
          // stores f = REDC(sum) - 2^15 . sum E (Montgomery)
          uint64_t* xch = reinterpret_cast<uint64_t*>(sm + DS_XCH) + line * 4;
          uint64_t col[8];
          if (grp == 1) {
            if (nx > 0 && !warp_wait(bars.xch_empty(), (nx - 1) & 1, wait_ns)) {
              ok = false;
              break;
            }
            digit_columns<16, 32, 1>(dg, h.nst, col);
#pragma unroll
            for (int j = 0; j < 4; j++) xch[j] = col[4 + j];
            __syncwarp();
            if (lane == 0) mbar_arrive(bars.xch_full());
          } else {
            if (!warp_wait(bars.xch_full(), nx & 1, wait_ns)) {
              ok = false;
              break;
            }
            digit_columns<0, 15, 1>(dg, h.nst, col);
            U64x8 acc;
#pragma unroll
            for (int j = 0; j < 8; j++) acc.v[j] = col[j] + (j >= 4 ? xch[j - 4] : 0ull);
            h.fR[line] = fr_sub(redc_columns_ni(acc), *h.corrR);
            __syncwarp();
            if (lane == 0) mbar_arrive(bars.xch_empty());
          }
          nx++;
        } else {
          unsigned long long* acc = h.accR + (size_t)line * 8;
          if (grp == 0) tc_epilogue<0, 15, 1>(dg, h.nst, acc);
          else tc_epilogue<16, 32, 1>(dg, h.nst, acc);
        }
#pragma unroll
        for (int t = 0; t < 17; t++) dg[t] = 0;
      }
    }
    if (!ok) du_mark_timeout(proofs, tiles, -1);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
  if (tid == 0) {
    for (int i = 0; i < DU_NBAR; i++) mbar_inval(bars.b + 8 * i);
  }
}

cudaError_t fold_dual_prepare() {
  static std::mutex mu;
  static bool done = false;
  std::lock_guard<std::mutex> lk(mu);
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fold_dual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DU_SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t launch_fold_dual(const DualTile* tiles, int ntiles, const DevProof* proofs, unsigned long long wait_ns,
                             cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  static std::atomic<int> sm_count{0};
  int sms = sm_count.load(std::memory_order_relaxed);
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    sm_count.store(sms, std::memory_order_relaxed);
  }
  const int grid = ntiles < sms ? ntiles : sms;
  fold_dual_kernel<<<grid, DU_THREADS, DU_SMEM, st>>>(tiles, ntiles, proofs, wait_ns);
  return cudaGetLastError();
}

cudaError_t fold_tc_prepare() {
  static std::mutex mu;  // plans are bound from several host threads
  static bool done = false;
  std::lock_guard<std::mutex> lk(mu);
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fold_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t launch_fold_tc(const TcTile* tiles, int ntiles, const DevProof* proofs, unsigned long long wait_ns,
                           cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  static std::atomic<int> sm_count{0};  // launches come from several host threads
  int sms = sm_count.load(std::memory_order_relaxed);
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    sm_count.store(sms, std::memory_order_relaxed);
  }
  const int grid = ntiles < sms ? ntiles : sms;
  fold_tc_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(tiles, ntiles, proofs, wait_ns);
  return cudaGetLastError();
}

}  // namespace vl
