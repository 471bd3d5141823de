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
// 255^2, so over one 64-entry accumulation period D_lo + D_hi < 2^23 and fp32
// accumulation is exact.  The lo accumulator of each period starts at 2^23
// (one MMA of constants), which puts D_lo + D_hi in [2^23, 2^24), where the fp32 bit
// pattern is 0x4B000000 + s_t: the drainers add bit patterns as 32-bit
// integers and remove the offsets once per tile.  At the end of a tile the 33
// digit sums become the eight 64-bit column sums sum_j 2^(32j) col_j of the
// CUDA-core fold (col_7 also takes s_32 . 2^32), added with red.add, so the
// rounds reduce them unchanged (Montgomery reduction, minus 2^15 . sum E).
//
// Roles in a CTA (one CTA per SM; CTA b takes tiles b, b + grid, ... of a
// list sorted longest first), each running at its own pace and linked only by
// mbarriers:
// A pipeline stage is 128 lines x 128 entries: two accumulation periods.
//   warp 0       producer: per stage the operand (row dots: two boxes of 64
//                entries x 128 lines, 128B-swizzled; column sums: one box of
//                128 lines x 128 entries) into one of TC_NR shared-memory
//                slots, and the stage's 8 KB of fp16 weight bytes into one of TC_NW
//   warps 1, 18-20  MMA issuers (warp 1 also owns TMEM, 512 columns): a
//                pair per stage parity, in each pair one thread for the lo
//                and one for the hi products; per period 4 MMAs (K = 16) with
//                A read from TMEM and B (weights) from shared memory, into one
//                of TC_NA accumulator buffers (one thread issues an
//                MMA only every ~60-120 cycles; four keep the tensor core fed)
//   warps 2-9    converters: one thread per (line, half of the stage's 128
//                entries) reads its entries from the box, forms the
//                fp16 lo/hi operand rows and stores them to TMEM (one of
//                TC_NC operand buffers) with tcgen05.st
//   warps 10-17  drainers: accumulator buffer -> per-line digit sums (two
//                groups of four warps, one warp per TMEM lane quarter, each
//                group half of the 33 digits); tile epilogue
// TMEM columns: accumulator buffer a at 128a (period p at +64p: [lo 32 |
// hi 32]), operand buffer c at 256 + 128c ([lo 64 | hi 64], two fp16 per
// column).  Stage headers (tile,
// stage) sit in a ring of TC_HR entries, longer than the stages any role can
// be ahead of another.  Every wait is bounded; a wait that runs out marks the
// proof VL_ETIMEOUT, and the CTA drains its copies and MMAs before it frees
// TMEM and returns.
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
// Completion of stage s's MMAs (both issuers) is one barrier of a ring of
// TC_ND: the converters (TMEM operand reuse), the producer (weight slot
// reuse) and the drainers (accumulator ready) all wait on it.  TC_ND exceeds
// the lead any waiter can have, so no phase is lapped.
constexpr int TC_ND = 16;
// Issuer pairs take alternate stages: stages that share an operand, weight or
// accumulator barrier (TC_NC, TC_NW, TC_NA apart) must belong to one pair.
static_assert(TC_NC % 2 == 0 && TC_NW % 2 == 0 && TC_NA % 2 == 0, "ring sizes even");
static_assert(TC_ND > TC_NW && TC_ND > TC_NC && TC_ND >= TC_NA, "stage-done ring");
constexpr int NBAR = 2 * TC_NR + TC_NC + TC_NA + TC_NW + TC_ND + 3;
constexpr int SM_TMEM = SM_BAR + NBAR * 8;
static_assert(SM_TMEM + 16 <= TC_SMEM - 1024, "shared-memory layout");
constexpr uint32_t TMEM_COLS = 512;

constexpr uint32_t ACONV_COL = 128 * TC_NA;
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

// Bounded wait: gives up after wait_ns of %globaltimer (read only when the
// first attempt fails).
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, unsigned long long wait_ns) {
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

// Drain one stage's accumulator columns (lo at ta, hi at ta + 32) into the
// digit sums s_t, t in [T0, T1]:  dg[t - T0] += bits(2^23 + s_t), with
// s_t = lo_t + hi_{t-1}; the lo accumulator starts at 2^23 (init MMA), so
// one fp32 add gives 2^23 + s_t, exact below 2^24.
template <int T0, int T1>
__device__ __forceinline__ void drain_digits(uint32_t ta, uint32_t (&dg)[17], uint32_t acc_empty) {
  static_assert((T0 == 0 && T1 == 16) || (T0 == 17 && T1 == 32), "digit groups");
  uint32_t L[32], H[32];
  if (T0 == 0) {
    tmem_ld32(ta, L);            // lo 0..31 (0..16 used)
    tmem_ld16<0>(ta + 32, H);    // hi 0..15
  } else {
    tmem_ld16<16>(ta + 16, L);   // lo 16..31 (17..31 used)
    tmem_ld16<16>(ta + 48, H);   // hi 16..31
  }
  tmem_wait_ld();
  if (acc_empty) {  // last period of the stage: the buffer is free
    tc_fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(acc_empty);
  }
#pragma unroll
  for (int t = T0; t <= T1; t++) {
    uint32_t v;
    if (t == 0) v = L[0];
    else if (t == 32) v = fbits_add(H[31], 0x4B000000u);
    else v = fbits_add(L[t], H[t - 1]);
    dg[t - T0] += v;
  }
}

// Column sums col_j = sum_q 2^(8q) s_{4j+q} of the digits s_t, t in [T0, T1]
// (s_32 into col_7 as s_32 . 2^32); columns outside the range are 0.
template <int T0, int T1>
__device__ __forceinline__ void digit_columns(const uint32_t (&dg)[17], int nst, uint64_t (&col)[8]) {
  const uint32_t off = (uint32_t)(2 * nst) * 0x4B000000u;  // two drains per stage
#pragma unroll
  for (int j = 0; j < 8; j++) col[j] = 0;
#pragma unroll
  for (int t = T0; t <= T1; t++) {
    const int c = t < 32 ? t >> 2 : 7, sh = t < 32 ? 8 * (t & 3) : 32;
    col[c] += (uint64_t)(dg[t - T0] - off) << sh;
  }
}

// Combine a tile's digit sums s_t, t in [T0, T1], into the column sums
// col_j = sum_q 2^(8q) s_{4j+q} and add them to the proof's accumulators;
// s_32 goes to col_7 as s_32 . 2^32 (2^256 = 2^32 . 2^224).
template <int T0, int T1>
__device__ __forceinline__ void tc_epilogue(uint32_t (&dg)[17], int nst, unsigned long long* acc) {
  const uint32_t off = (uint32_t)(2 * nst) * 0x4B000000u;  // two drains per stage
#pragma unroll
  for (int j = 0; j < 8; j++) {
    uint64_t c = 0;
    bool any = false;
#pragma unroll
    for (int t = T0; t <= T1; t++) {
      const int col = t < 32 ? t >> 2 : 7, sh = t < 32 ? 8 * (t & 3) : 32;
      if (col == j) {
        c += (uint64_t)(dg[t - T0] - off) << sh;
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
    mbar_init(bars.fin(), 4);
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
    // the lo accumulator starts at 2^23; every other entry 0.
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
          if (done) {
            mbar_arrive(bars.raw_full(slot));
            continue;
          }
          if (wuse > 0 && !tc_wait(bars.done(s - TC_NW), done_parity(s - TC_NW), wait_ns)) {
            ok = false;
            break;
          }
          const int kk = T.k0 + st * TC_KS;
          mbar_arrive_expect_tx(bars.w_full(ws), 8192);
          bulk_g2s(base + SM_W + ws * 8192, reinterpret_cast<const uint8_t*>(T.w8) + (size_t)(kk / TC_KP) * 4096,
                   8192, bars.w_full(ws));
          last_wuse[ws] = wuse;
          mbar_arrive_expect_tx(bars.raw_full(slot), 32768);
          if (T.mode == MODE_ROWDOT) {
            tma_load_2d(raw, T.tmap, kk, T.w0, bars.raw_full(slot));
            tma_load_2d(raw + 16384, T.tmap, kk + TC_KP, T.w0, bars.raw_full(slot));
          } else {
            tma_load_2d(raw, T.tmap, T.w0, kk, bars.raw_full(slot));
          }
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
  } else if (warp == 1 || warp >= TC_THREADS / 32 - 3) {
    // ---------------------------------------------------------------- MMA issuers
    if (lane == 0) {
      const int j = warp == 1 ? 0 : warp - (TC_THREADS / 32 - 3) + 1;  // 0..3
      const uint32_t half = (j & 1) ? 32 : 0;  // lo or hi: A and D column offset
      for (int s = j >> 1;; s += 2) {
        const int c = s % TC_NC, a = s % TC_NA;
        if (!tc_wait(bars.conv_full(c), (s / TC_NC) & 1, wait_ns)) {
          ok = false;
          break;
        }
        const StageHdr h = hdr[s % TC_HR];
        if (s >= TC_NA && !tc_wait(bars.acc_empty(a), ((s / TC_NA) - 1) & 1, wait_ns)) {
          ok = false;
          mark_timeout(proofs, tiles, h.tile);
          break;
        }
        if (h.tile < 0) {
          umma_commit(bars.done(s));  // end marker: the drainers stop at the first one
          break;
        }
        const int ws = s % TC_NW;
        if (!tc_wait(bars.w_full(ws), (s / TC_NW) & 1, wait_ns)) {
          ok = false;
          mark_timeout(proofs, tiles, h.tile);
          break;
        }
        tc_fence_after();
        const uint32_t wts = base + SM_W + ws * 8192;
#pragma unroll
        for (int p = 0; p < 2; p++) {  // the stage's two accumulation periods
          const uint32_t d = tmem + 128 * a + 64 * p + half;
          const uint32_t av = tmem + ACONV_COL + 128 * c + 2 * half + 32 * p;  // lo at +0, hi at +64
          if (half == 0)  // lo accumulator := 2^23 (A, B constants in shared memory)
            umma_ss(d, sdesc(base + SM_ACONST, 2048, 128), sdesc(base + SM_BCONST, 512, 128), IDESC, 0);
#pragma unroll
          for (int ks = 0; ks < 4; ks++)
            umma_ts(d, av + 8 * ks, sdesc(wts + (4 * p + ks) * 1024, 512, 128), IDESC, half == 0 || ks > 0);
        }
        umma_commit(bars.done(s));
      }
      // every MMA this thread issued has completed before TMEM is freed
      umma_commit(bars.fin());
      tc_wait(bars.fin(), 0, wait_ns);
    }
  } else if (warp < 2 + TC_CONV_WARPS) {
    // ---------------------------------------------------------------- converters
    // Thread = line m (its TMEM lane) x half kh of the stage's 64 entries.
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
      const StageHdr h = hdr[s % TC_HR];
      if (s >= TC_NC && !warp_wait(bars.done(s - TC_NC), done_parity(s - TC_NC), wait_ns)) {
        ok = false;
        mark_timeout(proofs, tiles, h.tile);
        break;
      }
      if (h.tile >= 0) {
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
        if (h.tile >= 0) mbar_arrive(bars.raw_empty(slot));
      }
      if (h.tile < 0 && ++ends == 2) break;
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
      const StageHdr h = hdr[s % TC_HR];
      if (h.tile < 0) break;
      tc_fence_after();
      const uint32_t ta = tq + 128 * a;
      if (grp == 0) {
        drain_digits<0, 16>(ta, dg, 0);
        drain_digits<0, 16>(ta + 64, dg, bars.acc_empty(a));
      } else {
        drain_digits<17, 32>(ta, dg, 0);
        drain_digits<17, 32>(ta + 64, dg, bars.acc_empty(a));
      }
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
            digit_columns<17, 32>(dg, h.nst, col);
#pragma unroll
            for (int j = 0; j < 4; j++) xch[j] = col[4 + j];
            __syncwarp();
            if (lane == 0) mbar_arrive(bars.xch_full());
          } else {
            if (!warp_wait(bars.xch_full(), nx & 1, wait_ns)) {
              ok = false;
              break;
            }
            digit_columns<0, 16>(dg, h.nst, col);
            if (line < h.nw) {
              U64x8 a;
#pragma unroll
              for (int j = 0; j < 8; j++) a.v[j] = col[j] + (j >= 4 ? xch[j - 4] : 0ull);
              h.f[line] = fr_sub(redc_columns_ni(a), *h.corr);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bars.xch_empty());
          }
          nx++;
        } else if (line < h.nw) {
          unsigned long long* acc = h.acc + (size_t)line * 8;
          if (grp == 0) tc_epilogue<0, 16>(dg, h.nst, acc);
          else tc_epilogue<17, 32>(dg, h.nst, acc);
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
