// Tensor-core fold of int16 operands (tcgen05.mma with TMEM accumulators,
// TMA tensor copies, mbarrier pipelines).
//
// The fold f[w] = sum_i E_i . x[i, w] (Sec. II-C: A~(u, w) is the eq-weighted
// sum of column w; row dots likewise) is an integer matrix-vector product with
// 255-bit weights.  Write each weight as 32 bytes, E_i = sum_b 2^(8b) e[i, b],
// and each offset entry p = x + 2^15 (in [0, 2^16)) as two bytes,
// p = lo + 2^8 hi.  Then
//     D_lo[w, b] = sum_i lo[i, w] e[i, b],   D_hi[w, b] = sum_i hi[i, w] e[i, b]
// are two dense products (M = 128 lines w, N = 32 bytes b, K = the reduced
// index i), and
//     sum_i E_i p[i, w] = sum_{t=0}^{32} 2^(8t) s_t,  s_t = D_lo[w, t] + D_hi[w, t-1].
// All operands are integers in [0, 255] (exact in fp16); a product is at most
// 255^2, so one 64-entry stage sums to less than 2^22 and fp32 accumulation is
// exact.  The lo accumulator of each stage starts at 2^23 (one MMA of
// constants), so D_lo + D_hi = 2^23 + s_t lies in [2^23, 2^24) and its fp32 bit
// pattern is 0x4B000000 + s_t: workers add the bit patterns as 32-bit integers
// and remove the offsets once per tile.  At the end of a tile the 33 digit
// sums become the eight 64-bit column sums sum_j 2^(32j) col_j of the
// CUDA-core fold (col_7 also takes s_32 . 2^32), added with red.add, so the
// rounds reduce them unchanged (Montgomery reduction, minus 2^15 . sum E).
//
// Roles in a CTA (one CTA per SM; tiles come from a global counter, longest
// first), each running at its own pace and linked only by mbarriers:
//   warp 0       producer: per stage one 128B-swizzled TMA box of the operand
//                (two for column sums) and the stage's 4 KB of fp16 weight
//                bytes, into one of TC_NR raw slots
//   warp 1       owns TMEM; per stage one init MMA and 4 + 4 MMAs (K = 16)
//                into one of TC_NA accumulator buffers
//   warps 2-9    converters: int16 box -> fp16 lo/hi operand tiles in one of
//                TC_NC slots (canonical core-matrix layout, no swizzle;
//                K-major for row dots, MN-major for column sums)
//   warps 10-17  drainers: accumulator buffer -> per-line digit sums (two
//                groups of four warps, one warp per TMEM lane quarter, each
//                group half of the 33 digits); tile epilogue
// Stage headers (tile, stage) sit in a ring of TC_HR entries, longer than
// the stages any role can be ahead of another.
// Every wait is bounded; a wait that runs out marks the proof VL_ETIMEOUT, and
// the CTA drains its copies and MMAs before it frees TMEM and returns.
#include "fold_dev.cuh"

namespace vl {
namespace {

constexpr int SM_CONV = 0;                         // TC_NC x 32 KB: [lo 16 KB | hi 16 KB]
constexpr int SM_RAW = SM_CONV + TC_NC * 32768;    // TC_NR x 20 KB: [operand 16 KB | weights 4 KB]
constexpr int SM_ACONST = SM_RAW + TC_NR * 20480;  // 128 x 16 fp16, K-major
constexpr int SM_BCONST = SM_ACONST + 4096;        // 16 x 32 fp16, MN-major
constexpr int SM_HDR = SM_BCONST + 1024;           // TC_HR stage headers
constexpr int SM_BAR = SM_HDR + TC_HR * 16;
constexpr int NBAR = 2 * TC_NR + 2 * TC_NC + 2 * TC_NA + 1;
constexpr int SM_TMEM = SM_BAR + NBAR * 8;
static_assert(SM_TMEM + 16 <= TC_SMEM - 1024, "shared-memory layout");
constexpr uint32_t TMEM_COLS = 64 * TC_NA;  // TC_NA buffers of [lo 32 | hi 32] fp32 columns
static_assert(TMEM_COLS == 256, "TMEM allocation is a power of two");

// Instruction descriptor of kind::f16: fp32 accumulator, fp16 A and B,
// B MN-major, N = 32, M = 128; bit 15 selects an MN-major A.
constexpr uint32_t IDESC = (1u << 4) | (1u << 16) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle: core matrices of 8 x 16 bytes
// stored contiguously, `lbo` bytes apart along K and `sbo` bytes apart along
// M or N.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Arrive on `bar` once every MMA this thread issued so far has completed.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define TC_R8(b) "=r"(r[b + 0]), "=r"(r[b + 1]), "=r"(r[b + 2]), "=r"(r[b + 3]), "=r"(r[b + 4]), "=r"(r[b + 5]), \
                 "=r"(r[b + 6]), "=r"(r[b + 7])

// 8 columns into r[OFF .. OFF + 7].
template <int OFF>
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : TC_R8(OFF)
               : "r"(taddr));
}
#undef TC_R8
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Two fp16 values from bytes of t selected by `sel` (bytes 0x64 fill the
// high halves): 0x64bb is 1024 + bb exactly, minus 1024 leaves bb.
__device__ __forceinline__ uint32_t bytes_f16x2(uint32_t t, uint32_t sel) {
  const uint32_t v = __byte_perm(t, 0x64646464u, sel);
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(0x64006400u));
  return r;
}

// A bounded wait taken by a whole warp: it succeeds only if every lane's did,
// so the warp never splits before a .sync.aligned instruction.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, unsigned long long wait_ns) {
  return __all_sync(0xffffffffu, mbar_wait_for(bar, parity, wait_ns));
}

__device__ __forceinline__ uint32_t fbits_add(uint32_t a, uint32_t b) {
  return __float_as_uint(__fadd_rn(__uint_as_float(a), __uint_as_float(b)));
}

struct StageHdr {
  int32_t tile;   // -1: no more tiles
  int32_t stage;  // stage within the tile
  int32_t nst;    // stages of the tile
  int32_t mode;
};

struct TcBars {
  uint32_t b;
  __device__ uint32_t raw_full(int s) const { return b + 8 * s; }
  __device__ uint32_t raw_empty(int s) const { return b + 8 * (TC_NR + s); }
  __device__ uint32_t conv_full(int c) const { return b + 8 * (2 * TC_NR + c); }
  __device__ uint32_t conv_empty(int c) const { return b + 8 * (2 * TC_NR + TC_NC + c); }
  __device__ uint32_t acc_full(int a) const { return b + 8 * (2 * TC_NR + 2 * TC_NC + a); }
  __device__ uint32_t acc_empty(int a) const { return b + 8 * (2 * TC_NR + 2 * TC_NC + TC_NA + a); }
  __device__ uint32_t fin() const { return b + 8 * (2 * TC_NR + 2 * TC_NC + 2 * TC_NA); }
};

__device__ __forceinline__ void mark_timeout(const DevProof* proofs, const FoldTask* tasks, const TcTile* tiles,
                                             int tile) {
  atomicExch(&proofs[tasks[tiles[tile < 0 ? 0 : tile].task].proof].scr->status, VL_ETIMEOUT);
}

// Drain one stage's accumulator columns (lo at ta, hi at ta + 32) into the
// digit sums s_t, t in [T0, T1]:  dg[t - T0] += bits(2^23 + s_t), with
// s_t = lo_t + hi_{t-1} (the lo accumulator starts at 2^23).
template <int T0, int T1>
__device__ __forceinline__ void drain_digits(uint32_t ta, uint32_t (&dg)[17], uint32_t acc_empty) {
  constexpr int LA = T0, LB = T1 < 31 ? T1 : 31;           // lo columns used
  constexpr int HA = T0 > 0 ? T0 - 1 : 0, HB = T1 - 1;      // hi columns used
  uint32_t L[32], H[32];
  if (LA <= 7 && LB >= 0) tmem_ld8<0>(ta + 0, L);
  if (LA <= 15 && LB >= 8) tmem_ld8<8>(ta + 8, L);
  if (LA <= 23 && LB >= 16) tmem_ld8<16>(ta + 16, L);
  if (LA <= 31 && LB >= 24) tmem_ld8<24>(ta + 24, L);
  if (HA <= 7 && HB >= 0) tmem_ld8<0>(ta + 32, H);
  if (HA <= 15 && HB >= 8) tmem_ld8<8>(ta + 40, H);
  if (HA <= 23 && HB >= 16) tmem_ld8<16>(ta + 48, H);
  if (HA <= 31 && HB >= 24) tmem_ld8<24>(ta + 56, H);
  tmem_wait_ld();
  tc_fence_before();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(acc_empty);
#pragma unroll
  for (int t = T0; t <= T1; t++) {
    uint32_t v;
    if (t == 0) v = L[0];
    else if (t == 32) v = fbits_add(H[31], 0x4B000000u);
    else v = fbits_add(L[t], H[t - 1]);
    dg[t - T0] += v;
  }
}

// Combine a tile's digit sums s_t, t in [T0, T1], into the column sums
// col_j = sum_q 2^(8q) s_{4j+q} and add them to the proof's accumulators;
// s_32 goes to col_7 as s_32 . 2^32 (2^256 = 2^32 . 2^224).
template <int T0, int T1>
__device__ __forceinline__ void tc_epilogue(uint32_t (&dg)[17], int nst, unsigned long long* acc) {
  const uint32_t off = (uint32_t)nst * 0x4B000000u;
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
    fold_tc_kernel(const TcTile* __restrict__ tiles, int ntiles, const FoldTask* __restrict__ tasks,
                   const DevProof* __restrict__ proofs, int* counter, unsigned long long wait_ns) {
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
      mbar_init(bars.raw_empty(s), TC_CONV_WARPS + 1);  // converters + the MMA commit (weights)
    }
    for (int c = 0; c < TC_NC; c++) {
      mbar_init(bars.conv_full(c), TC_CONV_WARPS);
      mbar_init(bars.conv_empty(c), 1);
    }
    for (int a = 0; a < TC_NA; a++) {
      mbar_init(bars.acc_full(a), 1);
      mbar_init(bars.acc_empty(a), TC_DRAIN_WARPS);
    }
    mbar_init(bars.fin(), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + SM_TMEM),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (warp >= 2 && warp < 2 + TC_CONV_WARPS) {
    // Constant operands of the init MMA: A[m][0] = 256, B[0][n] = 32768, so
    // D = 2^23 everywhere; every other entry 0.
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
      int last_use[TC_NR];
#pragma unroll
      for (int i = 0; i < TC_NR; i++) last_use[i] = -1;
      int s = 0, tile = -1;
      for (bool done = false; !done && ok;) {
        tile = atomicAdd(counter, 1);
        done = tile >= ntiles;
        TcTile T{};
        FoldTask K{};
        const uint32_t* w8 = nullptr;
        if (!done) {
          T = tiles[tile];
          K = tasks[T.task];
          const DevProof& P = proofs[K.proof];
          w8 = K.side ? P.w8B : P.w8A;
        }
        const int nst = done ? 1 : (T.nk + TC_KS - 1) / TC_KS;
        for (int st = 0; st < nst; st++, s++) {
          const int slot = s % TC_NR, use = s / TC_NR;
          if (use > 0 && !mbar_wait_for(bars.raw_empty(slot), (use - 1) & 1, wait_ns)) {
            ok = false;
            break;
          }
          hdr[s % TC_HR] = StageHdr{done ? -1 : tile, st, nst, K.mode};
          last_use[slot] = use;
          const uint32_t raw = base + SM_RAW + slot * 20480;
          if (done) {
            mbar_arrive(bars.raw_full(slot));
            break;
          }
          const int kk = T.k0 + st * TC_KS;
          if (K.mode == MODE_ROWDOT) {
            mbar_arrive_expect_tx(bars.raw_full(slot), 16384 + 4096);
            tma_load_2d(raw, K.tmap, kk, T.w0, bars.raw_full(slot));
          } else {
            const bool two = T.nw > 64;
            mbar_arrive_expect_tx(bars.raw_full(slot), (two ? 16384 : 8192) + 4096);
            tma_load_2d(raw, K.tmap, T.w0, kk, bars.raw_full(slot));
            if (two) tma_load_2d(raw + 8192, K.tmap, T.w0 + 64, kk, bars.raw_full(slot));
          }
          bulk_g2s(raw + 16384, reinterpret_cast<const uint8_t*>(w8) + (size_t)(kk / TC_KS) * 4096, 4096,
                   bars.raw_full(slot));
        }
      }
      if (!ok) mark_timeout(proofs, tasks, tiles, tile < ntiles ? tile : -1);
      // Copies still in flight must land before the CTA leaves.
      for (int i = 0; i < TC_NR; i++)
        if (last_use[i] >= 0) mbar_wait_for(bars.raw_full(i), last_use[i] & 1, wait_ns);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      bool issued = false;
      for (int s = 0;; s++) {
        const int c = s % TC_NC, slot = s % TC_NR, a = s % TC_NA;
        if (!mbar_wait_for(bars.conv_full(c), (s / TC_NC) & 1, wait_ns)) {
          ok = false;
          break;
        }
        const StageHdr h = hdr[s % TC_HR];
        if (s >= TC_NA && !mbar_wait_for(bars.acc_empty(a), ((s / TC_NA) - 1) & 1, wait_ns)) {
          ok = false;
          mark_timeout(proofs, tasks, tiles, h.tile);
          break;
        }
        if (h.tile < 0) {
          umma_commit(bars.acc_full(a));  // tells the drainers: no more stages
          break;
        }
        tc_fence_after();
        const uint32_t idesc = IDESC | (h.mode == MODE_COLSUM ? (1u << 15) : 0u);
        const uint32_t conv = base + SM_CONV + c * 32768;
        const uint32_t wts = base + SM_RAW + slot * 20480 + 16384;
        const uint32_t dlo = tmem + 64 * a, dhi = dlo + 32;
        umma(dlo, sdesc(base + SM_ACONST, 2048, 128), sdesc(base + SM_BCONST, 512, 128), IDESC, 0);
#pragma unroll
        for (int ks = 0; ks < 4; ks++)
          umma(dlo, sdesc(conv + ks * 4096, 2048, 128), sdesc(wts + ks * 1024, 512, 128), idesc, 1);
#pragma unroll
        for (int ks = 0; ks < 4; ks++)
          umma(dhi, sdesc(conv + 16384 + ks * 4096, 2048, 128), sdesc(wts + ks * 1024, 512, 128), idesc, ks > 0);
        umma_commit(bars.conv_empty(c));
        umma_commit(bars.raw_empty(slot));
        umma_commit(bars.acc_full(a));
        issued = true;
      }
      if (issued) {
        umma_commit(bars.fin());
        mbar_wait_for(bars.fin(), 0, wait_ns);
      }
    }
  } else if (warp < 2 + TC_CONV_WARPS) {
    // ---------------------------------------------------------------- converters
    constexpr int NCT = 32 * TC_CONV_WARPS;
    const int wi = tid - 64;
    for (int s = 0;; s++) {
      const int slot = s % TC_NR, c = s % TC_NC;
      if (!warp_wait(bars.raw_full(slot), (s / TC_NR) & 1, wait_ns)) {
        ok = false;
        break;
      }
      const StageHdr h = hdr[s % TC_HR];
      if (s >= TC_NC && !warp_wait(bars.conv_empty(c), ((s / TC_NC) - 1) & 1, wait_ns)) {
        ok = false;
        mark_timeout(proofs, tasks, tiles, h.tile);
        break;
      }
      if (h.tile >= 0) {
        const uint8_t* raw = sm + SM_RAW + slot * 20480;
        uint8_t* lo = sm + SM_CONV + c * 32768;
#pragma unroll
        for (int it = 0; it < 1024 / NCT; it++) {
          const int q = it * NCT + wi, r8 = q & 7, rest = q >> 3;
          int src, dst;
          if (h.mode == MODE_ROWDOT) {
            const int kc = rest & 7, mg = rest >> 3, m = mg * 8 + r8;
            src = m * 128 + ((kc ^ r8) << 4);
            dst = kc * 2048 + mg * 128 + r8 * 16;
          } else {
            const int mc = rest & 15, kg = rest >> 4, k = kg * 8 + r8;
            src = (mc >> 3) * 8192 + k * 128 + (((mc & 7) ^ r8) << 4);
            dst = kg * 2048 + mc * 128 + r8 * 16;
          }
          const uint4 x = *reinterpret_cast<const uint4*>(raw + src);
          const uint32_t t0 = x.x ^ 0x80008000u, t1 = x.y ^ 0x80008000u, t2 = x.z ^ 0x80008000u,
                         t3 = x.w ^ 0x80008000u;
          *reinterpret_cast<uint4*>(lo + dst) = make_uint4(bytes_f16x2(t0, 0x4240), bytes_f16x2(t1, 0x4240),
                                                           bytes_f16x2(t2, 0x4240), bytes_f16x2(t3, 0x4240));
          *reinterpret_cast<uint4*>(lo + 16384 + dst) = make_uint4(
              bytes_f16x2(t0, 0x4341), bytes_f16x2(t1, 0x4341), bytes_f16x2(t2, 0x4341), bytes_f16x2(t3, 0x4341));
        }
        fence_proxy_async_smem();
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bars.conv_full(c));
        if (h.tile >= 0) mbar_arrive(bars.raw_empty(slot));
      }
      if (h.tile < 0) break;
    }
  } else {
    // ---------------------------------------------------------------- drainers
    const int grp = (warp - 2 - TC_CONV_WARPS) >> 2, quarter = warp & 3;
    const int line = 32 * quarter + lane;
    const uint32_t tq = tmem + ((uint32_t)(32 * quarter) << 16);
    uint32_t dg[17];
#pragma unroll
    for (int t = 0; t < 17; t++) dg[t] = 0;
    for (int s = 0;; s++) {
      const int a = s % TC_NA;
      if (!warp_wait(bars.acc_full(a), (s / TC_NA) & 1, wait_ns)) {
        ok = false;
        break;
      }
      const StageHdr h = hdr[s % TC_HR];
      if (h.tile < 0) break;
      tc_fence_after();
      const uint32_t ta = tq + 64 * a;
      if (grp == 0) drain_digits<0, 16>(ta, dg, bars.acc_empty(a));
      else drain_digits<17, 32>(ta, dg, bars.acc_empty(a));
      if (h.stage == h.nst - 1) {
        const TcTile T = tiles[h.tile];
        if (line < T.nw) {
          const FoldTask& K = tasks[T.task];
          const DevProof& P = proofs[K.proof];
          unsigned long long* acc = (K.side ? P.accB : P.accA) + (size_t)(T.w0 + line) * 8;
          if (grp == 0) tc_epilogue<0, 16>(dg, h.nst, acc);
          else tc_epilogue<17, 32>(dg, h.nst, acc);
        }
#pragma unroll
        for (int t = 0; t < 17; t++) dg[t] = 0;
      }
    }
    if (!ok) mark_timeout(proofs, tasks, tiles, -1);
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
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fold_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t launch_fold_tc(const TcTile* tiles, int ntiles, const FoldTask* tasks, const DevProof* proofs,
                           int* counter, unsigned long long wait_ns, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int grid = ntiles < sms ? ntiles : sms;
  fold_tc_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(tiles, ntiles, tasks, proofs, counter, wait_ns);
  return cudaGetLastError();
}

}  // namespace vl
