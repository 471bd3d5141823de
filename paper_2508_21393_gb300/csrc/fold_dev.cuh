// Fold kernels: the restrictions of the operand MLEs to the sumcheck cube,
//   f_A[w] = A~(u, w) = sum_i E_u[i] . op(P)[i, w]
//   f_B[w] = B~(w, v) = sum_j op(Q)[w, j] . E_v[j]
// (Eq. eq:zk-mle-matmul, Sec. II-C).  This reads every operand entry once and
// is the bulk of the prover's work.
//
// int16 operands (fixed point).  An entry x is the field element x mod r.
// With p = x + 2^15 in [0, 2^16) and weights e = E.R^2 (8 limbs of 32 bits),
//   sum_i e_i . p_i = sum_l 2^(32 l) . (sum_i e_i[l] . p_i)
// and each limb column sum is an exact unsigned 64-bit integer for up to 2^16
// terms ((2^32 - 1)(2^16 - 1) 2^16 < 2^64).  So one entry costs 8 32x32->64
// multiply-adds and no modular reduction; a tile adds its eight column sums
// per output into global 64-bit accumulators (integer adds are exact, so the
// order of tiles does not matter), and the rounds kernel reduces each
// output once: REDC(sum e.p) = (sum E.p).R is the Montgomery form, minus the
// offset correction 2^15 . sum E (written by the prologue).
//
// Feeding the multipliers: for int16 operands whose rows are 16-byte aligned,
// a CTA streams its tile through NSTAGE shared-memory stages filled by bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier per
// stage), so loads of later stages are in flight while earlier stages are
// multiplied.  Every wait is bounded (FOLD_WAIT_NS of the global timer by
// default); a CTA whose wait runs out marks its proof VL_ETIMEOUT, waits
// (again bounded) for its own copies still in flight, and returns.  Operands
// that are not aligned take a register-load path.
//
// Montgomery operands (32 bytes per entry): one Montgomery product per entry,
// mont_mul(E.R^2, x.R) = E.x.R^2, summed mod r per thread; partial sums are
// added limb-wise into the same 64-bit accumulators, whose REDC again gives
// the Montgomery form.
#pragma once
#include "common.cuh"
#include "reduce.cuh"

namespace vl {

typedef unsigned long long u64;

__device__ __forceinline__ uint2 ld_nc_u2(const void* p) {
  uint2 r;
  asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
  return r;
}

__device__ __forceinline__ uint4 ld_nc_u4(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}

__device__ __forceinline__ void red_add_u64(u64* p, u64 v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of an mbarrier, giving up at `deadline` (global ns).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t deadline) {
  while (!mbar_try_wait(bar, parity))
    if (global_ns() > deadline) return false;
  return true;
}

// The same with a budget of `wait_ns` from the first failed attempt: the
// global timer is only read when the phase is not complete at once.
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, uint64_t wait_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  return mbar_wait_bounded(bar, parity, global_ns() + wait_ns);
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completion counted on mbarrier `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// 2D TMA load of one box of the tensor map at (x = column, y = row) into
// shared memory, completion counted on mbarrier `bar`.  x must be a multiple
// of 8 (16 bytes of int16); out-of-range rows and columns read as zero.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Order earlier generic-proxy accesses to shared memory before later
// async-proxy (bulk copy) writes into it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint4 lds_u4(uint32_t addr) {
  uint4 r;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(addr));
  return r;
}

__device__ __forceinline__ uint2 lds_u2(uint32_t addr) {
  uint2 r;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(addr));
  return r;
}

// Offset int16 -> [0, 2^16).
__device__ __forceinline__ uint32_t off16(int16_t x) { return (uint32_t)(uint16_t)x ^ 0x8000u; }

// Four consecutive int16 entries starting at `p` (offset form); entries at
// column >= limit read as 2^15 (value zero).  `vec`: p is 8-byte aligned.
__device__ __forceinline__ void load4_i16(const int16_t* p, int avail, bool vec, uint32_t out[4]) {
  if (vec && avail >= 4) {
    uint2 q = ld_nc_u2(p);
    q.x ^= 0x80008000u;
    q.y ^= 0x80008000u;
    out[0] = q.x & 0xffffu;
    out[1] = q.x >> 16;
    out[2] = q.y & 0xffffu;
    out[3] = q.y >> 16;
  } else {
#pragma unroll
    for (int c = 0; c < 4; c++) out[c] = c < avail ? off16(p[c]) : 0x8000u;
  }
}

// ---------------------------------------------------------------- int16 ---

// COLSUM over stored rows [r0, r1) and columns [c0, c1) (c1 - c0 <= 1024).
// Thread layout: G column groups of 4 columns (G a power of two covering the
// tile) times 256 / G row lanes.  Weights E[r] are staged in shared memory and
// read as a broadcast.
static __device__ void colsum_i16(const FoldTask& T, const FoldTile& t, const Fr* __restrict__ E,
                           u64* __restrict__ acc, uint4* sm) {
  const int tid = threadIdx.x;
  const int nrows = t.r1 - t.r0;
  const uint4* Eg = reinterpret_cast<const uint4*>(E + t.r0);
  for (int i = tid; i < 2 * nrows; i += FOLD_THREADS) sm[i] = Eg[i];
  __syncthreads();

  const int ncols = t.c1 - t.c0;
  const int ngroups = (ncols + 3) >> 2;
  int G = 1;
  while (G < ngroups) G <<= 1;
  const int RL = FOLD_THREADS / G;
  const int grp = tid & (G - 1);
  const int lr = tid / G;
  if (grp >= ngroups) return;

  const int c = t.c0 + 4 * grp;
  const int avail = t.c1 - c;
  const int16_t* base = static_cast<const int16_t*>(T.mat) + c;
  const bool vec = ((reinterpret_cast<uintptr_t>(base) & 7) == 0) && ((T.ld & 3) == 0);

  u64 a[4][8];
#pragma unroll
  for (int q = 0; q < 4; q++)
#pragma unroll
    for (int l = 0; l < 8; l++) a[q][l] = 0;

#pragma unroll 2
  for (int r = lr; r < nrows; r += RL) {
    uint32_t p[4];
    load4_i16(base + (int64_t)(t.r0 + r) * T.ld, avail, vec, p);
    const uint4 e0 = sm[2 * r], e1 = sm[2 * r + 1];
    const uint32_t e[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
      for (int l = 0; l < 8; l++) a[q][l] += (u64)e[l] * p[q];
  }
#pragma unroll
  for (int q = 0; q < 4; q++) {
    if (q < avail) {
      u64* dst = acc + (size_t)(c + q) * 8;
#pragma unroll
      for (int l = 0; l < 8; l++) red_add_u64(dst + l, a[q][l]);
    }
  }
}

// ROWDOT over stored rows [r0, r1) (<= 32: 4 per warp) and columns [c0, c1).
// Lanes stride over columns, 4 per lane; the weights of the tile's columns are
// staged in shared memory limb-major (conflict-free 16-byte reads).  At the
// end a transpose-reduction leaves lane L with (row L / 8, limb L % 8).
static __device__ void rowdot_i16(const FoldTask& T, const FoldTile& t, const Fr* __restrict__ E,
                           u64* __restrict__ acc, uint32_t* sm) {
  const int tid = threadIdx.x;
  const int ncols = t.c1 - t.c0;
  const int pitch = (ncols + 3) & ~3;
  for (int j = tid; j < pitch; j += FOLD_THREADS) {
    Fr e = j < ncols ? E[t.c0 + j] : fr_zero();
#pragma unroll
    for (int l = 0; l < 8; l++) sm[l * pitch + j] = e.v[l];
  }
  __syncthreads();

  const int warp = tid >> 5, lane = tid & 31;
  const int rb = t.r0 + warp * ROWDOT_ROWS_PER_WARP;
  const int16_t* M = static_cast<const int16_t*>(T.mat);
  const bool vec = ((reinterpret_cast<uintptr_t>(M) & 7) == 0) && ((T.ld & 3) == 0) && ((t.c0 & 3) == 0);

  u64 a[32];
#pragma unroll
  for (int i = 0; i < 32; i++) a[i] = 0;

  for (int j = 4 * lane; j < ncols; j += 128) {
    uint32_t e[4][8];
#pragma unroll
    for (int l = 0; l < 8; l++) {
      const uint4 q = *reinterpret_cast<const uint4*>(sm + l * pitch + j);
      e[0][l] = q.x;
      e[1][l] = q.y;
      e[2][l] = q.z;
      e[3][l] = q.w;
    }
    const int avail = ncols - j;
#pragma unroll
    for (int rr = 0; rr < ROWDOT_ROWS_PER_WARP; rr++) {
      const int r = rb + rr;
      if (r < t.r1) {
        uint32_t p[4];
        load4_i16(M + (int64_t)r * T.ld + t.c0 + j, avail, vec, p);
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
          for (int l = 0; l < 8; l++) a[rr * 8 + l] += (u64)e[q][l] * p[q];
      }
    }
  }
  const u64 s = warp_transpose_sum(a);
  const int r = rb + (lane >> 3);
  if (r < t.r1) red_add_u64(acc + (size_t)r * 8 + (lane & 7), s);
}


// ------------------------------------------------- int16, bulk pipeline ---
//
// NSTAGE shared-memory slots.  Slot q has a "full" mbarrier (one arrival with
// the expected byte count; the bulk copies complete it) and an "empty"
// mbarrier (one arrival per warp once the warp has read the slot).  Warp 0
// also produces: before refilling a slot it waits until every warp has
// released it, so warps drift apart by up to NSTAGE stages and no block-wide
// barrier is needed per stage.  Every wait is bounded; the block votes once,
// after its last stage, and drains on failure.

static constexpr int FOLD_WARPS = FOLD_THREADS / 32;

struct Pipe {
  uint32_t full0;   // shared address of full barrier 0 (NSTAGE consecutive 8-byte barriers)
  uint32_t empty0;  // shared address of empty barrier 0
  uint32_t stage0;  // shared address of stage 0
};

__device__ __forceinline__ uint32_t pipe_full(const Pipe& p, int s) { return p.full0 + 8u * (uint32_t)(s % NSTAGE); }
__device__ __forceinline__ uint32_t pipe_empty(const Pipe& p, int s) { return p.empty0 + 8u * (uint32_t)(s % NSTAGE); }
__device__ __forceinline__ uint32_t pipe_slot(const Pipe& p, int s) {
  return p.stage0 + (uint32_t)(s % NSTAGE) * (uint32_t)SLOT_BYTES;
}
__device__ __forceinline__ uint32_t pipe_parity(int s) { return (uint32_t)(s / NSTAGE) & 1u; }

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ Pipe pipe_init(uint8_t* smem, uint32_t stage_offset) {
  Pipe p;
  p.full0 = smem_addr(smem);
  p.empty0 = p.full0 + 8u * NSTAGE;
  p.stage0 = smem_addr(smem + stage_offset);
  if (threadIdx.x == 0) {
    for (int q = 0; q < NSTAGE; q++) {
      mbar_init(p.full0 + 8u * q, 1);
      mbar_init(p.empty0 + 8u * q, FOLD_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  return p;
}

// Producer (warp 0, all lanes): before filling the slot of stage s >= NSTAGE,
// wait until every warp has released stage s - NSTAGE.
__device__ __forceinline__ bool pipe_acquire_slot(const Pipe& p, int s, uint64_t wait_ns) {
  if (s < NSTAGE) return true;
  return mbar_wait_for(pipe_empty(p, s), pipe_parity(s - NSTAGE), wait_ns);
}

// Consumer warp: done reading stage s.
__device__ __forceinline__ void pipe_release_slot(const Pipe& p, int s) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(pipe_empty(p, s));
}

// End of a tile: block-wide vote; on failure mark the proof and wait
// (bounded by FOLD_WAIT_NS, independent of the caller's limit) for the last
// copy issued into each slot, so none lands after the CTA moves on.  Then the
// barriers are invalidated so that the shared memory can serve other
// purposes (the persistent step reuses it for the next work item).
__device__ __forceinline__ bool pipe_finish(const Pipe& p, bool ok, int issued, int* status) {
  const bool all_ok = __syncthreads_and(ok);
  if (!all_ok && threadIdx.x == 0) {
    atomicExch(status, VL_ETIMEOUT);
    const uint64_t deadline = global_ns() + FOLD_WAIT_NS;
    for (int s = max(0, issued - NSTAGE); s < issued; s++) mbar_wait_bounded(pipe_full(p, s), pipe_parity(s), deadline);
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < 2 * NSTAGE; q++) mbar_inval(p.full0 + 8u * q);
  return all_ok;
}

// Stage s of a COLSUM tile: stored rows [r0 + s*BH, ...) of the tile's
// columns, as ceil(ncols / BW) boxes of BH x BW side by side in the slot,
// then the weights of the stage's rows (32 bytes each, one bulk copy).
__device__ __forceinline__ void colsum_issue(const Pipe& p, const FoldTask& T, const FoldTile& t, const Fr* E, int s) {
  if ((threadIdx.x & 31) != 0) return;
  const int ncols = t.c1 - t.c0, bw = T.box_w, bh = T.box_h;
  const int nsub = (ncols + bw - 1) / bw;
  const int erows = min(bh, t.r1 - t.r0 - s * bh);
  const uint32_t box_bytes = (uint32_t)bw * (uint32_t)bh * 2u;
  const uint32_t bar = pipe_full(p, s), slot = pipe_slot(p, s);
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, (uint32_t)nsub * box_bytes + 32u * (uint32_t)erows);
  for (int q = 0; q < nsub; q++) tma_load_2d(slot + (uint32_t)q * box_bytes, T.tmap, t.c0 + q * bw, t.r0 + s * bh, bar);
  bulk_g2s(slot + (uint32_t)nsub * box_bytes, E + t.r0 + s * bh, 32u * (uint32_t)erows, bar);
}

// Column sums, TMA path.  Thread layout: G groups of 8 columns (G a power of
// two covering the tile) x 2 limb halves x 128 / G row lanes.  A thread keeps
// 8 columns x 4 limbs of 64-bit sums; per row it reads its 4 weight limbs
// (16 bytes) and its 8 int16 entries (16 bytes) from shared memory and does
// 32 multiply-adds.  Splitting the limbs between two threads (rather than 4
// columns x 8 limbs per thread) measured markedly faster on GB300.
static __device__ void colsum_i16_bulk(const FoldTask& T, const FoldTile& t, const Fr* __restrict__ E,
                                       u64* __restrict__ acc, uint8_t* smem, int* status, uint64_t wait_ns) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nrows = t.r1 - t.r0, ncols = t.c1 - t.c0;
  const int bw = T.box_w, SR = T.box_h;
  const uint32_t box_bytes = (uint32_t)bw * (uint32_t)SR * 2u;
  const int nsub = (ncols + bw - 1) / bw;
  const uint32_t e_off = (uint32_t)nsub * box_bytes;  // weights follow the boxes in a slot
  const int nst = (nrows + SR - 1) / SR;
  const Pipe p = pipe_init(smem, FOLD_SMEM_HEAD);
  int issued = 0;
  bool ok = true;
  if (warp == 0) {
    issued = min(nst, NSTAGE - 1);
    for (int s = 0; s < issued; s++) colsum_issue(p, T, t, E, s);
  }

  const int ngroups = ncols >> 3;  // ncols is a multiple of 8 on this path
  int G = 1;
  while (G < ngroups) G <<= 1;
  const int RL = (FOLD_THREADS / 2) / G;
  const int h = tid & 1, grp = (tid >> 1) & (G - 1), lr = tid / (2 * G);
  const bool active = grp < ngroups;

  u64 a[8][4];
#pragma unroll
  for (int q = 0; q < 8; q++)
#pragma unroll
    for (int l = 0; l < 4; l++) a[q][l] = 0;

  for (int s = 0; s < nst; s++) {
    if (ok && warp == 0 && s + NSTAGE - 1 < nst) {
      const int sn = s + NSTAGE - 1;
      if (pipe_acquire_slot(p, sn, wait_ns)) {
        colsum_issue(p, T, t, E, sn);
        issued = sn + 1;
      } else {
        ok = false;
      }
    }
    const bool got = ok && mbar_wait_for(pipe_full(p, s), pipe_parity(s), wait_ns);
    ok = got;
    if (got && active) {
      const int rb = s * SR, rc = min(SR, nrows - rb);
      // this thread's 8 columns: box q = 8 grp / bw, column 8 grp - q bw within it
      const int q0 = (8 * grp) / bw;
      const uint32_t row_bytes = (uint32_t)bw * 2u;
      const uint32_t dstep = (uint32_t)RL * row_bytes, estep = 32u * (uint32_t)RL;
      uint32_t da = pipe_slot(p, s) + (uint32_t)q0 * box_bytes + 2u * (uint32_t)(8 * grp - q0 * bw) +
                    (uint32_t)lr * row_bytes;
      uint32_t ea = pipe_slot(p, s) + e_off + 32u * (uint32_t)lr + 16u * (uint32_t)h;
      int rr = lr;
      uint4 dn = make_uint4(0u, 0u, 0u, 0u), en = dn;
      if (rr < rc) {
        dn = lds_u4(da);
        en = lds_u4(ea);
      }
      for (; rr < rc; rr += RL) {
        uint4 d = dn;
        const uint4 ev = en;
        da += dstep;
        ea += estep;
        if (rr + RL < rc) {  // the next row's data and weights, one row ahead
          dn = lds_u4(da);
          en = lds_u4(ea);
        }
        d.x ^= 0x80008000u;
        d.y ^= 0x80008000u;
        d.z ^= 0x80008000u;
        d.w ^= 0x80008000u;
        const uint32_t pv[8] = {d.x & 0xffffu, d.x >> 16, d.y & 0xffffu, d.y >> 16,
                                d.z & 0xffffu, d.z >> 16, d.w & 0xffffu, d.w >> 16};
        const uint32_t e[4] = {ev.x, ev.y, ev.z, ev.w};
#pragma unroll
        for (int q = 0; q < 8; q++)
#pragma unroll
          for (int l = 0; l < 4; l++) a[q][l] += (u64)e[l] * pv[q];
      }
    }
    pipe_release_slot(p, s);
  }
  if (!pipe_finish(p, ok, warp == 0 ? issued : 0, status)) return;
  if (active) {
    const int c = t.c0 + 8 * grp;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      u64* dst = acc + (size_t)(c + q) * 8 + 4 * h;
#pragma unroll
      for (int l = 0; l < 4; l++) red_add_u64(dst + l, a[q][l]);
    }
  }
}

// Stage s of a ROWDOT tile: row block s / SPB (64 rows) x columns
// [c0 + (s % SPB) * BW, ...): one box of 64 x BW entries, then a box of the
// weights of those columns, 8 limb rows x BW words.
__device__ __forceinline__ void rowdot_issue(const Pipe& p, const FoldTask& T, const FoldTile& t, int s, int spb) {
  if ((threadIdx.x & 31) != 0) return;
  const int bw = T.box_w;
  const int x = t.c0 + (s % spb) * bw;
  const uint32_t bar = pipe_full(p, s), slot = pipe_slot(p, s);
  const uint32_t data_bytes = (uint32_t)ROWDOT_BLOCK_ROWS * (uint32_t)bw * 2u;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, data_bytes + 8u * (uint32_t)bw * 4u);
  tma_load_2d(slot, T.tmap, x, t.r0 + (s / spb) * ROWDOT_BLOCK_ROWS, bar);
  tma_load_2d(slot + data_bytes, T.etmap, x, 0, bar);  // [8 limbs x BW] of the weights
}

// Row dots, TMA path.  Lane L of a warp owns 8 consecutive columns of a
// stage (L / 2) and one limb half (L % 2); the warp owns 8 rows of the 64-row
// block.  Per stage a lane reads 8 columns x 4 limbs of weights (limb-major
// in shared memory), then per row its 8 int16 entries, 32 multiply-adds.
// At the end of a row block the 64-bit sums of the 16 lanes of each limb
// half are added with a 4-level transpose-reduction (offsets 16, 8, 4, 2):
// lane L ends with (row, limb) pairs v = (L & 30) | j, j < 2, v = row*4 + l.
static __device__ void rowdot_i16_bulk(const FoldTask& T, const FoldTile& t, const Fr* __restrict__ E,
                                       u64* __restrict__ acc, uint8_t* smem, int* status, uint64_t wait_ns) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncols = t.c1 - t.c0;
  const int bw = T.box_w;                 // columns per stage
  const int spb = (ncols + bw - 1) / bw;  // stages per row block
  const int nblk = (t.r1 - t.r0 + ROWDOT_BLOCK_ROWS - 1) / ROWDOT_BLOCK_ROWS;
  const int nst = spb * nblk;
  const uint32_t e_off = (uint32_t)ROWDOT_BLOCK_ROWS * (uint32_t)bw * 2u;  // weights follow the entries
  const Pipe p = pipe_init(smem, FOLD_SMEM_HEAD);
  int issued = 0;
  bool ok = true;
  if (warp == 0) {
    issued = min(nst, NSTAGE - 1);
    for (int s = 0; s < issued; s++) rowdot_issue(p, T, t, s, spb);
  }

  const int h = lane & 1, g = lane >> 1;
  const int wr = warp * BULK_ROWS_PER_WARP;  // first row of this warp within a block
  u64 a[BULK_ROWS_PER_WARP][4];
#pragma unroll
  for (int r = 0; r < BULK_ROWS_PER_WARP; r++)
#pragma unroll
    for (int l = 0; l < 4; l++) a[r][l] = 0;

  for (int s = 0; s < nst; s++) {
    if (ok && warp == 0 && s + NSTAGE - 1 < nst) {
      const int sn = s + NSTAGE - 1;
      if (pipe_acquire_slot(p, sn, wait_ns)) {
        rowdot_issue(p, T, t, sn, spb);
        issued = sn + 1;
      } else {
        ok = false;
      }
    }
    const int blk = s / spb, chunk = s - blk * spb;
    const int rb0 = t.r0 + blk * ROWDOT_BLOCK_ROWS;
    const int nrows = min(ROWDOT_BLOCK_ROWS, t.r1 - rb0);
    const bool got = ok && mbar_wait_for(pipe_full(p, s), pipe_parity(s), wait_ns);
    ok = got;
    const int j = chunk * bw + 8 * g;  // tile-local first column of this lane
    if (got && 8 * g < bw && j < ncols) {
      uint32_t e[8][4];
      const uint32_t eb = pipe_slot(p, s) + e_off + 32u * (uint32_t)g;
#pragma unroll
      for (int l = 0; l < 4; l++) {
        const uint4 q0 = lds_u4(eb + (uint32_t)(4 * h + l) * (uint32_t)bw * 4u);
        const uint4 q1 = lds_u4(eb + (uint32_t)(4 * h + l) * (uint32_t)bw * 4u + 16u);
        e[0][l] = q0.x; e[1][l] = q0.y; e[2][l] = q0.z; e[3][l] = q0.w;
        e[4][l] = q1.x; e[5][l] = q1.y; e[6][l] = q1.z; e[7][l] = q1.w;
      }
      const uint32_t slot = pipe_slot(p, s) + 16u * (uint32_t)g;
#pragma unroll
      for (int rr = 0; rr < BULK_ROWS_PER_WARP; rr++) {
        if (wr + rr < nrows) {
          uint4 d = lds_u4(slot + (uint32_t)(wr + rr) * (uint32_t)bw * 2u);
          d.x ^= 0x80008000u;
          d.y ^= 0x80008000u;
          d.z ^= 0x80008000u;
          d.w ^= 0x80008000u;
          const uint32_t pv[8] = {d.x & 0xffffu, d.x >> 16, d.y & 0xffffu, d.y >> 16,
                                  d.z & 0xffffu, d.z >> 16, d.w & 0xffffu, d.w >> 16};
#pragma unroll
          for (int q = 0; q < 8; q++)
#pragma unroll
            for (int l = 0; l < 4; l++) a[rr][l] += (u64)e[q][l] * pv[q];
        }
      }
    }
    pipe_release_slot(p, s);
    if (chunk == spb - 1) {
      // Row block done: reduce over the 16 lanes of each limb half.
      u64 v[32];
#pragma unroll
      for (int i = 0; i < 32; i++) v[i] = a[i >> 2][i & 3];
#pragma unroll
      for (int off = 16; off >= 2; off >>= 1) {
        const bool upper = (lane & off) != 0;
        const int half = off;  // values still held: 2 * off
#pragma unroll
        for (int i = 0; i < half; i++) {
          const u64 send = upper ? v[i] : v[i + half];
          const u64 keep = upper ? v[i + half] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
      }
      if (got) {
#pragma unroll
        for (int jj = 0; jj < 2; jj++) {
          const int vi = (lane & 30) | jj;
          const int row = rb0 + wr + (vi >> 2);
          if (row < rb0 + nrows) red_add_u64(acc + (size_t)row * 8 + 4 * h + (vi & 3), v[jj]);
        }
      }
#pragma unroll
      for (int r = 0; r < BULK_ROWS_PER_WARP; r++)
#pragma unroll
        for (int l = 0; l < 4; l++) a[r][l] = 0;
    }
  }
  pipe_finish(p, ok, warp == 0 ? issued : 0, status);
}

// ------------------------------------------------------------ Montgomery ---

__device__ __forceinline__ Fr load_fr(const Fr* p) {
  const uint4 a = ld_nc_u4(p), b = ld_nc_u4(reinterpret_cast<const uint4*>(p) + 1);
  Fr x;
  x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
  x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
  return x;
}

// COLSUM of a Montgomery matrix: one column per thread (c1 - c0 <= 256).
static __device__ void colsum_fr(const FoldTask& T, const FoldTile& t, const Fr* __restrict__ E,
                          u64* __restrict__ acc, uint4* sm) {
  const int tid = threadIdx.x;
  const int nrows = t.r1 - t.r0;
  const uint4* Eg = reinterpret_cast<const uint4*>(E + t.r0);
  for (int i = tid; i < 2 * nrows; i += FOLD_THREADS) sm[i] = Eg[i];
  __syncthreads();
  const int ncols = t.c1 - t.c0;
  int G = 1;
  while (G < ncols) G <<= 1;
  const int RL = FOLD_THREADS / G;
  const int col = tid & (G - 1), lr = tid / G;
  if (col >= ncols) return;
  const Fr* M = static_cast<const Fr*>(T.mat) + t.c0 + col;
  Fr s = fr_zero();
  for (int r = lr; r < nrows; r += RL) {
    const Fr x = load_fr(M + (int64_t)(t.r0 + r) * T.ld);
    const Fr* e = reinterpret_cast<const Fr*>(sm + 2 * r);
    s = fr_add(s, mont_mul(x, *e));
  }
  u64* dst = acc + (size_t)(t.c0 + col) * 8;
#pragma unroll
  for (int l = 0; l < 8; l++) red_add_u64(dst + l, s.v[l]);
}

// ROWDOT of a Montgomery matrix: 4 rows per warp, lanes over columns.
static __device__ void rowdot_fr(const FoldTask& T, const FoldTile& t, const Fr* __restrict__ E,
                          u64* __restrict__ acc, uint32_t* sm) {
  const int tid = threadIdx.x;
  const int ncols = t.c1 - t.c0;
  const int pitch = ncols;
  for (int j = tid; j < ncols; j += FOLD_THREADS) {
    Fr e = E[t.c0 + j];
#pragma unroll
    for (int l = 0; l < 8; l++) sm[l * pitch + j] = e.v[l];
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const int rb = t.r0 + warp * ROWDOT_ROWS_PER_WARP;
  const Fr* M = static_cast<const Fr*>(T.mat);
  Fr s[ROWDOT_ROWS_PER_WARP];
#pragma unroll
  for (int rr = 0; rr < ROWDOT_ROWS_PER_WARP; rr++) s[rr] = fr_zero();
  for (int j = lane; j < ncols; j += 32) {
    Fr e;
#pragma unroll
    for (int l = 0; l < 8; l++) e.v[l] = sm[l * pitch + j];
#pragma unroll
    for (int rr = 0; rr < ROWDOT_ROWS_PER_WARP; rr++) {
      const int r = rb + rr;
      if (r < t.r1) s[rr] = fr_add(s[rr], mont_mul(load_fr(M + (int64_t)r * T.ld + t.c0 + j), e));
    }
  }
  u64 a[32];
#pragma unroll
  for (int rr = 0; rr < ROWDOT_ROWS_PER_WARP; rr++)
#pragma unroll
    for (int l = 0; l < 8; l++) a[rr * 8 + l] = s[rr].v[l];
  const u64 tot = warp_transpose_sum(a);
  const int r = rb + (lane >> 3);
  if (r < t.r1) red_add_u64(acc + (size_t)r * 8 + (lane & 7), tot);
}

// One fold tile by the whole block (FOLD_THREADS threads).
__device__ __forceinline__ void fold_tile(const FoldTask& T, const FoldTile& t, const DevProof& P, uint8_t* smem,
                                          uint64_t wait_ns) {
  const Fr* E = T.side ? P.eqB : P.eqA;
  u64* acc = T.side ? P.accB : P.accA;
  uint4* sm4 = reinterpret_cast<uint4*>(smem + FOLD_SMEM_HEAD);
  if (T.dtype == VL_I16) {
    if (T.bulk) {
      if (T.mode == MODE_COLSUM) colsum_i16_bulk(T, t, E, acc, smem, &P.scr->status, wait_ns);
      else rowdot_i16_bulk(T, t, E, acc, smem, &P.scr->status, wait_ns);
    } else if (T.mode == MODE_COLSUM) {
      colsum_i16(T, t, E, acc, sm4);
    } else {
      for (int r0 = t.r0; r0 < t.r1; r0 += FB_BLOCK_ROWS) {  // 32-row blocks
        FoldTile b = t;
        b.r0 = r0;
        b.r1 = min(t.r1, r0 + FB_BLOCK_ROWS);
        rowdot_i16(T, b, E, acc, reinterpret_cast<uint32_t*>(sm4));
        __syncthreads();
      }
    }
  } else if (T.mode == MODE_COLSUM) {
    colsum_fr(T, t, E, acc, sm4);
  } else {
    for (int r0 = t.r0; r0 < t.r1; r0 += FB_BLOCK_ROWS) {
      FoldTile b = t;
      b.r0 = r0;
      b.r1 = min(t.r1, r0 + FB_BLOCK_ROWS);
      rowdot_fr(T, b, E, acc, reinterpret_cast<uint32_t*>(sm4));
      __syncthreads();
    }
  }
}

}  // namespace vl
