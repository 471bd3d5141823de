// Chained proof of one LoRA projection (Sec. IV, putting everything together:
// sequential composition).  The claims the sumchecks leave on the
// intermediate tensors H and dH are not opened: through the rescale
// relations X.A + 2^7 = 2^8 H + rhoH and dY.B^T + 2^7 = 2^8 dH + rhodH
// (Sec. IV-A, quantisation with zeta = 2^8), each becomes a claim on X.A or
// dY.B^T at the same point, which a sumcheck of that product (Eq.
// eq:zk-mle-matmul with the point given) reduces to claims on the inputs.
//
// A batch of chains runs as
//   chain_start   one CTA per chain: transcript start, the stage-1 points
//                 (counter-mode squeeze, one thread per coordinate), the six
//                 stage-1 member start states
//   stage 1       one matmul plan over all chains' six members (prologue
//                 with the given points, tensor-core fold, rounds storing
//                 their challenges)
//   chain_eval    four CTAs per chain: the remainder MLEs at the points the
//                 stage-1 members end on
//   chain_link    one CTA per chain: bind the stage-1 proofs and the
//                 evaluations, the four stage-3 member starts and points
//   stage 3       one matmul plan over all chains' four members
//   chain_finish  one CTA per chain: final state, the proof record
// The transcript format is written out in include/verilora.h.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "abi_guard.h"
#include "common.cuh"
#include "fr_dev.cuh"
#include "reduce.cuh"
#include "transcript.cuh"

struct vl_plan;

namespace vl {
int plan_make(const vl_job* jobs, int32_t njobs, const vl_batch_opts* opts, vl_plan** out);
size_t plan_bytes(const vl_plan* p);
void plan_set_points(vl_plan* p, const std::vector<const GivenPoint*>& given, const std::vector<Fr*>& rch);
int plan_enqueue(vl_plan* p, uint8_t* ws, size_t bytes, vl_proof* dout, cudaStream_t st);
void set_last_error(const char* msg);
}  // namespace vl

extern "C" void vl_plan_destroy(vl_plan* plan);

namespace vl {
namespace {

constexpr int NS1 = 6, NS3 = 4;   // members of the two stages
constexpr int RCH = VL_MAX_ROUNDS;  // challenges kept per stage-1 member

// One chain on the device.
struct ChainDev {
  int32_t n, d, k, r;
  int32_t ln, ld, lk, lr;
  uint64_t seed;
  uint8_t binds[7][32];
  const int16_t* rho[2];    // rhoH, rhodH (n x r)
  int64_t rho_ld[2];
  GivenPoint* g1;           // stage-1 member starts and points
  GivenPoint* g3;           // stage-3
  Fr* rch;                  // NS1 x RCH stage-1 challenges (Montgomery)
  const vl_proof* out1;     // stage-1 proofs of this chain
  const vl_proof* out3;     // stage-3 proofs
  Fr e[4];                  // remainder evaluations (canonical)
  uint8_t S1[32], S3[32];
};

__device__ void member_start(uint8_t out[32], const uint8_t S[32], uint32_t p) {
  Sha256 h;
  h.init();
  h.update(S, 32);
  h.byte('M');
  h.u32le(p);
  h.finish(out);
}

// Transcript start, the stage-1 points, the stage-1 member starts.
__global__ void chain_start_kernel(ChainDev* chains) {
  ChainDev& C = chains[blockIdx.x];
  __shared__ uint8_t S0[32];
  const int tid = threadIdx.x;
  if (tid == 0) {
    const uint8_t dom[25] = {'v', 'e', 'r', 'i', 'l', 'o', 'r', 'a', '-', 'g', 'b', '3', '0',
                             '0', '/', 'z', 'k', 'c', 'h', 'a', 'i', 'n', '/', 'v', '1'};
    Sha256 h;
    h.init();
    h.update(dom, 25);
    h.u32le((uint32_t)C.seed);
    h.u32le((uint32_t)(C.seed >> 32));
    h.u32le((uint32_t)C.n);
    h.u32le((uint32_t)C.d);
    h.u32le((uint32_t)C.k);
    h.u32le((uint32_t)C.r);
    h.update(&C.binds[0][0], 7 * 32);
    h.finish(S0);
  }
  __syncthreads();
  // coordinates: u_Y, v_Y, u_dX, v_dX, u_dA, v_dA, u_dB, v_dB
  const int sz[8] = {C.ln, C.lk, C.ln, C.ld, C.ld, C.lr, C.lr, C.lk};
  int total = 0;
  for (int i = 0; i < 8; i++) total += sz[i];
  for (int t = tid; t < total; t += blockDim.x) {
    const Fr x = to_mont_ni(ts_challenge(S0, 'p', (uint32_t)t));
    int sl = 0, o = t;
    while (o >= sz[sl]) o -= sz[sl++];
    // slice -> members: the u or v of the members proved at that point
    switch (sl) {
      case 0: C.g1[0].u[o] = x; C.g1[1].u[o] = x; break;
      case 1: C.g1[0].v[o] = x; C.g1[1].v[o] = x; break;
      case 2: C.g1[2].u[o] = x; C.g1[3].u[o] = x; break;
      case 3: C.g1[2].v[o] = x; C.g1[3].v[o] = x; break;
      case 4: C.g1[4].u[o] = x; break;
      case 5: C.g1[4].v[o] = x; break;
      case 6: C.g1[5].u[o] = x; break;
      default: C.g1[5].v[o] = x; break;
    }
  }
  __syncthreads();
  if (tid == 0) {
    uint8_t S[32];
    memcpy(S, S0, 32);
    ts_squeeze_done(S, 'p', (uint32_t)total);
    memcpy(C.S1, S, 32);
    memcpy(S0, S, 32);
  }
  __syncthreads();
  if (tid < NS1) member_start(C.g1[tid].state, S0, (uint32_t)tid);
}

// Points of the four claims on H (p1, p2) and dH (q1, q2): x over the row
// bits (log n), y over the column bits (log r).
__device__ void claim_point(const ChainDev& C, int q, const Fr** x, const Fr** y) {
  switch (q) {
    case 0: *x = C.g1[1].u; *y = C.rch + 1 * RCH; break;  // p1 = (u_Y, r^1)
    case 1: *x = C.rch + 5 * RCH; *y = C.g1[5].u; break;  // p2 = (r^5, u_dB)
    case 2: *x = C.g1[3].u; *y = C.rch + 3 * RCH; break;  // q1 = (u_dX, r^3)
    default: *x = C.rch + 4 * RCH; *y = C.g1[4].v; break; // q2 = (r^4, v_dA)
  }
}

// eq(x, bits(i)) over `nv` variables, MSB first (Montgomery).
__device__ Fr eq_at(const Fr* x, int nv, int i) {
  Fr acc = fr_r1();
  for (int t = 0; t < nv; t++) acc = mont_mul_ni(acc, ((i >> (nv - 1 - t)) & 1) ? x[t] : fr_sub(fr_r1(), x[t]));
  return acc;
}

// rho~(x, y) = sum_{i < n, j < r} eq(x, i) rho[i, j] eq(y, j), one CTA per
// evaluation (blockIdx.y), canonical result.
__global__ void chain_eval_kernel(ChainDev* chains) {
  ChainDev& C = chains[blockIdx.x];
  const int q = blockIdx.y;
  __shared__ Fr ey[VL_CHAIN_MAX_RANK];
  __shared__ Fr red[32];
  const Fr *x, *y;
  claim_point(C, q, &x, &y);
  const int16_t* rho = C.rho[q >> 1];
  const int64_t ld = C.rho_ld[q >> 1];
  for (int j = threadIdx.x; j < C.r; j += blockDim.x) ey[j] = eq_at(y, C.lr, j);
  __syncthreads();
  Fr acc[1] = {fr_zero()};
  for (int i = threadIdx.x; i < C.n; i += blockDim.x) {
    Fr row = fr_zero();  // sum_j eq(y, j) rho[i, j]: Montgomery times plain = plain
    for (int j = 0; j < C.r; j++) row = fr_add(row, mont_mul_ni(ey[j], fr_from_i64(rho[(int64_t)i * ld + j])));
    acc[0] = fr_add(acc[0], mont_mul_ni(eq_at(x, C.ln, i), row));
  }
  block_sum_fr<1>(acc, red);
  if (threadIdx.x == 0) C.e[q] = acc[0];
}

// Bind the stage-1 proofs and the evaluations; the stage-3 starts and points.
__global__ void chain_link_kernel(ChainDev* chains) {
  ChainDev& C = chains[blockIdx.x];
  __shared__ uint8_t S3[32];
  const int tid = threadIdx.x;
  if (tid == 0) {
    uint8_t S[32];
    Sha256 h;
    h.init();
    h.update(C.S1, 32);
    h.byte('L');
    for (int p = 0; p < NS1; p++) h.update(C.out1[p].state, 32);
    h.finish(S);
    ts_absorb_fr(S, 'e', C.e, 4);
    memcpy(C.S3, S, 32);
    memcpy(S3, S, 32);
  }
  __syncthreads();
  if (tid < NS3) member_start(C.g3[tid].state, S3, (uint32_t)(NS1 + tid));
  // stage-3 points: (X.A at p1, p2; dY.B^T at q1, q2) = the claim points
  for (int q = 0; q < NS3; q++) {
    const Fr *x, *y;
    claim_point(C, q, &x, &y);
    for (int t = tid; t < C.ln + C.lr; t += blockDim.x) {
      if (t < C.ln) C.g3[q].u[t] = x[t];
      else C.g3[q].v[t - C.ln] = y[t - C.ln];
    }
  }
}

// Final state and the proof record (device).
__global__ void chain_finish_kernel(ChainDev* chains, vl_chain_proof* out) {
  ChainDev& C = chains[blockIdx.x];
  vl_chain_proof& P = out[blockIdx.x];
  const int tid = threadIdx.x;
  constexpr int W = sizeof(vl_proof) / 4;
  for (int i = tid; i < VL_CHAIN_MEMBERS * W; i += blockDim.x) {
    const int p = i / W, w = i % W;
    const vl_proof* src = p < NS1 ? C.out1 + p : C.out3 + (p - NS1);
    reinterpret_cast<uint32_t*>(&P.sub[p])[w] = reinterpret_cast<const uint32_t*>(src)[w];
  }
  if (tid == 0) {
    uint8_t S[32];
    Sha256 h;
    h.init();
    h.update(C.S3, 32);
    h.byte('Z');
    for (int p = 0; p < NS3; p++) h.update(C.out3[p].state, 32);
    h.finish(S);
    memcpy(P.state, S, 32);
    P.n = C.n; P.d = C.d; P.k = C.k; P.r = C.r;
    P.reserved = 0;
    int st = VL_OK;
    for (int p = 0; p < NS1 && st == VL_OK; p++) st = C.out1[p].status;
    for (int p = 0; p < NS3 && st == VL_OK; p++) st = C.out3[p].status;
    P.status = st;
    for (int q = 0; q < 4; q++)
      for (int l = 0; l < 8; l++) P.e[q].limb[l] = C.e[q].v[l];
  }
}

int ceil_log2(int64_t x) {
  int d = 0;
  while ((int64_t(1) << d) < x) d++;
  return d;
}

int check_i16(const vl_mat& M, int64_t rows, int64_t cols) {
  if (!M.data || M.space != VL_DEVICE || M.dtype != VL_I16 || M.trans != 0 || M.reserved != 0) return VL_EINVAL;
  if (M.rows != rows || M.cols != cols) return VL_ESHAPE;
  if (M.ld < M.cols) return VL_EINVAL;
  return VL_OK;
}

int check_job(const vl_chain_job& J) {
  const int64_t n = J.X.rows, d = J.X.cols, k = J.W.cols, r = J.A.cols;
  if (n < 1 || d < 1 || k < 1 || r < 1) return VL_ESHAPE;
  if (n > VL_MAX_REDUCE || d > VL_MAX_REDUCE || k > VL_MAX_REDUCE || r > VL_CHAIN_MAX_RANK) return VL_ESHAPE;
  int e;
  if ((e = check_i16(J.X, n, d)) || (e = check_i16(J.W, d, k)) || (e = check_i16(J.A, d, r)) ||
      (e = check_i16(J.B, r, k)) || (e = check_i16(J.dY, n, k)) || (e = check_i16(J.H, n, r)) ||
      (e = check_i16(J.dH, n, r)) || (e = check_i16(J.rhoH, n, r)) || (e = check_i16(J.rhodH, n, r)))
    return e;
  return VL_OK;
}

vl_mat tr(vl_mat M) {
  M.trans = 1;
  return M;
}

}  // namespace
}  // namespace vl

using namespace vl;

// A batch of chains: the two stage plans and the chain records.
struct ChainBatch {
  std::vector<vl_chain_job> jobs;
  vl_plan* s1 = nullptr;
  vl_plan* s3 = nullptr;
  size_t off_cd = 0, off_g1 = 0, off_g3 = 0, off_rch = 0, off_out1 = 0, off_out3 = 0, off_out = 0;
  size_t off_s1 = 0, off_s3 = 0, total = 0;
  ~ChainBatch() {
    if (s1) vl_plan_destroy(s1);
    if (s3) vl_plan_destroy(s3);
  }
};

namespace {

constexpr size_t CALIGN = 256;
size_t cal(size_t x) { return (x + CALIGN - 1) & ~(CALIGN - 1); }

int chain_build(ChainBatch* B, const vl_chain_job* jobs, int32_t njobs) {
  if (!jobs || njobs < 1) return VL_EINVAL;
  B->jobs.assign(jobs, jobs + njobs);
  for (const vl_chain_job& J : B->jobs) {
    const int e = check_job(J);
    if (e != VL_OK) return e;
  }
  std::vector<vl_job> j1, j3;
  for (const vl_chain_job& J : B->jobs) {
    vl_job t{};
    auto add = [&](std::vector<vl_job>& v, const vl_mat& P, const vl_mat& Q) {
      t.P = P;
      t.Q = Q;
      v.push_back(t);
    };
    add(j1, J.X, J.W);         // 0 X.W
    add(j1, J.H, J.B);         // 1 H.B
    add(j1, J.dY, tr(J.W));    // 2 dY.W^T
    add(j1, J.dH, tr(J.A));    // 3 dH.A^T
    add(j1, tr(J.X), J.dH);    // 4 X^T.dH
    add(j1, tr(J.H), J.dY);    // 5 H^T.dY
    add(j3, J.X, J.A);         // 6 X.A at p1
    add(j3, J.X, J.A);         // 7 X.A at p2
    add(j3, J.dY, tr(J.B));    // 8 dY.B^T at q1
    add(j3, J.dY, tr(J.B));    // 9 dY.B^T at q2
  }
  vl_batch_opts o{};
  o.persistent = 2;
  o.use_graph = 2;
  o.timing_runs = 1;
  int e = plan_make(j1.data(), (int32_t)j1.size(), &o, &B->s1);
  if (e == VL_OK) e = plan_make(j3.data(), (int32_t)j3.size(), &o, &B->s3);
  if (e != VL_OK) return e;
  const size_t nc = B->jobs.size();
  size_t off = 0;
  B->off_cd = off;
  off = cal(off + sizeof(ChainDev) * nc);
  B->off_g1 = off;
  off = cal(off + sizeof(GivenPoint) * NS1 * nc);
  B->off_g3 = off;
  off = cal(off + sizeof(GivenPoint) * NS3 * nc);
  B->off_rch = off;
  off = cal(off + sizeof(Fr) * RCH * NS1 * nc);
  B->off_out1 = off;
  off = cal(off + sizeof(vl_proof) * NS1 * nc);
  B->off_out3 = off;
  off = cal(off + sizeof(vl_proof) * NS3 * nc);
  B->off_out = off;
  off = cal(off + sizeof(vl_chain_proof) * nc);
  B->off_s1 = off;
  off = cal(off + plan_bytes(B->s1));
  B->off_s3 = off;
  off = cal(off + plan_bytes(B->s3));
  B->total = off;
  return VL_OK;
}

int cuda_err(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return VL_OK;
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", where, cudaGetErrorString(e));
  set_last_error(msg);
  return VL_ECUDA;
}

int chain_run(ChainBatch* B, uint8_t* ws, size_t bytes, vl_chain_proof* out, cudaStream_t st) {
  if (!ws || !out) return VL_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) & (CALIGN - 1)) return VL_EINVAL;
  if (bytes < B->total) return VL_ENOMEM;
  const int nc = (int)B->jobs.size();
  ChainDev* dcd = reinterpret_cast<ChainDev*>(ws + B->off_cd);
  GivenPoint* g1 = reinterpret_cast<GivenPoint*>(ws + B->off_g1);
  GivenPoint* g3 = reinterpret_cast<GivenPoint*>(ws + B->off_g3);
  Fr* rch = reinterpret_cast<Fr*>(ws + B->off_rch);
  vl_proof* out1 = reinterpret_cast<vl_proof*>(ws + B->off_out1);
  vl_proof* out3 = reinterpret_cast<vl_proof*>(ws + B->off_out3);
  vl_chain_proof* dout = reinterpret_cast<vl_chain_proof*>(ws + B->off_out);
  std::vector<ChainDev> cd(nc);
  std::vector<const GivenPoint*> giv1(NS1 * nc), giv3(NS3 * nc);
  std::vector<Fr*> r1(NS1 * nc), r3;
  for (int c = 0; c < nc; c++) {
    const vl_chain_job& J = B->jobs[c];
    ChainDev& C = cd[c];
    std::memset(&C, 0, sizeof(C));
    C.n = (int32_t)J.X.rows;
    C.d = (int32_t)J.X.cols;
    C.k = (int32_t)J.W.cols;
    C.r = (int32_t)J.A.cols;
    C.ln = ceil_log2(C.n);
    C.ld = ceil_log2(C.d);
    C.lk = ceil_log2(C.k);
    C.lr = ceil_log2(C.r);
    C.seed = J.seed;
    std::memcpy(C.binds, J.bind, sizeof(C.binds));
    C.rho[0] = static_cast<const int16_t*>(J.rhoH.data);
    C.rho[1] = static_cast<const int16_t*>(J.rhodH.data);
    C.rho_ld[0] = J.rhoH.ld;
    C.rho_ld[1] = J.rhodH.ld;
    C.g1 = g1 + NS1 * c;
    C.g3 = g3 + NS3 * c;
    C.rch = rch + (size_t)RCH * NS1 * c;
    C.out1 = out1 + NS1 * c;
    C.out3 = out3 + NS3 * c;
    for (int p = 0; p < NS1; p++) {
      giv1[NS1 * c + p] = C.g1 + p;
      r1[NS1 * c + p] = C.rch + (size_t)RCH * p;
    }
    for (int p = 0; p < NS3; p++) giv3[NS3 * c + p] = C.g3 + p;
  }
  plan_set_points(B->s1, giv1, r1);
  plan_set_points(B->s3, giv3, r3);
  cudaError_t ce = cudaMemcpyAsync(dcd, cd.data(), sizeof(ChainDev) * nc, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) {
    chain_start_kernel<<<nc, 128, 0, st>>>(dcd);
    ce = cudaGetLastError();
  }
  if (ce != cudaSuccess) return cuda_err(ce, "chain_start_kernel");
  int e = plan_enqueue(B->s1, ws + B->off_s1, plan_bytes(B->s1), out1, st);
  if (e != VL_OK) return e;
  chain_eval_kernel<<<dim3(nc, 4), 256, 0, st>>>(dcd);
  ce = cudaGetLastError();
  if (ce == cudaSuccess) {
    chain_link_kernel<<<nc, 64, 0, st>>>(dcd);
    ce = cudaGetLastError();
  }
  if (ce != cudaSuccess) return cuda_err(ce, "chain_link_kernel");
  e = plan_enqueue(B->s3, ws + B->off_s3, plan_bytes(B->s3), out3, st);
  if (e != VL_OK) return e;
  chain_finish_kernel<<<nc, 256, 0, st>>>(dcd, dout);
  ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, dout, sizeof(vl_chain_proof) * nc, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);  // the host copy of cd must outlive its upload too
  if (ce != cudaSuccess) return cuda_err(ce, "vl_prove_chain");
  for (int c = 0; c < nc; c++)
    if (out[c].status != VL_OK) return out[c].status;
  return VL_OK;
}

}  // namespace

extern "C" size_t vl_chain_workspace_bytes(const vl_chain_job* jobs, int32_t njobs) {
  VL_ABI_TRY
  std::unique_ptr<ChainBatch> B(new ChainBatch);
  return chain_build(B.get(), jobs, njobs) == VL_OK ? B->total : 0;
  VL_ABI_CATCH(0)
}

extern "C" int32_t vl_prove_chain(const vl_chain_job* jobs, int32_t njobs, void* workspace, size_t workspace_bytes,
                                  vl_chain_proof* out, void* stream) {
  VL_ABI_TRY
  std::unique_ptr<ChainBatch> B(new ChainBatch);
  int e = chain_build(B.get(), jobs, njobs);
  if (e != VL_OK) return e;
  return chain_run(B.get(), static_cast<uint8_t*>(workspace), workspace_bytes, out, static_cast<cudaStream_t>(stream));
  VL_ABI_CATCH(VL_ENOMEM)
}

struct vl_chain_plan : ChainBatch {};

extern "C" int32_t vl_chain_plan_create(const vl_chain_job* jobs, int32_t njobs, vl_chain_plan** plan) {
  VL_ABI_TRY
  if (!plan) return VL_EINVAL;
  *plan = nullptr;
  std::unique_ptr<vl_chain_plan> P(new (std::nothrow) vl_chain_plan);
  if (!P) return VL_ENOMEM;
  const int e = chain_build(P.get(), jobs, njobs);
  if (e != VL_OK) return e;
  *plan = P.release();
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" size_t vl_chain_plan_workspace_bytes(const vl_chain_plan* plan) { return plan ? plan->total : 0; }

extern "C" int32_t vl_chain_plan_run(vl_chain_plan* plan, void* workspace, size_t workspace_bytes,
                                     vl_chain_proof* out, void* stream) {
  VL_ABI_TRY
  if (!plan) return VL_EINVAL;
  return chain_run(plan, static_cast<uint8_t*>(workspace), workspace_bytes, out, static_cast<cudaStream_t>(stream));
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" void vl_chain_plan_destroy(vl_chain_plan* plan) { delete plan; }
