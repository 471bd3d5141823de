// Autotuner: launch and tile options for a job list, chosen by timing.
//
// Coordinate descent from the caller's options: for each knob in turn (fold
// engine, tensor-core segment length, rounds kernel variant and threads, launch mode,
// CUDA-core tile shapes when CUDA-core tiles exist) every listed value is
// tried with the other knobs fixed, and the fastest kept.  A candidate is a
// real plan run on the caller's workspace and stream: one untimed run (bind,
// graph capture), then `runs` timed runs between CUDA events; its time is the
// median run.  Candidates needing more workspace than given are skipped.  The
// winner is cached per shape signature (dimensions, transposes, dtypes,
// memory spaces and TMA addressability of every job) for the process, so
// later calls with the same shapes return at once.  Proofs do not depend on
// any of these options.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "verilora.h"
#include "abi_guard.h"

namespace {

struct Entry {
  vl_batch_opts opts;
  float ms;
};

std::mutex g_mu;
std::map<std::string, Entry> g_cache;

std::string signature(const vl_job* jobs, int32_t njobs) {
  std::vector<std::string> parts;
  parts.reserve(njobs);
  char buf[160];
  for (int32_t i = 0; i < njobs; i++) {
    const vl_mat* M[2] = {&jobs[i].P, &jobs[i].Q};
    std::string s;
    for (const vl_mat* m : M) {
      const bool tma = (m->ld % 8 == 0) && (m->space == VL_HOST || (reinterpret_cast<uintptr_t>(m->data) & 15) == 0);
      snprintf(buf, sizeof(buf), "%lldx%lld/%lld:%d%d%d%d;", (long long)m->rows, (long long)m->cols,
               (long long)m->ld % 8, m->trans, m->dtype, m->space, tma ? 1 : 0);
      s += buf;
    }
    parts.push_back(s);
  }
  std::sort(parts.begin(), parts.end());
  std::string sig;
  for (const std::string& s : parts) sig += s;
  return sig;
}

constexpr size_t ALIGN = 256;

// Median time of `runs` plan runs (ms), or a negative value if the candidate
// cannot run (workspace too small, plan rejected, launch failure).
float time_candidate(const vl_job* jobs, int32_t njobs, const vl_batch_opts& o, uint8_t* ws, size_t ws_bytes,
                     cudaStream_t st, int runs, int32_t* err) {
  vl_plan* plan = nullptr;
  int32_t e = vl_plan_create(jobs, njobs, &o, &plan);
  if (e != VL_OK) return -1.0f;
  const size_t outb = (sizeof(vl_proof) * (size_t)njobs + ALIGN - 1) & ~(ALIGN - 1);
  const size_t need = vl_plan_workspace_bytes(plan);
  if (ws_bytes < outb || need > ws_bytes - outb) {
    vl_plan_destroy(plan);
    return -1.0f;
  }
  vl_proof* dout = reinterpret_cast<vl_proof*>(ws + ws_bytes - outb);
  std::vector<float> t;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) e = VL_ECUDA;
  if (e == VL_OK) e = vl_plan_run(plan, ws, ws_bytes - outb, dout, VL_DEVICE, st);  // bind, capture, warm
  for (int r = 0; r < runs && e == VL_OK; r++) {
    if (cudaEventRecord(a, st) != cudaSuccess) e = VL_ECUDA;
    if (e == VL_OK) e = vl_plan_run(plan, ws, ws_bytes - outb, dout, VL_DEVICE, st);
    if (e == VL_OK && cudaEventRecord(b, st) != cudaSuccess) e = VL_ECUDA;
    float ms = 0;
    if (e == VL_OK && (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
      e = VL_ECUDA;
    t.push_back(ms);
  }
  if (e == VL_OK && cudaStreamSynchronize(st) != cudaSuccess) e = VL_ECUDA;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  vl_plan_destroy(plan);
  if (e != VL_OK) {
    if (e == VL_ECUDA) *err = e;  // a CUDA failure ends the search
    return -1.0f;
  }
  std::sort(t.begin(), t.end());
  return t.empty() ? -1.0f : t[t.size() / 2];
}

}  // namespace

extern "C" int32_t vl_autotune(const vl_job* jobs, int32_t njobs, const vl_batch_opts* base, void* workspace,
                               size_t workspace_bytes, void* stream, int32_t runs, vl_batch_opts* best,
                               float* best_ms) {
  VL_ABI_TRY
  if (!jobs || njobs < 1 || !workspace || !best) return VL_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) & (ALIGN - 1)) return VL_EINVAL;
  const std::string sig = signature(jobs, njobs);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(sig);
    if (it != g_cache.end()) {
      *best = it->second.opts;
      if (best_ms) *best_ms = it->second.ms;
      return VL_OK;
    }
  }
  if (runs < 1) runs = 3;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  vl_batch_opts cur{};
  if (base) cur = *base;
  cur.timing_runs = std::max(cur.timing_runs, 1);
  int32_t err = VL_OK;
  float cur_ms = time_candidate(jobs, njobs, cur, ws, workspace_bytes, st, runs, &err);
  if (cur_ms < 0) return err != VL_OK ? err : VL_ENOMEM;

  struct Knob {
    int32_t vl_batch_opts::*field;
    std::vector<int32_t> values;
  };
  const std::vector<Knob> knobs = {
      {&vl_batch_opts::fold_engine, {0, 1}},
      {&vl_batch_opts::fold_dual, {0, 1}},
      {&vl_batch_opts::tc_seg, {0, 8192, 4096, 2048}},
      {&vl_batch_opts::rounds_variant, {7, 6, 5, 4, 3, 2, 8}},
      {&vl_batch_opts::rounds_threads, {0, 192, 256}},
      // The persistent single launch (persistent = 1) is not a candidate: it
      // runs the CUDA-core fold (its fold tiles are pulled from a work queue
      // by CTAs that also run prologues and rounds, which the tensor-core
      // fold's one-CTA-per-SM pipeline with all of TMEM cannot share), and
      // is about 3x slower than phase launches on the LoRA steps.  Callers
      // can still ask for it.
      {&vl_batch_opts::colsum_rows, {0, 128, 512}},
      {&vl_batch_opts::rowdot_cols, {0, 512, 2048}},
  };
  for (const Knob& k : knobs) {
    // Tensor-core segments only matter on that engine; CUDA-core tile shapes
    // only where CUDA-core tiles run.
    if (k.field == &vl_batch_opts::tc_seg && (cur.fold_engine == 1 || cur.persistent == 1)) continue;
    const bool cuda_core = cur.fold_engine == 1 || cur.persistent == 1;
    if ((k.field == &vl_batch_opts::colsum_rows || k.field == &vl_batch_opts::rowdot_cols) && !cuda_core) continue;
    for (int32_t v : k.values) {
      if (cur.*(k.field) == v) continue;
      vl_batch_opts cand = cur;
      cand.*(k.field) = v;
      const float ms = time_candidate(jobs, njobs, cand, ws, workspace_bytes, st, runs, &err);
      if (err != VL_OK) return err;
      if (ms >= 0 && ms < cur_ms * 0.99f) {
        cur = cand;
        cur_ms = ms;
      }
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[sig] = Entry{cur, cur_ms};
  }
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" void vl_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
}
