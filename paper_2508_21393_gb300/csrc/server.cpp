// Proving server: continuous batching of proving requests under a device
// memory budget.
//
// The paper proves one fine-tuning step at a time; a service receives
// requests (typically one projection's products) while others are on the
// GPU.  The server owns no device memory: the caller gives it an arena (the
// admission budget).  A worker thread
//   * completes finished batches (event query), copies their proofs to the
//     requests' outputs, records submit-to-completion latency, frees their
//     arena blocks;
//   * admits queued requests in arrival order into a new batch while a stream
//     slot is free: as many as fit the largest free arena block (plan
//     workspace + proof outputs) and the batch limit; a request that cannot
//     fit even an empty arena fails with VL_ENOMEM;
//   * runs each batch as one plan (phase launches, no graph: a batch runs
//     once) on its own stream, so batches overlap on the device.
// Operands may be resident device matrices (e.g. frozen weights kept on the
// device across requests) or host matrices, which the plan stages into its
// workspace (pinned host memory keeps those copies asynchronous).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "verilora.h"
#include "abi_guard.h"

namespace {

constexpr size_t ARENA_ALIGN = 256;

size_t round_up(size_t x) { return (x + ARENA_ALIGN - 1) & ~(ARENA_ALIGN - 1); }

// First-fit allocator over the caller's arena, with coalescing frees.
class Arena {
 public:
  void reset(uint8_t* base, size_t bytes) {
    base_ = base;
    free_.clear();
    const size_t skew = round_up(reinterpret_cast<uintptr_t>(base)) - reinterpret_cast<uintptr_t>(base);
    if (bytes > skew) free_[skew] = (bytes - skew) & ~(ARENA_ALIGN - 1);
  }
  size_t largest() const {
    size_t m = 0;
    for (const auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
  size_t total_free() const {
    size_t t = 0;
    for (const auto& kv : free_) t += kv.second;
    return t;
  }
  uint8_t* alloc(size_t bytes) {
    bytes = round_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      return base_ + off;
    }
    return nullptr;
  }
  void release(uint8_t* p, size_t bytes) {
    bytes = round_up(bytes);
    size_t off = p - base_;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }

 private:
  uint8_t* base_ = nullptr;
  std::map<size_t, size_t> free_;  // offset -> bytes
};

struct Request {
  uint64_t ticket;
  std::vector<vl_job> jobs;
  vl_proof* out;
  std::chrono::steady_clock::time_point submitted;
};

struct Batch {
  std::vector<Request> reqs;
  vl_plan* plan = nullptr;
  uint8_t* block = nullptr;
  size_t block_bytes = 0;
  vl_proof* dout = nullptr;   // device proofs (inside the block)
  vl_proof* hout = nullptr;   // pinned staging
  size_t nproofs = 0;
  int stream = -1;
  cudaEvent_t start = nullptr;  // recorded before the batch's work on its stream
  cudaEvent_t done = nullptr;   // after its proofs reach the host
  int id = 0;
};

}  // namespace

struct vl_server {
  vl_server_opts opts{};
  int device = 0;
  Arena arena;
  std::vector<cudaStream_t> streams;
  std::vector<bool> stream_busy;
  std::mutex mu;  // queue, done list, stats
  std::condition_variable cv;
  std::deque<Request> queue;
  std::vector<vl_server_done> done;
  std::vector<Batch*> inflight;
  std::vector<std::pair<vl_proof*, size_t>> pinned;  // free pinned staging buffers
  vl_server_stats stats{};
  uint64_t next_ticket = 1;
  int next_batch = 0;
  cudaEvent_t base = nullptr;  // device clock origin of the batches' intervals
  std::atomic<bool> stop{false};
  std::thread worker;
  int32_t fatal = VL_OK;
};

namespace {

vl_proof* take_pinned(vl_server* s, size_t n) {
  for (size_t i = 0; i < s->pinned.size(); i++)
    if (s->pinned[i].second >= n) {
      vl_proof* p = s->pinned[i].first;
      s->pinned.erase(s->pinned.begin() + i);
      return p;
    }
  void* p = nullptr;
  if (cudaHostAlloc(&p, sizeof(vl_proof) * n, cudaHostAllocDefault) != cudaSuccess) return nullptr;
  return static_cast<vl_proof*>(p);
}

void give_pinned(vl_server* s, vl_proof* p, size_t n) { s->pinned.emplace_back(p, n); }

void finish_batch(vl_server* s, Batch* b, int32_t status) {
  const auto now = std::chrono::steady_clock::now();
  float t0 = 0.f, t1 = 0.f;
  if (status == VL_OK && b->start && b->done) {
    if (cudaEventElapsedTime(&t0, s->base, b->start) != cudaSuccess ||
        cudaEventElapsedTime(&t1, s->base, b->done) != cudaSuccess)
      t0 = t1 = 0.f;
  }
  size_t k = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  for (Request& r : b->reqs) {
    int32_t st = status;
    if (st == VL_OK) {
      std::memcpy(r.out, b->hout + k, sizeof(vl_proof) * r.jobs.size());
      for (size_t i = 0; i < r.jobs.size(); i++)
        if (r.out[i].status != VL_OK && st == VL_OK) st = r.out[i].status;
    }
    k += r.jobs.size();
    vl_server_done d{};
    d.ticket = r.ticket;
    d.status = st;
    d.batch = b->id;
    d.latency_ms = std::chrono::duration<double, std::milli>(now - r.submitted).count();
    d.dev_start_ms = t0;
    d.dev_end_ms = t1;
    s->done.push_back(d);
    s->stats.completed++;
    s->stats.proofs += (int64_t)r.jobs.size();
  }
  s->stats.batches++;
}

void release_batch(vl_server* s, Batch* b) {
  if (b->plan) vl_plan_destroy(b->plan);
  if (b->block) s->arena.release(b->block, b->block_bytes);
  if (b->hout) give_pinned(s, b->hout, b->nproofs);
  if (b->done) cudaEventDestroy(b->done);
  if (b->start) cudaEventDestroy(b->start);
  if (b->stream >= 0) s->stream_busy[b->stream] = false;
  delete b;
}

// Plan for the first `n` queued requests; on success *plan and *bytes are set.
int32_t plan_for(vl_server* s, const std::vector<Request>& reqs, size_t n, vl_plan** plan, size_t* bytes) {
  std::vector<vl_job> jobs;
  for (size_t i = 0; i < n; i++) jobs.insert(jobs.end(), reqs[i].jobs.begin(), reqs[i].jobs.end());
  vl_batch_opts o{};
  o.persistent = 2;
  o.use_graph = 2;
  o.timing_runs = 1;
  o.groups = 1;
  o.wait_limit_us = s->opts.wait_limit_us;
  int32_t e = vl_plan_create(jobs.data(), (int32_t)jobs.size(), &o, plan);
  if (e != VL_OK) return e;
  *bytes = round_up(vl_plan_workspace_bytes(*plan)) + round_up(sizeof(vl_proof) * jobs.size());
  return VL_OK;
}

// Admit queued requests into one batch if a stream is free (worker thread).
bool admit(vl_server* s) {
  int stream = -1;
  for (size_t i = 0; i < s->streams.size(); i++)
    if (!s->stream_busy[i]) {
      stream = (int)i;
      break;
    }
  if (stream < 0) return false;
  std::vector<Request> cand;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t maxn = (size_t)std::max(1, s->opts.max_batch_requests);
    for (size_t i = 0; i < s->queue.size() && i < maxn; i++) cand.push_back(s->queue[i]);
  }
  if (cand.empty()) return false;
  const size_t avail = s->arena.largest();
  size_t n = cand.size();
  vl_plan* plan = nullptr;
  size_t bytes = 0;
  for (;;) {
    int32_t e = plan_for(s, cand, n, &plan, &bytes);
    if (e != VL_OK) {
      // A request the library rejects fails alone.
      if (n == 1) {
        std::lock_guard<std::mutex> lk(s->mu);
        vl_server_done d{};
        d.ticket = cand[0].ticket;
        d.status = e;
        d.batch = -1;
        s->done.push_back(d);
        s->stats.failed++;
        s->queue.pop_front();
        return true;
      }
      n = n / 2;
      continue;
    }
    if (bytes <= avail) break;
    vl_plan_destroy(plan);
    plan = nullptr;
    if (n == 1) {
      // Does not fit now; fails only if it could never fit.
      if (bytes > s->opts.arena_bytes) {
        std::lock_guard<std::mutex> lk(s->mu);
        vl_server_done d{};
        d.ticket = cand[0].ticket;
        d.status = VL_ENOMEM;
        d.batch = -1;
        s->done.push_back(d);
        s->stats.failed++;
        s->queue.pop_front();
        return true;
      }
      return false;  // wait for memory to free up
    }
    n = std::max<size_t>(1, n * avail / bytes);
    if (n >= cand.size()) n = cand.size() - 1;
  }
  Batch* b = new (std::nothrow) Batch();
  if (!b) {
    vl_plan_destroy(plan);
    return false;
  }
  b->plan = plan;
  b->block_bytes = bytes;
  b->block = s->arena.alloc(bytes);
  b->reqs.assign(cand.begin(), cand.begin() + n);
  for (const Request& r : b->reqs) b->nproofs += r.jobs.size();
  b->stream = stream;
  b->id = s->next_batch++;
  s->stream_busy[stream] = true;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < n; i++) s->queue.pop_front();
  }
  const size_t wsb = bytes - round_up(sizeof(vl_proof) * b->nproofs);
  b->dout = reinterpret_cast<vl_proof*>(b->block + wsb);
  b->hout = take_pinned(s, b->nproofs);
  cudaStream_t st = s->streams[stream];
  int32_t e = b->hout ? VL_OK : VL_ECUDA;
  if (e == VL_OK && (cudaEventCreate(&b->start) != cudaSuccess || cudaEventRecord(b->start, st) != cudaSuccess))
    e = VL_ECUDA;
  if (e == VL_OK) e = vl_plan_run(plan, b->block, wsb, b->dout, VL_DEVICE, st);
  if (e == VL_OK &&
      cudaMemcpyAsync(b->hout, b->dout, sizeof(vl_proof) * b->nproofs, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    e = VL_ECUDA;
  if (e == VL_OK && cudaEventCreate(&b->done) != cudaSuccess) e = VL_ECUDA;
  if (e == VL_OK && cudaEventRecord(b->done, st) != cudaSuccess) e = VL_ECUDA;
  if (e != VL_OK) {
    cudaStreamSynchronize(st);
    finish_batch(s, b, e);
    release_batch(s, b);
    return true;
  }
  s->inflight.push_back(b);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.launched++;
  }
  return true;
}

// Complete finished batches (worker thread).
bool reap(vl_server* s) {
  bool any = false;
  for (size_t i = 0; i < s->inflight.size();) {
    Batch* b = s->inflight[i];
    const cudaError_t q = cudaEventQuery(b->done);
    if (q == cudaErrorNotReady) {
      i++;
      continue;
    }
    finish_batch(s, b, q == cudaSuccess ? VL_OK : VL_ECUDA);
    release_batch(s, b);
    s->inflight.erase(s->inflight.begin() + i);
    any = true;
  }
  return any;
}

void worker_main(vl_server* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    bool progress = reap(s);
    while (admit(s)) progress = true;
    if (!progress) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 2000 : 20));
    }
  }
  // Drain: finish what is on the device.
  while (!s->inflight.empty()) {
    if (!reap(s)) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" int32_t vl_server_create(const vl_server_opts* opts, vl_server** out) {
  VL_ABI_TRY
  if (!opts || !out || !opts->arena || opts->arena_bytes < ARENA_ALIGN) return VL_EINVAL;
  for (int i = 0; i < 4; i++)
    if (opts->reserved[i]) return VL_EINVAL;
  vl_server* s = new (std::nothrow) vl_server();
  if (!s) return VL_ENOMEM;
  s->opts = *opts;
  if (s->opts.max_inflight <= 0) s->opts.max_inflight = 4;
  if (s->opts.max_batch_requests <= 0) s->opts.max_batch_requests = 64;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return VL_ECUDA;
  }
  s->arena.reset(static_cast<uint8_t*>(opts->arena), opts->arena_bytes);
  s->streams.resize(s->opts.max_inflight);
  s->stream_busy.assign(s->opts.max_inflight, false);
  for (cudaStream_t& st : s->streams)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams)
        if (x) cudaStreamDestroy(x);
      delete s;
      return VL_ECUDA;
    }
  if (cudaEventCreate(&s->base) != cudaSuccess || cudaEventRecord(s->base, s->streams[0]) != cudaSuccess ||
      cudaEventSynchronize(s->base) != cudaSuccess) {
    for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
    if (s->base) cudaEventDestroy(s->base);
    delete s;
    return VL_ECUDA;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" int32_t vl_server_submit(vl_server* s, const vl_job* jobs, int32_t njobs, vl_proof* out,
                                    uint64_t* ticket) {
  VL_ABI_TRY
  if (!s || !jobs || njobs < 1 || !out || !ticket) return VL_EINVAL;
  Request r;
  r.jobs.assign(jobs, jobs + njobs);
  r.out = out;
  r.submitted = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r.ticket = s->next_ticket++;
    *ticket = r.ticket;
    s->queue.push_back(std::move(r));
    s->stats.submitted++;
  }
  s->cv.notify_one();
  return VL_OK;
  VL_ABI_CATCH(VL_ENOMEM)
}

extern "C" int32_t vl_server_poll(vl_server* s, vl_server_done* done, int32_t max, int32_t* ndone) {
  if (!s || !ndone || max < 0 || (max > 0 && !done)) return VL_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  const int32_t n = std::min<int32_t>(max, (int32_t)s->done.size());
  for (int32_t i = 0; i < n; i++) done[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + n);
  *ndone = n;
  return VL_OK;
}

extern "C" int32_t vl_server_stats_get(vl_server* s, vl_server_stats* out) {
  if (!s || !out) return VL_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->queued = (int64_t)s->queue.size();
  return VL_OK;
}

extern "C" int32_t vl_server_destroy(vl_server* s) {
  if (!s) return VL_EINVAL;
  s->stop.store(true);
  s->cv.notify_one();
  if (s->worker.joinable()) s->worker.join();
  for (auto& pb : s->pinned) cudaFreeHost(pb.first);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  if (s->base) cudaEventDestroy(s->base);
  delete s;
  return VL_OK;
}
