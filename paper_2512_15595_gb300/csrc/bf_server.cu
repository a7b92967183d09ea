// Lookup serving runtime: many device-resident filters of one geometry, lookup
// requests (filter, host keys, host results) arriving over time, admitted
// into a device key arena while it has room, and batched across filters into
// one launch of the batched lookup kernel.  Host code only; the lookup itself
// is sbf_batch_kernel (same per-tile code as bf_contains).
//
// Worker loop (one thread per server):
//   admit    pending requests in arrival order while the arena (a ring of
//            keys, freed in completion order), the launch's request slots
//            and its share of the arena (a kMaxInflight-th; a larger request
//            goes alone) have room;
//   launch   copy the admitted requests' keys into the arena, write one
//            batch descriptor per request, one kernel over all of them, copy
//            every request's results back to its host buffer, record an event;
//   complete the oldest in-flight launch whose event has fired: stamp its
//            requests done, release their arena space.
// At most kMaxInflight launches are in flight.  Copies in, kernels and copies
// out run on three streams chained by events, so one batch's keys travel to
// the device while the previous batch's kernel runs; each stream is FIFO, so
// launches still complete in submission order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bloomgb.h"
#include "host_stage.h"
#include "key_ring.h"
#include "registry.h"

using namespace bloomgb;

namespace {

constexpr int kMaxInflight = 4;
using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

struct Request {
  uint64_t ticket = 0;
  uint32_t filter = 0;
  const uint64_t* h_keys = nullptr;
  uint64_t n = 0;
  uint8_t* h_out = nullptr;
  uint64_t arena_off = 0;  // first key slot in the arena
  double t_submit = 0, t_done = 0;
  bool done = false;
  bool addressable = false;  // the kernels can read h_keys and write h_out in place
};

struct Launch {
  std::vector<Request*> reqs;
  cudaEvent_t done = nullptr;     // results are on the host
  cudaEvent_t copied = nullptr;   // keys are on the device
  cudaEvent_t looked = nullptr;   // kernel finished
  // timing: start of each stage on its stream (the stage ends at copied,
  // looked and done)
  cudaEvent_t in0 = nullptr, look0 = nullptr, out0 = nullptr;
  BatchFilter* h_desc = nullptr;  // pinned
  uint64_t* h_begin = nullptr;    // pinned
  const uint64_t** h_src = nullptr;  // pinned: each request's host keys
  uint8_t** h_dst = nullptr;         // pinned: each request's host results
  BatchFilter* d_desc = nullptr;
  uint64_t* d_begin = nullptr;
  const uint64_t** d_src = nullptr;
  uint8_t** d_dst = nullptr;
  uint64_t arena_end = 0;         // ring position after this launch's keys
  uint64_t arena_used = 0;        // ring slots this launch consumed
  bool busy = false;
};

// uniform double in [0, 1) from a SplitMix64 state (load generator only)
double uniform01(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace

struct bf_server {
  bf_params p{};
  std::vector<BatchFilter> filters;  // words + nblocks; key fields set per launch
  int device = 0;
  cudaStream_t stream = nullptr;  // kernels
  cudaStream_t h2d = nullptr;     // copies in
  cudaStream_t d2h = nullptr;     // copies out
  const KernelEntry* kernel = nullptr;
  uint32_t threads = 256;
  uint32_t max_grid = 0;         // batched lookup CTAs when the copy engines stage
  uint32_t max_grid_beside = 0;  // ... when staging kernels share the SMs (one CTA slot per SM left)
  uint32_t gather_ctas = 0;      // key gather CTAs (two per SM: about 2.5 MB of host loads in flight)
  uint32_t scatter_ctas = 0;     // result scatter CTAs (one per SM)
  int pageable_access = 0;       // the device reads pageable host memory
  uint32_t max_reqs = 0;
  // key / result arena: a ring of `cap` key slots
  uint64_t* d_keys = nullptr;
  uint8_t* d_out = nullptr;
  KeyRing ring;
  Launch launches[kMaxInflight];
  std::deque<int> inflight;  // launch slots in submission order
  // requests
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> by_ticket;
  uint64_t next_ticket = 1;
  std::vector<double> latencies;  // completed requests since the last stats reset
  uint64_t keys_done = 0, reqs_done = 0, launches_done = 0;
  double stage_in_s = 0, lookup_s = 0, stage_out_s = 0;  // device time of completed launches
  double first_submit = 0, last_done = 0;
  std::thread worker;
  std::atomic<bool> stop{false};
  cudaError_t error = cudaSuccess;
};

namespace {

void complete_front(bf_server* s) {
  const int slot = s->inflight.front();
  Launch& L = s->launches[slot];
  const double t = now_s();
  std::lock_guard<std::mutex> g(s->mu);
  for (Request* r : L.reqs) {
    r->t_done = t;
    r->done = true;
    s->latencies.push_back(t - r->t_submit);
    s->keys_done += r->n;
    s->reqs_done += 1;
  }
  s->last_done = t;
  s->launches_done += 1;
  float ms = 0;
  if (cudaEventElapsedTime(&ms, L.in0, L.copied) == cudaSuccess) s->stage_in_s += ms * 1e-3;
  if (cudaEventElapsedTime(&ms, L.look0, L.looked) == cudaSuccess) s->lookup_s += ms * 1e-3;
  if (cudaEventElapsedTime(&ms, L.out0, L.done) == cudaSuccess) s->stage_out_s += ms * 1e-3;
  cudaGetLastError();
  s->ring.release(L.arena_used, L.arena_end);
  L.reqs.clear();
  L.busy = false;
  s->inflight.pop_front();
  s->cv_done.notify_all();
}

// Can the kernels read (keys) or write (results) this host buffer in place?
bool kernels_can_address(const bf_server* s, const void* p) {
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) return true;
  if (attr.type == cudaMemoryTypeHost) return attr.devicePointer == p;
  return s->pageable_access == 1;
}

// One launch: the requests' keys into the arena, one batched lookup, the
// results back.  When the kernels can address every request's buffers the
// staging kernels move them (gather on the copy-in stream, scatter on the
// copy-out stream; the batched lookup leaves them a CTA slot per SM), else
// the copy engine does, one copy per request and direction.
bool launch_batch(bf_server* s, int slot) {
  Launch& L = s->launches[slot];
  cudaError_t e = cudaSuccess;
  uint64_t chunks = 0;
  bool sm = true;
  for (const Request* r : L.reqs) sm = sm && r->addressable;
  e = cudaEventRecord(L.in0, s->h2d);
  for (size_t i = 0; i < L.reqs.size(); ++i) {
    Request* r = L.reqs[i];
    const BatchFilter& f = s->filters[r->filter];
    L.h_desc[i] = BatchFilter{f.words, f.nblocks, r->arena_off, r->n};
    L.h_begin[i] = chunks;
    L.h_src[i] = r->h_keys;
    L.h_dst[i] = r->h_out;
    chunks += (r->n + kBatchChunk - 1) / kBatchChunk;
    if (!sm && e == cudaSuccess && r->n)
      e = cudaMemcpyAsync(s->d_keys + r->arena_off, r->h_keys, r->n * 8, cudaMemcpyHostToDevice, s->h2d);
  }
  L.h_begin[L.reqs.size()] = chunks;
  const size_t nr = L.reqs.size();
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_desc, L.h_desc, sizeof(BatchFilter) * nr, cudaMemcpyHostToDevice, s->h2d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_begin, L.h_begin, sizeof(uint64_t) * (nr + 1), cudaMemcpyHostToDevice, s->h2d);
  if (sm) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_src, L.h_src, sizeof(void*) * nr, cudaMemcpyHostToDevice, s->h2d);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_dst, L.h_dst, sizeof(void*) * nr, cudaMemcpyHostToDevice, s->h2d);
    if (e == cudaSuccess)
      e = launch_batch_gather(L.d_desc, L.d_begin, static_cast<uint32_t>(nr), chunks, L.d_src, s->d_keys, s->gather_ctas,
                              s->h2d);
  }
  if (e == cudaSuccess) e = cudaEventRecord(L.copied, s->h2d);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, L.copied, 0);
  if (e == cudaSuccess) e = cudaEventRecord(L.look0, s->stream);
  if (e == cudaSuccess && chunks) {
    BatchArgs a{L.d_desc, L.d_begin, static_cast<uint32_t>(nr), chunks, s->d_keys, s->d_out,
                s->p.seed + 0x27D4EB2F165667C5ull + 8ull, 0u};
    const uint64_t ctas = (chunks + s->threads / 32 - 1) / (s->threads / 32);
    const uint32_t cap = sm ? s->max_grid_beside : s->max_grid;
    const uint32_t grid = static_cast<uint32_t>(std::max<uint64_t>(1, std::min<uint64_t>(ctas, cap)));
    void* args[] = {&a};
    e = cudaLaunchKernel(s->kernel->fn, dim3(grid), dim3(s->threads), args, 0, s->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(L.looked, s->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->d2h, L.looked, 0);
  if (e == cudaSuccess) e = cudaEventRecord(L.out0, s->d2h);
  if (sm) {
    if (e == cudaSuccess)
      e = launch_batch_scatter(L.d_desc, L.d_begin, static_cast<uint32_t>(nr), chunks, L.d_dst, s->d_out,
                               s->scatter_ctas, s->d2h);
  } else {
    for (size_t i = 0; i < nr && e == cudaSuccess; ++i) {
      Request* r = L.reqs[i];
      if (r->n) e = cudaMemcpyAsync(r->h_out, s->d_out + r->arena_off, r->n, cudaMemcpyDeviceToHost, s->d2h);
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(L.done, s->d2h);
  if (e != cudaSuccess) {
    s->error = e;
    return false;
  }
  s->inflight.push_back(slot);
  return true;
}

void worker_loop(bf_server* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    // complete finished launches, oldest first
    while (!s->inflight.empty()) {
      cudaError_t q = cudaEventQuery(s->launches[s->inflight.front()].done);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) s->error = q;
      complete_front(s);
    }
    // admit and launch
    int slot = -1;
    for (int i = 0; i < kMaxInflight; ++i)
      if (!s->launches[i].busy) slot = i;
    bool launched = false;
    if (slot >= 0) {
      Launch& L = s->launches[slot];
      {
        std::unique_lock<std::mutex> g(s->mu);
        L.arena_used = 0;
        // at most a kMaxInflight-th of the arena per launch (a larger request
        // goes alone), so that one launch's copies overlap another's kernel
        const uint64_t launch_cap = std::max<uint64_t>(1, s->ring.cap / kMaxInflight);
        uint64_t keys = 0;
        while (!s->pending.empty() && L.reqs.size() < s->max_reqs) {
          Request* r = s->pending.front();
          if (!L.reqs.empty() && keys + r->n > launch_cap) break;
          uint64_t off = 0, consumed = 0;
          if (!s->ring.take(r->n, &off, &consumed)) break;
          r->arena_off = off;
          L.arena_used += consumed;
          keys += r->n;
          L.reqs.push_back(r);
          s->pending.pop_front();
        }
        L.arena_end = s->ring.head;
      }
      if (!L.reqs.empty()) {
        L.busy = true;
        launched = launch_batch(s, slot);
        if (!launched) L.busy = false;
      }
    }
    if (!launched) {
      if (!s->inflight.empty()) {
        // nothing new to launch: wait briefly for the oldest launch or new work
        std::unique_lock<std::mutex> g(s->mu);
        s->cv_work.wait_for(g, std::chrono::microseconds(20));
      } else {
        std::unique_lock<std::mutex> g(s->mu);
        s->cv_work.wait_for(g, std::chrono::milliseconds(1), [s] { return !s->pending.empty() || s->stop.load(); });
      }
    }
  }
  while (!s->inflight.empty()) {
    cudaEventSynchronize(s->launches[s->inflight.front()].done);
    complete_front(s);
  }
}

}  // namespace

extern "C" {

bf_status bf_server_create(const bf_params* params, const bf_batch_filter* filters, uint32_t nfilters,
                           uint64_t arena_keys, uint32_t max_requests_per_launch, bf_server** out) {
  if (!out || !params || !filters || nfilters == 0 || arena_keys == 0 || max_requests_per_launch == 0)
    return BF_EINVAL;
  *out = nullptr;
  bf_params p = *params;
  p.num_blocks = 1;
  bf_status st = bf_params_check(&p);
  if (st != BF_OK) return st;
  const uint32_t s_words = p.block_bits / p.word_bits;
  if (p.groups != 0 && p.groups != s_words) return BF_EUNSUPPORTED;
  const uint64_t align = std::max<uint64_t>(32, p.block_bits / 8);
  for (uint32_t i = 0; i < nfilters; ++i)
    if (!filters[i].d_words || reinterpret_cast<uintptr_t>(filters[i].d_words) % align || filters[i].num_blocks == 0)
      return BF_EINVAL;
  // lookup layout: one thread per key, the whole block in one step, 4 keys per thread
  const KernelEntry* k = find_kernel(8, p.block_bits, p.word_bits, p.k, 1, s_words, 4, 0, static_cast<int>(p.salts));
  if (!k) return BF_EUNSUPPORTED;
  bf_server* s = new (std::nothrow) bf_server();
  if (!s) return BF_ENOMEM;
  s->p = p;
  s->kernel = k;
  s->ring.cap = arena_keys;
  s->max_reqs = max_requests_per_launch;
  for (uint32_t i = 0; i < nfilters; ++i) s->filters.push_back(BatchFilter{filters[i].d_words, filters[i].num_blocks, 0, 0});
  cudaError_t e = cudaGetDevice(&s->device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  const int per_sm = e == cudaSuccess ? kernel_resident_ctas(k->fn, s->threads, s->device) : 0;
  s->max_grid = static_cast<uint32_t>(std::max(1, sms * std::max(per_sm, 1)));
  s->max_grid_beside = static_cast<uint32_t>(std::max(1, sms * std::max(per_sm - 1, 1)));
  // two gather CTAs per SM: faster than one and four, as fast as three
  s->gather_ctas = static_cast<uint32_t>(std::max(1, 2 * sms));
  s->scatter_ctas = static_cast<uint32_t>(std::max(1, sms));
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->pageable_access, cudaDevAttrPageableMemoryAccess, s->device);
  int least = 0, greatest = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  // staging streams at the highest priority: the staging kernels' CTAs take free slots first
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->h2d, cudaStreamNonBlocking, greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->d2h, cudaStreamNonBlocking, greatest);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_keys, arena_keys * 8);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_out, arena_keys);
  for (int i = 0; i < kMaxInflight && e == cudaSuccess; ++i) {
    Launch& L = s->launches[i];
    e = cudaEventCreate(&L.done);
    if (e == cudaSuccess) e = cudaEventCreate(&L.copied);
    if (e == cudaSuccess) e = cudaEventCreate(&L.looked);
    if (e == cudaSuccess) e = cudaEventCreate(&L.in0);
    if (e == cudaSuccess) e = cudaEventCreate(&L.look0);
    if (e == cudaSuccess) e = cudaEventCreate(&L.out0);
    if (e == cudaSuccess) e = cudaHostAlloc(&L.h_desc, sizeof(BatchFilter) * s->max_reqs, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&L.h_begin, sizeof(uint64_t) * (s->max_reqs + 1), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&L.h_src, sizeof(void*) * s->max_reqs, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&L.h_dst, sizeof(void*) * s->max_reqs, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_desc, sizeof(BatchFilter) * s->max_reqs);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_begin, sizeof(uint64_t) * (s->max_reqs + 1));
    if (e == cudaSuccess) e = cudaMalloc(&L.d_src, sizeof(void*) * s->max_reqs);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_dst, sizeof(void*) * s->max_reqs);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    bf_server_destroy(s);
    return e == cudaErrorMemoryAllocation ? BF_ENOMEM : BF_ECUDA;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return BF_OK;
}

bf_status bf_server_destroy(bf_server* s) {
  if (!s) return BF_EINVAL;
  s->stop.store(true);
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->by_ticket) delete kv.second;
  for (Request* r : s->pending)
    if (!s->by_ticket.count(r->ticket)) delete r;
  for (auto& L : s->launches) {
    if (L.done) cudaEventDestroy(L.done);
    if (L.copied) cudaEventDestroy(L.copied);
    if (L.looked) cudaEventDestroy(L.looked);
    for (cudaEvent_t ev : {L.in0, L.look0, L.out0})
      if (ev) cudaEventDestroy(ev);
    if (L.h_desc) cudaFreeHost(L.h_desc);
    if (L.h_begin) cudaFreeHost(L.h_begin);
    if (L.h_src) cudaFreeHost(L.h_src);
    if (L.h_dst) cudaFreeHost(L.h_dst);
    if (L.d_desc) cudaFree(L.d_desc);
    if (L.d_begin) cudaFree(L.d_begin);
    if (L.d_src) cudaFree(L.d_src);
    if (L.d_dst) cudaFree(L.d_dst);
  }
  if (s->d_keys) cudaFree(s->d_keys);
  if (s->d_out) cudaFree(s->d_out);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->h2d) cudaStreamDestroy(s->h2d);
  if (s->d2h) cudaStreamDestroy(s->d2h);
  delete s;
  return BF_OK;
}

bf_status bf_server_submit(bf_server* s, uint32_t filter, const uint64_t* h_keys, uint64_t n, uint8_t* h_out,
                           uint64_t* ticket) {
  if (!s || !ticket || filter >= s->filters.size() || (n && (!h_keys || !h_out)) || n > s->ring.cap) return BF_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return BF_ENOMEM;
  r->filter = filter;
  r->h_keys = h_keys;
  r->n = n;
  r->h_out = h_out;
  r->t_submit = now_s();
  r->addressable = n == 0 || (reinterpret_cast<uintptr_t>(h_keys) % 8 == 0 && kernels_can_address(s, h_keys) &&
                              kernels_can_address(s, h_out));
  {
    std::lock_guard<std::mutex> g(s->mu);
    r->ticket = s->next_ticket++;
    if (s->first_submit == 0) s->first_submit = r->t_submit;
    s->by_ticket[r->ticket] = r;
    s->pending.push_back(r);
  }
  s->cv_work.notify_one();
  *ticket = r->ticket;
  return BF_OK;
}

bf_status bf_server_wait(bf_server* s, uint64_t ticket, double timeout_s, double* latency_s) {
  if (!s) return BF_EINVAL;
  std::unique_lock<std::mutex> g(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return BF_EINVAL;
  Request* r = it->second;
  const bool ok = s->cv_done.wait_for(g, std::chrono::duration<double>(timeout_s),
                                      [r, s] { return r->done || s->error != cudaSuccess; });
  if (s->error != cudaSuccess) return BF_ECUDA;
  if (!ok) return BF_ETIMEDOUT;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  s->by_ticket.erase(it);
  delete r;
  return BF_OK;
}

bf_status bf_server_get_stats(bf_server* s, int reset, bf_server_stats* out) {
  if (!s || !out) return BF_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->requests = s->reqs_done;
  out->keys = s->keys_done;
  out->launches = s->launches_done;
  if (!s->latencies.empty()) {
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&v](double q) { return v[std::min(v.size() - 1, static_cast<size_t>(q * (v.size() - 1) + 0.5))]; };
    out->p50_s = pct(0.50);
    out->p99_s = pct(0.99);
    out->max_s = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_s = sum / v.size();
  }
  out->span_s = s->last_done > s->first_submit ? s->last_done - s->first_submit : 0;
  out->stage_in_s = s->stage_in_s;
  out->lookup_s = s->lookup_s;
  out->stage_out_s = s->stage_out_s;
  if (reset) {
    s->latencies.clear();
    s->keys_done = s->reqs_done = s->launches_done = 0;
    s->first_submit = s->last_done = 0;
    s->stage_in_s = s->lookup_s = s->stage_out_s = 0;
  }
  return s->error == cudaSuccess ? BF_OK : BF_ECUDA;
}

bf_status bf_server_run_poisson(bf_server* s, double rate_per_s, double duration_s, uint64_t min_keys,
                                uint64_t max_keys, const uint64_t* h_key_pool, uint64_t pool_keys, uint8_t* h_out_pool,
                                uint64_t seed, bf_server_stats* out) {
  if (!s || !out || rate_per_s <= 0 || duration_s <= 0 || min_keys == 0 || max_keys < min_keys || !h_key_pool ||
      !h_out_pool || pool_keys < max_keys || max_keys > s->ring.cap)
    return BF_EINVAL;
  bf_server_stats dummy;
  bf_server_get_stats(s, 1, &dummy);
  uint64_t rng = seed;
  std::vector<uint64_t> tickets;
  uint64_t pool_pos = 0;
  const double t0 = now_s();
  double t_next = t0;
  const double lmin = std::log(static_cast<double>(min_keys)), lmax = std::log(static_cast<double>(max_keys) + 1.0);
  while (true) {
    t_next += -std::log(1.0 - uniform01(&rng)) / rate_per_s;  // exponential inter-arrival
    if (t_next - t0 > duration_s) break;
    const uint64_t n = std::min<uint64_t>(max_keys, static_cast<uint64_t>(std::exp(lmin + uniform01(&rng) * (lmax - lmin))));
    const uint32_t f = static_cast<uint32_t>(uniform01(&rng) * s->filters.size());
    if (pool_pos + n > pool_keys) pool_pos = 0;  // the pool is far larger than the keys in flight
    while (now_s() < t_next) {
    }
    uint64_t t = 0;
    bf_status st = bf_server_submit(s, f, h_key_pool + pool_pos, n, h_out_pool + pool_pos, &t);
    if (st != BF_OK) return st;
    tickets.push_back(t);
    pool_pos += n;
  }
  for (uint64_t t : tickets) {
    bf_status st = bf_server_wait(s, t, 600.0, nullptr);
    if (st != BF_OK) return st;
  }
  const bf_status st = bf_server_get_stats(s, 0, out);
  out->offered_s = duration_s;
  return st;
}

}  // extern "C"
