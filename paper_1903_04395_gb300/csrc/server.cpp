// server.cpp - a counting server over one device-resident graph, with
// continuous batching: requests (template, colorings) queue on the host; a
// scheduler thread admits them as soon as their device workspace fits in the
// free part of a fixed memory budget and an execution slot is free - of the
// first few queued requests the shortest (estimated device time) first, the
// head of the queue overtaken a bounded number of times; every admitted
// request runs its passes on its own stream, so requests overlap on the GPU; completions are
// detected with events, results copied back, memory returned, and the wait
// of the submitter released.  Latency = completion time - submission time.
// A request's stream takes a priority from its estimated device time (the
// planner's cost model times its colorings): shorter requests get higher
// priorities, so the GPU's block scheduler lets them through while long ones
// run (no request is ever held back: priorities only order ready blocks).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sgc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  const sgc_template* t = nullptr;
  std::vector<uint64_t> seeds;
  int precision = SGC_FP32;
  Clock::time_point t_submit, t_start, t_done;
  // execution
  std::shared_ptr<sgc::PlanSet> plans;
  std::map<int, const uint32_t*> tabs;
  int64_t off = 0, bytes = 0;  // workspace range in the arena
  int slot = -1;
  cudaStream_t st = nullptr;   // the slot's stream at this request's priority
  int bypassed = 0;            // admissions that overtook this request at the head
  // result
  bool finished = false;
  sgc_status status = SGC_OK;
  std::string error;
  std::vector<double> maps;
  double estimate = 0;
};

struct Range {
  int64_t off, len;
};

}  // namespace

struct sgc_server {
  const sgc_graph* g = nullptr;
  int64_t budget = 0;
  int max_inflight = 0;
  char* arena = nullptr;
  std::vector<Range> free_ranges;
  std::vector<std::vector<cudaStream_t>> streams;  // [priority level][slot], level 0 highest
  std::vector<cudaEvent_t> events;
  std::vector<std::shared_ptr<Request>> slots;  // in flight, by slot
  std::deque<std::shared_ptr<Request>> pending;
  std::map<uint64_t, std::shared_ptr<Request>> tickets;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  // statistics
  std::vector<double> latencies_ms, queue_ms;
  int64_t completed = 0, rejected = 0, peak_bytes = 0, used_bytes = 0, kernels = 0;
  int peak_inflight = 0;
  Clock::time_point t_first, t_last;
};

namespace sgc {
namespace {

constexpr int kLookahead = 8;  // queued requests considered for admission
constexpr int kMaxBypass = 8;  // admissions that may overtake the head of the queue

int64_t take_range(sgc_server* s, int64_t need) {
  need = (need + 255) / 256 * 256;
  for (size_t i = 0; i < s->free_ranges.size(); ++i) {
    Range& r = s->free_ranges[i];
    if (r.len >= need) {
      const int64_t off = r.off;
      r.off += need;
      r.len -= need;
      if (r.len == 0) s->free_ranges.erase(s->free_ranges.begin() + (int64_t)i);
      s->used_bytes += need;
      s->peak_bytes = std::max(s->peak_bytes, s->used_bytes);
      return off;
    }
  }
  return -1;
}

bool fits(const sgc_server* s, int64_t need) {
  need = (need + 255) / 256 * 256;
  for (const Range& r : s->free_ranges)
    if (r.len >= need) return true;
  return false;
}

void give_range(sgc_server* s, int64_t off, int64_t len) {
  len = (len + 255) / 256 * 256;
  s->used_bytes -= len;
  s->free_ranges.push_back({off, len});
  std::sort(s->free_ranges.begin(), s->free_ranges.end(), [](const Range& a, const Range& b) { return a.off < b.off; });
  std::vector<Range> merged;
  for (const Range& r : s->free_ranges) {
    if (!merged.empty() && merged.back().off + merged.back().len == r.off) merged.back().len += r.len;
    else merged.push_back(r);
  }
  s->free_ranges.swap(merged);
}

// workspace a request's passes need: the largest of its plans' (a pass of fewer colorings can need
// more than the top plan: one coloring per pass adds the neighbour-group buffers of the grouped SpMM)
int64_t request_ws(const Request& r) {
  int64_t ws = 0;
  for (const auto& kv : r.plans->by_batch) ws = std::max(ws, kv.second.ws_bytes);
  return (ws + 255) / 256 * 256;
}

// bytes a request needs: its workspace plus device room for seeds and results
int64_t request_bytes(const Request& r) { return request_ws(r) + (int64_t)r.seeds.size() * 16 + 256; }

void finish(sgc_server* s, const std::shared_ptr<Request>& r, sgc_status st, const std::string& err) {
  r->status = st;
  r->error = err;
  r->finished = true;
  r->t_done = Clock::now();
  if (st == SGC_OK) {
    s->completed++;
    s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    s->queue_ms.push_back(std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count());
    s->t_last = r->t_done;
  } else {
    s->rejected++;
  }
}

// Estimated device seconds of a request: the planner's cost model per coloring
// times its colorings.
double request_cost(const Request& r) {
  const Plan& top = r.plans->by_batch.at(r.plans->bfit);
  return top.est_cost * (double)r.seeds.size();
}

// Priority level of a request: level 0 (highest) below ~1 ms of estimated
// device time, one level lower for every factor of 4 more.
int priority_level(const sgc_server* s, const Request& r) {
  const double est_ms = 1e3 * request_cost(r);
  int level = 0;
  for (double x = 1.0; est_ms > x && level + 1 < (int)s->streams.size(); x *= 4.0) ++level;
  return level;
}

// Enqueue all passes of `r` on slot `slot`'s stream at its priority; the caller holds s->mu.
sgc_status launch(sgc_server* s, const std::shared_ptr<Request>& r, int slot) {
  const sgc_graph* g = s->g;
  r->st = s->streams[(size_t)priority_level(s, *r)][(size_t)slot];
  cudaStream_t st = r->st;
  char* base = s->arena + r->off;
  char* ws = base;
  const int64_t ws_len = request_ws(*r);
  uint64_t* d_seeds = reinterpret_cast<uint64_t*>(base + ws_len);
  double* d_maps = reinterpret_cast<double*>(d_seeds + r->seeds.size());
  const int32_t n = (int32_t)r->seeds.size();
  SGC_CUDA_TRY(cudaMemcpyAsync(d_seeds, r->seeds.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st));
  for (int32_t i = 0; i < n;) {
    int b = r->plans->bfit;
    while (b > n - i) b /= 2;
    const Plan& plan = r->plans->by_batch.at(b);
    if (plan.ws_bytes > ws_len) return fail(SGC_ERR_INTERNAL, "a pass's workspace exceeds the request's range");
    SGC_CUDA_TRY(cudaMemcpyAsync(ws + plan.bufs[plan.buf_seeds].offset, d_seeds + i, sizeof(uint64_t) * b,
                                 cudaMemcpyDeviceToDevice, st));
    int64_t nk = 0;
    sgc_status rc = run_pass(g, plan, r->tabs.at(b), ws, st, nullptr, &nk);
    if (rc != SGC_OK) return rc;
    s->kernels += nk;
    SGC_CUDA_TRY(cudaMemcpyAsync(d_maps + i, ws + plan.bufs[plan.buf_out].offset, sizeof(double) * b,
                                 cudaMemcpyDeviceToDevice, st));
    i += b;
  }
  SGC_CUDA_TRY(cudaEventRecord(s->events[slot], st));
  return SGC_OK;
}

// Plan a request (graph-level plan cache, under the graph's lock) and upload its tables.
sgc_status prepare(sgc_server* s, const std::shared_ptr<Request>& r) {
  sgc_options o;
  sgc_options_init(&o);
  o.precision = r->precision;
  const int bmax = pow2_floor(std::min<int>(32, (int)r->seeds.size()));
  {
    std::lock_guard<std::mutex> glock(s->g->mu);
    sgc_status rc = plan_batches(s->g, r->t, o, bmax, s->budget, &r->plans);
    if (rc != SGC_OK) return rc;
  }
  for (auto& kv : r->plans->by_batch) {
    const uint32_t* d = nullptr;
    sgc_status rc = template_tables(r->t, kv.second, s->g->device, &d);
    if (rc != SGC_OK) return rc;
    r->tabs[kv.first] = d;
  }
  return SGC_OK;
}

void scheduler(sgc_server* s) {
  cudaSetDevice(s->g->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (true) {
    // completions
    bool progressed = false;
    for (int slot = 0; slot < s->max_inflight; ++slot) {
      std::shared_ptr<Request> r = s->slots[slot];
      if (!r) continue;
      const cudaError_t q = cudaEventQuery(s->events[slot]);
      if (q == cudaErrorNotReady) continue;
      if (q == cudaSuccess) {
        const double* d_maps = reinterpret_cast<const double*>(s->arena + r->off + request_ws(*r) +
                                                               (int64_t)r->seeds.size() * 8);
        r->maps.assign(r->seeds.size(), 0.0);
        cudaError_t e = cudaMemcpyAsync(r->maps.data(), d_maps, sizeof(double) * r->maps.size(),
                                        cudaMemcpyDeviceToHost, r->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->st);
        if (e == cudaSuccess) {
          const int k = r->t->k;
          long double scale = 1.0L, sum = 0;
          for (int i = 1; i <= k; ++i) scale *= (long double)k / (long double)i;
          for (double m : r->maps) sum += (long double)m;
          r->estimate = (double)(sum / (long double)r->maps.size() / (long double)r->t->aut * scale);
          finish(s, r, SGC_OK, "");
        } else {
          finish(s, r, SGC_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
        }
      } else {
        finish(s, r, SGC_ERR_CUDA, std::string("request failed on the device: ") + cudaGetErrorString(q));
      }
      give_range(s, r->off, r->bytes);
      s->slots[slot].reset();
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    if (s->stop) {
      bool busy = false;
      for (auto& r : s->slots) busy = busy || (bool)r;
      if (!busy) break;
    }
    // admissions: among the first kLookahead queued requests, the shortest (estimated
    // device time) that fits in a free slot and the free budget; the head of the queue
    // is bypassed at most kMaxBypass times before it goes first
    while (!s->stop && !s->pending.empty()) {
      int slot = -1;
      for (int i = 0; i < s->max_inflight; ++i)
        if (!s->slots[i]) {
          slot = i;
          break;
        }
      if (slot < 0) break;
      // settle the window: trivial requests finish at once, the others get their plans
      bool restart = false;
      for (int look = 0; look < kLookahead && look < (int)s->pending.size(); ++look) {
        std::shared_ptr<Request> r = s->pending[look];
        if (r->t->k == 1 || s->g->n_act == 0) {
          // no pass needed: every vertex is a map (k = 1) or nothing maps (no edges)
          r->t_start = Clock::now();
          r->maps.assign(r->seeds.size(), r->t->k == 1 ? (double)s->g->n : 0.0);
          r->estimate = r->t->k == 1 ? (double)s->g->n : 0.0;
          finish(s, r, SGC_OK, "");
          s->pending.erase(s->pending.begin() + look);
          s->cv_done.notify_all();
          restart = true;
          break;
        }
        if (!r->plans) {
          // plan without holding the server lock; the queue may change meanwhile
          // (new submissions, or a shutdown that cancels everything queued)
          lock.unlock();
          sgc_status rc = prepare(s, r);
          std::string err = rc != SGC_OK ? std::string(sgc_last_error()) : std::string();
          lock.lock();
          auto pos = std::find(s->pending.begin(), s->pending.end(), r);
          if (s->stop || pos == s->pending.end()) {  // cancelled while planning
            restart = true;
            break;
          }
          if (rc == SGC_OK) {
            r->bytes = request_bytes(*r);
            if (r->bytes > s->budget) {
              rc = SGC_ERR_OOM;
              err = "request needs " + std::to_string(r->bytes) + " bytes, budget " + std::to_string(s->budget);
            }
          }
          if (rc != SGC_OK) {
            finish(s, r, rc, err);
            s->pending.erase(pos);
            s->cv_done.notify_all();
            restart = true;
            break;
          }
        }
      }
      if (restart) continue;
      // choose
      const std::shared_ptr<Request> head = s->pending.front();
      int best = -1;
      double best_cost = 0;
      const int window = head->bypassed >= kMaxBypass ? 1 : std::min<int>(kLookahead, (int)s->pending.size());
      for (int look = 0; look < window; ++look) {
        const Request& r = *s->pending[look];
        if (!fits(s, r.bytes)) continue;
        const double cost = request_cost(r);
        if (best < 0 || cost < best_cost) {
          best = look;
          best_cost = cost;
        }
      }
      if (best < 0) break;  // nothing fits until running requests finish
      if (best != 0) head->bypassed++;
      std::shared_ptr<Request> r = s->pending[best];
      r->off = take_range(s, r->bytes);
      r->slot = slot;
      r->t_start = Clock::now();
      s->pending.erase(s->pending.begin() + best);
      sgc_status rc = launch(s, r, slot);
      if (rc != SGC_OK) {
        cudaStreamSynchronize(r->st);
        give_range(s, r->off, r->bytes);
        finish(s, r, rc, sgc_last_error());
        s->cv_done.notify_all();
        continue;
      }
      s->slots[slot] = r;
      int inflight = 0;
      for (auto& x : s->slots) inflight += x ? 1 : 0;
      s->peak_inflight = std::max(s->peak_inflight, inflight);
    }
    bool any_inflight = false;
    for (auto& x : s->slots) any_inflight = any_inflight || (bool)x;
    // poll in-flight events at a fine grain; otherwise sleep until a submission arrives
    if (any_inflight) s->cv_work.wait_for(lock, std::chrono::microseconds(100));
    else if (!s->stop && s->pending.empty()) s->cv_work.wait(lock);
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
}

}  // namespace
}  // namespace sgc

using namespace sgc;

extern "C" {

sgc_status sgc_server_create(const sgc_graph* g, int64_t mem_budget, int32_t max_inflight, sgc_server** out) {
  if (!g || !out) return fail(SGC_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (mem_budget <= 0) return fail(SGC_ERR_INVALID, "mem_budget must be positive");
  if (max_inflight <= 0 || max_inflight > 64) return fail(SGC_ERR_INVALID, "max_inflight must be in [1, 64]");
  SGC_CUDA_TRY(cudaSetDevice(g->device));
  auto s = new sgc_server();
  s->g = g;
  s->budget = (mem_budget + 255) / 256 * 256;
  s->max_inflight = max_inflight;
  cudaError_t e = cudaMalloc(&s->arena, (size_t)s->budget);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return fail(SGC_ERR_OOM, "server memory budget of " + std::to_string(mem_budget) + " bytes: " +
                                 cudaGetErrorString(e));
  }
  s->free_ranges.push_back({0, s->budget});
  int least = 0, greatest = 0;  // numerically lower = higher priority
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  const int levels = std::max(1, least - greatest + 1);
  s->streams.assign((size_t)levels, std::vector<cudaStream_t>((size_t)max_inflight, nullptr));
  s->events.resize(max_inflight);
  s->slots.resize(max_inflight);
  for (int l = 0; l < levels; ++l)
    for (int i = 0; i < max_inflight; ++i)
      cudaStreamCreateWithPriority(&s->streams[(size_t)l][(size_t)i], cudaStreamNonBlocking, greatest + l);
  for (int i = 0; i < max_inflight; ++i) cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming);
  s->worker = std::thread(scheduler, s);
  *out = s;
  return SGC_OK;
}

sgc_status sgc_server_submit(sgc_server* s, const sgc_template* t, const uint64_t* seeds, int32_t n,
                             int32_t precision, uint64_t* ticket) {
  if (!s || !t || !ticket) return fail(SGC_ERR_INVALID, "NULL argument");
  if (n <= 0 || !seeds) return fail(SGC_ERR_INVALID, "need at least one seed");
  if (precision != SGC_FP32 && precision != SGC_FP64) return fail(SGC_ERR_INVALID, "unknown precision");
  auto r = std::make_shared<Request>();
  r->t = t;
  r->seeds.assign(seeds, seeds + n);
  r->precision = precision;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return fail(SGC_ERR_INVALID, "server is shutting down");
    if (s->next_ticket == 1) s->t_first = r->t_submit;
    r->ticket = s->next_ticket++;
    s->tickets[r->ticket] = r;
    s->pending.push_back(r);
  }
  s->cv_work.notify_one();
  *ticket = r->ticket;
  return SGC_OK;
}

sgc_status sgc_server_wait(sgc_server* s, uint64_t ticket, int32_t timeout_ms, double* estimate, double* maps,
                           double* latency_ms) {
  if (!s) return fail(SGC_ERR_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return fail(SGC_ERR_INVALID, "unknown ticket (or already waited for)");
  std::shared_ptr<Request> r = it->second;
  auto done = [&] { return r->finished; };
  if (timeout_ms < 0) s->cv_done.wait(lock, done);
  else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), done))
    return fail(SGC_ERR_TIMEOUT, "request " + std::to_string(ticket) + " not finished yet");
  s->tickets.erase(it);
  if (r->status != SGC_OK) return fail(r->status, r->error);
  if (estimate) *estimate = r->estimate;
  if (maps) std::memcpy(maps, r->maps.data(), sizeof(double) * r->maps.size());
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  return SGC_OK;
}

sgc_status sgc_server_stats_get(sgc_server* s, sgc_server_stats* out) {
  if (!s || !out) return fail(SGC_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  out->completed = s->completed;
  out->failed = s->rejected;
  out->pending = (int64_t)s->pending.size();
  int inflight = 0;
  for (auto& x : s->slots) inflight += x ? 1 : 0;
  out->inflight = inflight;
  out->peak_inflight = s->peak_inflight;
  out->peak_bytes = s->peak_bytes;
  out->kernel_launches = s->kernels;
  out->latency_p50_ms = percentile(s->latencies_ms, 0.50);
  out->latency_p99_ms = percentile(s->latencies_ms, 0.99);
  out->queue_p50_ms = percentile(s->queue_ms, 0.50);
  out->span_s = s->completed ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
  return SGC_OK;
}

void sgc_server_destroy(sgc_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    for (auto& r : s->pending) finish(s, r, SGC_ERR_INVALID, "server destroyed before the request started");
    s->pending.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->g->device);
  for (auto& level : s->streams)
    for (cudaStream_t st : level) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (int i = 0; i < s->max_inflight; ++i) {
    cudaEventDestroy(s->events[i]);
  }
  cudaFree(s->arena);
  delete s;
}

}  // extern "C"
