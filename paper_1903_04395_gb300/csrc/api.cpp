// api.cpp - the C ABI of libsgc (include/sgc.h): argument checks, handles,
// and the host-side driver of sgc_count (batching colorings, workspace,
// result read-back and the k^k/k! estimator of Section 2.1).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sgc_internal.h"

namespace sgc {

static bool trace_enabled() {
  static const bool on = std::getenv("SGC_TRACE") != nullptr;
  return on;
}

static long long now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

TraceScope::TraceScope(const char* n) : name(n), t0_ns(0), on(trace_enabled()) {
  nvtxRangePushA(n);
  if (on) t0_ns = now_ns();
}

TraceScope::~TraceScope() {
  nvtxRangePop();
  if (on) std::fprintf(stderr, "[sgc] %-16s %9.3f ms\n", name, 1e-6 * (double)(now_ns() - t0_ns));
}

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

sgc_status fail(sgc_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

sgc_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? SGC_ERR_OOM : SGC_ERR_CUDA;
}

// 1 / P(a fixed copy of a t-vertex template is colorful) with k colors:
// k^t (k - t)! / k! (k^k / k! for k = t, Section 2.1); colors = 0 means k = t
long double inverse_colorful_probability(int t, int colors) {
  const int k = colors > t ? colors : t;
  long double x = 1.0L;
  for (int i = 0; i < t; ++i) x *= (long double)k / (long double)(k - i);
  return x;
}

int pow2_floor(int x) {
  int p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

// device copy of a plan's index tables, cached per (device, content hash, size)
sgc_status template_tables(const sgc_template* t, const Plan& plan, int device, const uint32_t** out) {
  std::lock_guard<std::mutex> lock(t->mu);
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the table words
  for (uint32_t w : plan.tabs) {
    h ^= w;
    h *= 1099511628211ull;
  }
  std::array<uint64_t, 3> key{(uint64_t)device, h, (uint64_t)plan.tabs.size()};
  for (auto& kv : t->tab_cache)
    if (kv.first == key) {
      *out = kv.second;
      return SGC_OK;
    }
  uint32_t* d = nullptr;
  const size_t bytes = std::max<size_t>(plan.tabs.size(), 4) * sizeof(uint32_t);
  SGC_CUDA_TRY(cudaMalloc(&d, bytes));
  if (!plan.tabs.empty()) {
    cudaError_t e = cudaMemcpy(d, plan.tabs.data(), plan.tabs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "uploading index tables");
    }
  }
  t->tab_cache.push_back({key, d});
  *out = d;
  return SGC_OK;
}

namespace {

// One workspace per device, shared by every graph on it.  Passes on
// different streams are ordered through `last`, an event recorded after the
// most recent pass that used the workspace.
struct DevicePool {
  std::mutex mu;
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaEvent_t last = nullptr;
};

DevicePool& device_pool(int dev) {
  static DevicePool pools[64];
  return pools[dev & 63];
}

sgc_status ensure_workspace(DevicePool& pool, int64_t bytes) {
  if ((int64_t)pool.bytes >= bytes) return SGC_OK;
  if (pool.ptr) {
    if (pool.last) SGC_CUDA_TRY(cudaEventSynchronize(pool.last));
    cudaFree(pool.ptr);
    pool.ptr = nullptr;
    pool.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&pool.ptr, (size_t)bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SGC_ERR_OOM, "device workspace of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  pool.bytes = (size_t)bytes;
  return SGC_OK;
}

sgc_status check_handles(const sgc_graph* g, const sgc_template* t) {
  if (!g) return fail(SGC_ERR_INVALID, "graph is NULL");
  if (!t) return fail(SGC_ERR_INVALID, "template is NULL");
  return SGC_OK;
}

}  // namespace

sgc_options resolve(const sgc_options* opt) {
  sgc_options o;
  sgc_options_init(&o);
  if (opt) o = *opt;
  return o;
}

// Plans for every power-of-two batch up to bmax that fits mem_limit; the
// root and cut order come from the cost model once and are shared.  Cached on
// the graph per (template, precision, root, bmax).
// the largest workspace among a plan set's batch sizes (a pass of one coloring can need more than a
// larger batch's: the grouped SpMM's neighbour-group buffers)
static int64_t max_ws(const PlanSet& set) {
  int64_t ws = 0;
  for (const auto& kv : set.by_batch) ws = std::max(ws, kv.second.ws_bytes);
  return ws;
}

// Untuned plan sets depend on the graph only through its sizes (active vertices, stored entries,
// heavy rows and their segments) and the device's SM count and shared memory, so they are also kept
// process-wide: a new handle for a graph of the same shape (a graph uploaded again) reuses them.
// Tuned sets hold measurements of one graph and stay with it.
static std::mutex g_shared_plans_mu;
static std::vector<std::pair<std::string, std::shared_ptr<PlanSet>>> g_shared_plans;

static std::string graph_signature(const sgc_graph* g) {
  return std::to_string(g->n_act) + "," + std::to_string(g->nnz) + "," + std::to_string(g->n_heavy) + "," +
         std::to_string(g->n_seg) + "," + std::to_string(g->num_sms) + "," + std::to_string(g->smem_optin) + "|";
}

sgc_status plan_batches(const sgc_graph* g, const sgc_template* t, const sgc_options& o, int bmax, int64_t mem_limit,
                        std::shared_ptr<PlanSet>* out) {
  const std::string key = std::to_string(t->uid) + "/" + std::to_string(o.precision) + "/" + std::to_string(o.root) +
                          "/" + std::to_string(bmax) + (o.autotune ? "/tuned" : "") + "/s" +
                          std::to_string(o.spmm_shape) + "/e" + std::to_string(o.ema_rows) + "/c" +
                          std::to_string(o.colors) + (o.unpruned ? "/unpruned" + std::to_string(o.unpruned) : "");
  for (auto& kv : g->plan_cache)
    if (kv.first == key && max_ws(*kv.second) <= mem_limit) {
      *out = kv.second;
      return SGC_OK;
    }
  const std::string shared_key = graph_signature(g) + key;
  if (!o.autotune) {
    std::lock_guard<std::mutex> lock(g_shared_plans_mu);
    for (auto& kv : g_shared_plans)
      if (kv.first == shared_key && max_ws(*kv.second) <= mem_limit) {
        if (g->plan_cache.size() >= 64) g->plan_cache.erase(g->plan_cache.begin());
        g->plan_cache.push_back({key, kv.second});
        *out = kv.second;
        return SGC_OK;
      }
  }
  auto set = std::make_shared<PlanSet>();
  const bool forced = o.spmm_shape != 0 || o.ema_rows != 0;
  // forced launch shapes, as one code per op index of a plan
  auto forced_shapes = [&](const Plan& p) {
    std::vector<int> sh(p.ops.size(), 0);
    for (size_t i = 0; i < p.ops.size(); ++i)
      sh[i] = p.ops[i].kind == OP_SPMM ? o.spmm_shape : p.ops[i].kind == OP_EMA ? o.ema_rows : 0;
    return sh;
  };
  Plan p1;
  sgc_status rc = make_plan(g, t, o.precision, o.root, -1, 1, true, &p1, nullptr, o.colors, o.unpruned);
  if (rc != SGC_OK) return rc;
  if (forced) {
    const std::vector<int> sh = forced_shapes(p1);
    if ((rc = make_plan(g, t, o.precision, p1.root, p1.policy, 1, true, &p1, &sh,
                        o.colors, o.unpruned)) != SGC_OK) return rc;
  }
  if (p1.ws_bytes > mem_limit)
    return fail(SGC_ERR_OOM, "one coloring needs " + std::to_string(p1.ws_bytes) +
                                 " bytes of device workspace, limit " +
                                 std::to_string(mem_limit));
  const int root = p1.root, policy = p1.policy;
  // Occupancy cap: a SpMM warp keeps a whole output row of `batch` colorings in
  // shared memory, so wide rows take fewer colorings per pass (at most ~8 KB
  // per warp keeps several blocks resident per SM).
  int64_t widest = 0;
  for (const PlanOp& op : p1.ops)
    if (op.kind == OP_SPMM) widest = std::max<int64_t>(widest, op.ld_out * p1.elem);
  while (bmax > 1 && widest * bmax > kSpmmRowBytesPerWarp) bmax /= 2;
  // one coloring per pass by default where the staged SpMM takes an op of more than 256 columns
  // (R-MAT 21: the 12-vertex path at 39 ms per coloring against 58 at 4 per pass, the 13-vertex
  // tree 59 against 83 at 2; the autotuner still measures the larger batches)
  bool one = false;
  for (const PlanOp& op : p1.ops)
    one |= op.kind == OP_SPMM && (op.spmm_variant == 16 || op.spmm_variant == 17) && op.cols_p > 256;
  set->by_batch[1] = std::move(p1);
  set->bfit = 1;
  set->btop = 1;
  for (int b = 2; b <= bmax; b *= 2) {
    Plan pb;
    rc = make_plan(g, t, o.precision, root, policy, b, true, &pb, nullptr, o.colors, o.unpruned);
    if (rc != SGC_OK) return rc;
    if (forced) {
      const std::vector<int> sh = forced_shapes(pb);
      if ((rc = make_plan(g, t, o.precision, root, policy, b, true, &pb, &sh,
                          o.colors, o.unpruned)) != SGC_OK) return rc;
    }
    if (pb.ws_bytes > mem_limit) break;
    set->by_batch[b] = std::move(pb);
    set->btop = b;
    if (!one) set->bfit = b;
  }
  for (auto& kv : g->plan_cache)
    if (kv.first == key) {
      kv.second = set;
      *out = set;
      return SGC_OK;
    }
  if (g->plan_cache.size() >= 64) g->plan_cache.erase(g->plan_cache.begin());
  g->plan_cache.push_back({key, set});
  if (!o.autotune) {
    std::lock_guard<std::mutex> lock(g_shared_plans_mu);
    if (g_shared_plans.size() >= 64) g_shared_plans.erase(g_shared_plans.begin());
    g_shared_plans.push_back({shared_key, set});
  }
  *out = set;
  return SGC_OK;
}

namespace {

// ------------------------------------------------------------ autotuner
// Times every candidate launch shape of each SpMM and eMA op of the plans for
// the two largest batch sizes, on this graph, and keeps the fastest shape per
// op and the batch size with the lower time per coloring.  Shapes only change
// how the same sums are scheduled (Eq. 2 and the eMA of Section 4.5).

struct TimedPass {
  std::vector<double> op_ms;  // per op index
  double total_ms = 0;
};

sgc_status time_pass(const sgc_graph* g, const Plan& plan, DevicePool& pool, cudaStream_t st, TimedPass* out) {
  sgc_status rc = ensure_workspace(pool, plan.ws_bytes);
  if (rc != SGC_OK) return rc;
  char* ws = static_cast<char*>(pool.ptr);
  uint32_t* d_tabs = nullptr;
  const size_t tab_bytes = std::max<size_t>(plan.tabs.size(), 4) * sizeof(uint32_t);
  SGC_CUDA_TRY(cudaMalloc(&d_tabs, tab_bytes));
  std::vector<uint64_t> seeds((size_t)plan.batch);
  for (int b = 0; b < plan.batch; ++b) seeds[(size_t)b] = 0x5EEDull + (uint64_t)b;
  cudaError_t e = cudaSuccess;
  if (!plan.tabs.empty())
    e = cudaMemcpyAsync(d_tabs, plan.tabs.data(), plan.tabs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + plan.bufs[plan.buf_seeds].offset, seeds.data(), seeds.size() * sizeof(uint64_t),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(d_tabs);
    return cuda_fail(e, "autotuner set-up");
  }
  Profiler prof;
  prof.on = true;
  prof.by_index = true;
  int64_t nk = 0;
  // one untimed pass (first-touch of the tables), then the timed one
  rc = run_pass(g, plan, d_tabs, ws, st, nullptr, &nk);
  if (rc == SGC_OK) rc = run_pass(g, plan, d_tabs, ws, st, &prof, &nk);
  e = cudaStreamSynchronize(st);
  out->op_ms.assign(plan.ops.size(), 0.0);
  out->total_ms = 0;
  for (auto& pe : prof.pending) {
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pe.e0, pe.e1);
    out->op_ms[(size_t)pe.slot] += ms;
    out->total_ms += ms;
    cudaEventDestroy(pe.e0);
    cudaEventDestroy(pe.e1);
  }
  cudaFree(d_tabs);
  if (rc != SGC_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "autotuner pass");
  return SGC_OK;
}

sgc_status tune_plans(const sgc_graph* g, const sgc_template* t, const sgc_options& o, PlanSet* set,
                      DevicePool& pool, cudaStream_t st) {
  SGC_TRACE_SCOPE("autotune");
  // the largest batch and up to two halvings: wide rows favour smaller batches
  std::vector<int> batches{set->btop};
  for (int b = set->btop / 2; b >= 1 && batches.size() < 3 && set->by_batch.count(b); b /= 2) batches.push_back(b);
  std::vector<sgc_tune_entry> report;
  sgc_tune_entry bt{};
  bt.kind = -1;
  int best_b = set->btop;
  double best_per = 0;
  for (int b : batches) {
    const Plan& base = set->by_batch.at(b);
    const size_t nops = base.ops.size();
    std::vector<std::vector<int>> cands(nops);
    size_t ncand = 1;
    for (size_t i = 0; i < nops; ++i) {
      cands[i] = op_shape_candidates(g, base, (int)i);
      if (cands[i].size() > 8) cands[i].resize(8);
      ncand = std::max(ncand, cands[i].size());
    }
    std::vector<std::vector<double>> ms(nops, std::vector<double>(ncand, -1.0));
    std::vector<double> fixed_ms(nops, 0.0);
    for (size_t c = 0; c < ncand; ++c) {
      std::vector<int> shapes(nops, 0);
      for (size_t i = 0; i < nops; ++i)
        if (!cands[i].empty()) shapes[i] = cands[i][std::min(c, cands[i].size() - 1)];
      Plan p;
      sgc_status rc = make_plan(g, t, o.precision, base.root, base.policy, b, true, &p, &shapes,
                                o.colors, o.unpruned);
      if (rc != SGC_OK) return rc;
      TimedPass tp;
      if ((rc = time_pass(g, p, pool, st, &tp)) != SGC_OK) return rc;
      for (size_t i = 0; i < nops; ++i) {
        if (cands[i].empty()) {
          fixed_ms[i] = c == 0 ? tp.op_ms[i] : std::min(fixed_ms[i], tp.op_ms[i]);
        } else if (c < cands[i].size()) {
          ms[i][c] = tp.op_ms[i];
        }
      }
    }
    std::vector<int> best(nops, 0);
    double pass_ms = 0;
    for (size_t i = 0; i < nops; ++i) {
      if (cands[i].empty()) {
        pass_ms += fixed_ms[i];
        continue;
      }
      size_t arg = 0;
      for (size_t c = 1; c < cands[i].size(); ++c)
        if (ms[i][c] < ms[i][arg]) arg = c;
      best[i] = cands[i][arg];
      pass_ms += ms[i][arg];
      const PlanOp& op = base.ops[i];
      sgc_tune_entry te{};
      te.kind = op.kind;
      te.t = op.t;
      te.a = op.a;
      te.p = op.p;
      te.batch = b;
      te.n_candidates = (int32_t)cands[i].size();
      te.chosen = (int32_t)arg;
      for (size_t c = 0; c < cands[i].size(); ++c) {
        te.shapes[c] = cands[i][c];
        te.ms[c] = ms[i][c];
      }
      report.push_back(te);
    }
    Plan tuned;
    sgc_status rc = make_plan(g, t, o.precision, base.root, base.policy, b, true, &tuned, &best,
                              o.colors, o.unpruned);
    if (rc != SGC_OK) return rc;
    set->by_batch[b] = std::move(tuned);
    const double per = pass_ms / b;
    bt.shapes[bt.n_candidates] = b;
    bt.ms[bt.n_candidates] = per;
    if (bt.n_candidates == 0 || per < best_per) {
      best_per = per;
      best_b = b;
      bt.chosen = bt.n_candidates;
    }
    bt.n_candidates++;
  }
  bt.batch = best_b;
  report.push_back(bt);
  set->bfit = best_b;
  set->tuned = true;
  set->report = std::move(report);
  return SGC_OK;
}

// --------------------------------------------------------------- counting

struct Job {
  const sgc_template* t = nullptr;
  std::shared_ptr<PlanSet> plans;
  std::map<int, const uint32_t*> d_tabs;  // device index tables per batch size
  int lane = 0;                           // stream: 0 = the call's stream, l > 0 = g->lanes[l - 1]
  double cost = 0;                        // cost-model seconds for all its colorings
  int64_t ws = 0;                         // workspace of its largest pass
};

constexpr int kMaxLanes = 4;
constexpr int64_t kAlign = 256;

int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

sgc_status ensure_lanes(const sgc_graph* g, int n_lanes) {
  while ((int)g->lanes.size() < n_lanes - 1) {
    cudaStream_t s = nullptr;
    SGC_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    g->lanes.push_back(s);
  }
  while ((int)g->lane_events.size() < n_lanes) {
    cudaEvent_t e = nullptr;
    SGC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    g->lane_events.push_back(e);
  }
  return SGC_OK;
}

// Every pass of every job.  Seeds are read from, and colorful maps written to,
// the staging arrays at the front of the workspace (job j, coloring i at
// j * n_iter + i), so that a recorded launch sequence serves any seeds.
sgc_status enqueue_jobs(const sgc_graph* g, const std::vector<Job>& jobs, int n_lanes,
                        const std::vector<int64_t>& lane_off, char* ws, const uint64_t* d_seeds, double* d_maps,
                        int32_t n_iter, cudaStream_t st, Profiler* prof, int64_t* kernels) {
  if (n_lanes > 1) {
    SGC_CUDA_TRY(cudaEventRecord(g->lane_events[0], st));
    for (int l = 1; l < n_lanes; ++l) SGC_CUDA_TRY(cudaStreamWaitEvent(g->lanes[l - 1], g->lane_events[0], 0));
  }
  for (size_t j = 0; j < jobs.size(); ++j) {
    const Job& J = jobs[j];
    cudaStream_t ls = J.lane == 0 ? st : g->lanes[J.lane - 1];
    char* w = ws + lane_off[J.lane];
    for (int32_t i = 0; i < n_iter;) {
      int b = J.plans->bfit;
      while (b > n_iter - i) b /= 2;
      const Plan& plan = J.plans->by_batch.at(b);
      const size_t at = j * (size_t)n_iter + (size_t)i;
      SGC_CUDA_TRY(cudaMemcpyAsync(w + plan.bufs[plan.buf_seeds].offset, d_seeds + at, sizeof(uint64_t) * b,
                                   cudaMemcpyDeviceToDevice, ls));
      sgc_status rc = run_pass(g, plan, J.d_tabs.at(b), w, ls, prof, kernels);
      if (rc != SGC_OK) return rc;
      SGC_CUDA_TRY(cudaMemcpyAsync(d_maps + at, w + plan.bufs[plan.buf_out].offset, sizeof(double) * b,
                                   cudaMemcpyDeviceToDevice, ls));
      i += b;
    }
  }
  if (n_lanes > 1) {
    for (int l = 1; l < n_lanes; ++l) {
      SGC_CUDA_TRY(cudaEventRecord(g->lane_events[l], g->lanes[l - 1]));
      SGC_CUDA_TRY(cudaStreamWaitEvent(st, g->lane_events[l], 0));
    }
  }
  return SGC_OK;
}

// Record the jobs' launch sequence as one CUDA graph (or reuse the recording
// made by an earlier call with the same key) and launch it on st.
sgc_status launch_recorded(const sgc_graph* g, const std::string& key, const std::vector<Job>& jobs, int n_lanes,
                           const std::vector<int64_t>& lane_off, char* ws, const uint64_t* d_seeds, double* d_maps,
                           int32_t n_iter, cudaStream_t st) {
  for (auto& x : g->exec_cache)
    if (x.key == key && x.ws == ws) {
      SGC_CUDA_TRY(cudaGraphLaunch(x.exec, st));
      g->kernel_launches += x.kernels;
      return SGC_OK;
    }
  SGC_TRACE_SCOPE("count.record");
  int64_t nk = 0;
  SGC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  sgc_status rc = enqueue_jobs(g, jobs, n_lanes, lane_off, ws, d_seeds, d_maps, n_iter, st, nullptr, &nk);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc != SGC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "recording the launch sequence");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "instantiating the launch sequence");
  ExecEntry x;
  x.key = key;
  x.exec = exec;
  x.ws = ws;
  x.kernels = nk;
  for (const Job& J : jobs) x.plans.push_back(J.plans);
  if (g->exec_cache.size() >= 16) {
    cudaGraphExecDestroy(g->exec_cache.front().exec);
    g->exec_cache.erase(g->exec_cache.begin());
  }
  g->exec_cache.push_back(std::move(x));
  SGC_CUDA_TRY(cudaGraphLaunch(exec, st));
  g->kernel_launches += nk;
  return SGC_OK;
}

// The counting driver behind sgc_count, sgc_count_device and sgc_count_many:
// n_t templates, n_iter colorings each; seeds[j * n_iter + i] is coloring i of
// template j (host or, with device_io, device), maps the same layout.
sgc_status count_core(const sgc_graph* g, int32_t n_t, const sgc_template* const* ts, const uint64_t* seeds,
                      int32_t n_iter, const sgc_options* opt_in, bool device_io, double* estimates, double* maps_out) {
  if (!g) return fail(SGC_ERR_INVALID, "graph is NULL");
  if (n_t < 0) return fail(SGC_ERR_INVALID, "n_templates must be >= 0");
  if (n_t > 0 && !ts) return fail(SGC_ERR_INVALID, "templates is NULL");
  for (int32_t j = 0; j < n_t; ++j)
    if (!ts[j]) return fail(SGC_ERR_INVALID, "template is NULL");
  if (n_iter < 0) return fail(SGC_ERR_INVALID, "n_iter must be >= 0");
  if (n_iter > 0 && n_t > 0 && !seeds) return fail(SGC_ERR_INVALID, "seeds is NULL");
  if (device_io && n_iter > 0 && n_t > 0 && !maps_out) return fail(SGC_ERR_INVALID, "colorful_maps is NULL");
  const sgc_options o = resolve(opt_in);
  if (o.precision != SGC_FP32 && o.precision != SGC_FP64) return fail(SGC_ERR_INVALID, "unknown precision");
  for (int32_t j = 0; j < n_t; ++j) {
    if (o.root >= ts[j]->k || o.root < -1) return fail(SGC_ERR_INVALID, "options.root out of range");
    if (o.colors != 0 && (o.colors < ts[j]->k || o.colors > SGC_MAX_K))
      return fail(SGC_ERR_INVALID, "options.colors must be 0 or in [|T|, " + std::to_string(SGC_MAX_K) + "]");
  }
  if (o.batch < 0) return fail(SGC_ERR_INVALID, "options.batch must be >= 0");
  if (o.unpruned < 0 || o.unpruned > 2) return fail(SGC_ERR_INVALID, "options.unpruned must be 0, 1 or 2");
  if (o.spmm_shape < 0 || o.spmm_shape > kShapeSpmmStaged8)
    return fail(SGC_ERR_INVALID, "options.spmm_shape must be 0.." + std::to_string(kShapeSpmmStaged8));
  if (o.ema_rows != 0 && o.ema_rows != 64 && o.ema_rows != 32 && o.ema_rows != 16 && o.ema_rows != 8 &&
      o.ema_rows != 4 && o.ema_rows != 2 && o.ema_rows != 1 && o.ema_rows != kShapeEmaVertex1 &&
      o.ema_rows != kShapeEmaVertex2 && o.ema_rows != kShapeEmaReg && o.ema_rows != kShapeEmaSched &&
      o.ema_rows != kShapeEmaSched2)
    return fail(SGC_ERR_INVALID, "options.ema_rows must be 0, 64, 32, 16, 8, 4, 2, 1, 101, 102, 103, 104 or 105");
  SGC_CUDA_TRY(cudaSetDevice(g->device));
  std::lock_guard<std::mutex> lock(g->mu);
  DevicePool& pool = device_pool(g->device);
  std::lock_guard<std::mutex> pool_lock(pool.mu);
  cudaStream_t st = o.stream ? (cudaStream_t)o.stream : g->stream;
  if (estimates)
    for (int32_t j = 0; j < n_t; ++j) estimates[j] = 0.0;
  if (n_iter == 0 || n_t == 0) return SGC_OK;
  sgc_status rc = SGC_OK;
  const size_t total = (size_t)n_t * (size_t)n_iter;
  std::vector<double> host_maps(total, 0.0);

  // templates with one vertex, and graphs without edges, need no DP
  std::vector<Job> jobs;
  std::vector<int32_t> job_of(n_t, -1);
  bool special_only = true;
  for (int32_t j = 0; j < n_t; ++j) {
    if (ts[j]->k == 1 || g->n_act == 0) {
      const double v = ts[j]->k == 1 ? (double)g->n : 0.0;
      std::fill(host_maps.begin() + (size_t)j * n_iter, host_maps.begin() + (size_t)(j + 1) * n_iter, v);
    } else {
      special_only = false;
    }
  }

  if (!special_only) {
    size_t free_b = 0, total_b = 0;
    SGC_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const int64_t staging = 2 * align_up((int64_t)(total * sizeof(double)));
    const int64_t mem_limit =
        (o.mem_limit > 0 ? o.mem_limit : (int64_t)((free_b + pool.bytes) * 0.9)) - staging;
    if (mem_limit <= 0) return fail(SGC_ERR_OOM, "no device memory left for the workspace");
    const int bmax = pow2_floor(std::min(32, o.batch > 0 ? o.batch : std::max(1, (int)n_iter)));
    SGC_TRACE_SCOPE("count.plan");
    for (int32_t j = 0; j < n_t; ++j) {
      if (ts[j]->k == 1 || g->n_act == 0) continue;
      Job J;
      J.t = ts[j];
      if ((rc = plan_batches(g, ts[j], o, bmax, mem_limit, &J.plans)) != SGC_OK) return rc;
      if (o.autotune && !J.plans->tuned && o.spmm_shape == 0 && o.ema_rows == 0) {
        if (pool.last) SGC_CUDA_TRY(cudaEventSynchronize(pool.last));
        if ((rc = tune_plans(g, ts[j], o, J.plans.get(), pool, st)) != SGC_OK) return rc;
      }
      // every batch size has its own plan and index tables (the SpMM form can
      // depend on the batch), each uploaded once and cached by content
      for (auto& kv : J.plans->by_batch) {
        const uint32_t* d = nullptr;
        if ((rc = template_tables(ts[j], kv.second, g->device, &d)) != SGC_OK) return rc;
        J.d_tabs[kv.first] = d;
        J.ws = std::max(J.ws, kv.second.ws_bytes);
      }
      const Plan& top = J.plans->by_batch.at(J.plans->bfit);
      J.cost = top.est_cost * (double)n_iter;
      job_of[j] = (int32_t)jobs.size();
      jobs.push_back(std::move(J));
    }

    // side-by-side streams: longest job first onto the least loaded stream,
    // fewer streams while the workspaces do not fit
    std::vector<size_t> order(jobs.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return jobs[x].cost > jobs[y].cost; });
    int n_lanes = std::min<int>(kMaxLanes, (int)jobs.size());
    std::vector<int64_t> lane_ws;
    for (;; --n_lanes) {
      std::vector<double> load((size_t)n_lanes, 0.0);
      lane_ws.assign((size_t)n_lanes, 0);
      for (size_t x : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        jobs[x].lane = l;
        load[(size_t)l] += jobs[x].cost;
        lane_ws[(size_t)l] = std::max(lane_ws[(size_t)l], align_up(jobs[x].ws));
      }
      int64_t sum = 0;
      for (int64_t w : lane_ws) sum += w;
      if (sum <= mem_limit || n_lanes == 1) break;
    }
    std::vector<int64_t> lane_off((size_t)n_lanes, 0);
    int64_t ws_total = staging;
    for (int l = 0; l < n_lanes; ++l) {
      lane_off[(size_t)l] = ws_total;
      ws_total += lane_ws[(size_t)l];
    }
    if ((rc = ensure_lanes(g, n_lanes)) != SGC_OK) return rc;
    if ((rc = ensure_workspace(pool, ws_total)) != SGC_OK) return rc;
    if (!pool.last) SGC_CUDA_TRY(cudaEventCreateWithFlags(&pool.last, cudaEventDisableTiming));
    SGC_CUDA_TRY(cudaStreamWaitEvent(st, pool.last, 0));
    char* ws = static_cast<char*>(pool.ptr);
    uint64_t* d_seeds = reinterpret_cast<uint64_t*>(ws);
    double* d_maps = reinterpret_cast<double*>(ws + staging / 2);

    // seeds of the jobs, in job order
    std::vector<uint64_t> job_seeds;
    if (!device_io) job_seeds.resize(jobs.size() * (size_t)n_iter);
    for (int32_t j = 0; j < n_t; ++j) {
      if (job_of[j] < 0) continue;
      const size_t dst = (size_t)job_of[j] * n_iter, src = (size_t)j * n_iter;
      if (device_io) {
        SGC_CUDA_TRY(cudaMemcpyAsync(d_seeds + dst, seeds + src, sizeof(uint64_t) * n_iter,
                                     cudaMemcpyDeviceToDevice, st));
      } else {
        std::copy(seeds + src, seeds + src + n_iter, job_seeds.begin() + dst);
      }
    }
    if (!device_io)
      SGC_CUDA_TRY(cudaMemcpyAsync(d_seeds, job_seeds.data(), job_seeds.size() * sizeof(uint64_t),
                                   cudaMemcpyHostToDevice, st));

    Profiler* prof = g->prof.on ? &g->prof : nullptr;
    if (o.use_graph && !prof) {
      std::string key = "n" + std::to_string(n_iter) + "/l" + std::to_string(n_lanes);
      for (const Job& J : jobs)
        key += "/" + std::to_string(J.t->uid) + ":" + std::to_string(reinterpret_cast<uintptr_t>(J.plans.get())) +
               ":" + std::to_string(J.plans->bfit) + ":" + std::to_string(J.lane);
      rc = launch_recorded(g, key, jobs, n_lanes, lane_off, ws, d_seeds, d_maps, n_iter, st);
    } else {
      rc = enqueue_jobs(g, jobs, n_lanes, lane_off, ws, d_seeds, d_maps, n_iter, st, prof, &g->kernel_launches);
    }
    if (rc != SGC_OK) return rc;

    // results back, template order
    for (int32_t j = 0; j < n_t; ++j) {
      if (job_of[j] < 0) continue;
      const size_t src = (size_t)job_of[j] * n_iter, dst = (size_t)j * n_iter;
      if (device_io) {
        SGC_CUDA_TRY(cudaMemcpyAsync(maps_out + dst, d_maps + src, sizeof(double) * n_iter,
                                     cudaMemcpyDeviceToDevice, st));
      } else {
        SGC_CUDA_TRY(cudaMemcpyAsync(host_maps.data() + dst, d_maps + src, sizeof(double) * n_iter,
                                     cudaMemcpyDeviceToHost, st));
      }
    }
    SGC_CUDA_TRY(cudaEventRecord(pool.last, st));
  }
  if (device_io) {
    // templates that needed no DP
    bool copied = false;
    for (int32_t j = 0; j < n_t; ++j)
      if (job_of[j] < 0) {
        SGC_CUDA_TRY(cudaMemcpyAsync(maps_out + (size_t)j * n_iter, host_maps.data() + (size_t)j * n_iter,
                                     sizeof(double) * n_iter, cudaMemcpyHostToDevice, st));
        copied = true;
      }
    if (copied) SGC_CUDA_TRY(cudaStreamSynchronize(st));  // host_maps is released on return
    SGC_CUDA_TRY(cudaGetLastError());
    return SGC_OK;
  }
  {
    SGC_TRACE_SCOPE("count.wait");
    SGC_CUDA_TRY(cudaStreamSynchronize(st));
  }
  SGC_CUDA_TRY(cudaGetLastError());
  if (maps_out) std::memcpy(maps_out, host_maps.data(), sizeof(double) * total);
  if (estimates)
    for (int32_t j = 0; j < n_t; ++j) {
      const long double scale = inverse_colorful_probability(ts[j]->k, o.colors);
      long double s = 0;
      for (int32_t i = 0; i < n_iter; ++i) s += (long double)host_maps[(size_t)j * n_iter + (size_t)i];
      estimates[j] = (double)(s / (long double)n_iter / (long double)ts[j]->aut * scale);
    }
  return SGC_OK;
}

}  // namespace
}  // namespace sgc

using namespace sgc;

extern "C" {

void sgc_options_init(sgc_options* opt) {
  if (!opt) return;
  opt->precision = SGC_FP32;
  opt->batch = 0;
  opt->mem_limit = 0;
  opt->stream = nullptr;
  opt->root = -1;
  opt->use_graph = 1;
  opt->autotune = 0;
  opt->spmm_shape = 0;
  opt->ema_rows = 0;
  opt->colors = 0;
  opt->unpruned = 0;
}

const char* sgc_last_error(void) { return g_last_error.c_str(); }

int32_t sgc_version(void) { return 100; }

sgc_status sgc_graph_create(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, uint32_t flags,
                            sgc_graph** out) {
  return graph_create_impl(n, nnz, row_ptr, col_idx, false, flags, nullptr, out);
}

sgc_status sgc_graph_create_device(int32_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col_idx,
                                   uint32_t flags, void* stream, sgc_graph** out) {
  return graph_create_impl(n, nnz, d_row_ptr, d_col_idx, true, flags, (cudaStream_t)stream, out);
}

sgc_status sgc_graph_stats_get(const sgc_graph* g, sgc_graph_stats* out) {
  if (!g || !out) return fail(SGC_ERR_INVALID, "NULL argument");
  out->n = g->n;
  out->n_active = g->n_act;
  out->nnz = g->nnz;
  out->max_degree = g->max_deg;
  out->n_heavy = g->n_heavy;
  out->n_segments = g->n_seg;
  out->device = g->device;
  std::lock_guard<std::mutex> lock(g->mu);
  out->kernel_launches = g->kernel_launches;
  out->ordering = g->ordering;
  return SGC_OK;
}

void sgc_graph_destroy(sgc_graph* g) { graph_destroy_impl(g); }

sgc_status sgc_template_create(int32_t k, const int32_t* parent, sgc_template** out) {
  if (!out) return fail(SGC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (k < 1 || k > SGC_MAX_K) return fail(SGC_ERR_INVALID, "k must be in [1, " + std::to_string(SGC_MAX_K) + "]");
  if (!parent) return fail(SGC_ERR_INVALID, "parent is NULL");
  int roots = 0, root = -1;
  for (int i = 0; i < k; ++i) {
    if (parent[i] == -1) {
      ++roots;
      root = i;
    } else if (parent[i] < 0 || parent[i] >= k || parent[i] == i) {
      return fail(SGC_ERR_INVALID, "parent[" + std::to_string(i) + "] is not a vertex of the template");
    }
  }
  if (roots != 1) return fail(SGC_ERR_INVALID, "parent must have exactly one root (-1)");
  static std::atomic<int64_t> next_uid{1};
  sgc_template* t = new sgc_template();
  t->uid = next_uid++;
  t->k = k;
  t->parent.assign(parent, parent + k);
  t->adj.assign(k, {});
  for (int i = 0; i < k; ++i)
    if (parent[i] >= 0) {
      t->adj[i].push_back(parent[i]);
      t->adj[parent[i]].push_back(i);
    }
  for (auto& a : t->adj) std::sort(a.begin(), a.end());
  // connected (k-1 edges + connected = tree)
  std::vector<int> seen(k, 0), stack{root};
  seen[root] = 1;
  int cnt = 1;
  while (!stack.empty()) {
    int x = stack.back();
    stack.pop_back();
    for (int y : t->adj[x])
      if (!seen[y]) {
        seen[y] = 1;
        ++cnt;
        stack.push_back(y);
      }
  }
  if (cnt != k) {
    delete t;
    return fail(SGC_ERR_INVALID, "parent array does not describe one tree (cycle or disconnected)");
  }
  t->aut = automorphisms(t);
  *out = t;
  return SGC_OK;
}

sgc_status sgc_template_automorphisms(const sgc_template* t, uint64_t* aut) {
  if (!t || !aut) return fail(SGC_ERR_INVALID, "NULL argument");
  *aut = t->aut;
  return SGC_OK;
}

void sgc_template_destroy(sgc_template* t) {
  if (!t) return;
  for (auto& kv : t->tab_cache) {
    cudaSetDevice((int)kv.first[0]);
    cudaFree(kv.second);
  }
  delete t;
}

sgc_status sgc_plan_get(const sgc_graph* g, const sgc_template* t, const sgc_options* opt, sgc_plan_info* out) {
  sgc_status rc = check_handles(g, t);
  if (rc != SGC_OK) return rc;
  if (!out) return fail(SGC_ERR_INVALID, "out is NULL");
  const sgc_options o = resolve(opt);
  if (o.root >= t->k || o.root < -1) return fail(SGC_ERR_INVALID, "options.root out of range");
  Plan p;
  const int b = pow2_floor(std::max(1, std::min(32, o.batch > 0 ? o.batch : 1)));
  if ((rc = make_plan(g, t, o.precision, o.root, -1, b, false, &p, nullptr,
                      o.colors, o.unpruned)) != SGC_OK) return rc;
  out->root = p.root;
  out->n_tables = p.n_tables;
  out->n_spmm = p.n_spmm;
  out->n_ema = p.n_ema;
  out->batch = b;
  out->workspace_bytes = p.ws_bytes;
  out->est_bytes = p.est_bytes;
  out->est_spmm_bytes = p.est_spmm_bytes;
  out->est_fma = p.est_fma;
  return SGC_OK;
}

sgc_status sgc_count(const sgc_graph* g, const sgc_template* t, const uint64_t* seeds, int32_t n_iter,
                     const sgc_options* opt, double* estimate, double* colorful_maps) {
  if (!t) return fail(SGC_ERR_INVALID, "template is NULL");
  return count_core(g, 1, &t, seeds, n_iter, opt, false, estimate, colorful_maps);
}

sgc_status sgc_count_device(const sgc_graph* g, const sgc_template* t, const uint64_t* d_seeds, int32_t n_iter,
                            const sgc_options* opt, double* d_colorful_maps) {
  if (!t) return fail(SGC_ERR_INVALID, "template is NULL");
  return count_core(g, 1, &t, d_seeds, n_iter, opt, true, nullptr, d_colorful_maps);
}

sgc_status sgc_count_many(const sgc_graph* g, int32_t n_templates, const sgc_template* const* templates,
                          const uint64_t* seeds, int32_t n_iter, const sgc_options* opt, double* estimates,
                          double* colorful_maps) {
  return count_core(g, n_templates, templates, seeds, n_iter, opt, false, estimates, colorful_maps);
}

int64_t sgc_iterations_bound(int32_t k, double eps, double delta) {
  if (k < 1 || k > SGC_MAX_K || !(eps > 0) || !(delta > 0) || !(delta < 1)) return -1;
  const long double x = std::exp((long double)k) * std::log(1.0L / (long double)delta) / ((long double)eps * eps);
  if (!(x < 9.0e18L)) return INT64_MAX;
  return (int64_t)std::ceil(x);
}

sgc_status sgc_estimate(const sgc_graph* g, const sgc_template* t, double eps, double delta, uint64_t first_seed,
                        int64_t min_iter, int64_t max_iter, const sgc_options* opt, double* estimate,
                        int64_t* n_used, double* rel_half_width) {
  sgc_status rc = check_handles(g, t);
  if (rc != SGC_OK) return rc;
  if (!estimate || !n_used) return fail(SGC_ERR_INVALID, "NULL argument");
  if (!(eps > 0) || !(delta > 0) || !(delta < 1)) return fail(SGC_ERR_INVALID, "need eps > 0 and 0 < delta < 1");
  if (min_iter < 0 || max_iter < 0) return fail(SGC_ERR_INVALID, "min_iter and max_iter must be >= 0");
  const sgc_options o = resolve(opt);
  const int64_t cap = max_iter > 0 ? max_iter : sgc_iterations_bound(t->k, eps, delta);
  const int64_t chunk = o.batch > 0 ? o.batch : 32;
  // z with P(|Z| > z) = delta for a standard normal Z: erfc(z / sqrt 2) = delta, by bisection
  long double lo = 0.0L, hi = 40.0L;
  for (int i = 0; i < 200; ++i) {
    const long double mid = 0.5L * (lo + hi);
    if (std::erfc(mid / std::sqrt(2.0L)) > (long double)delta) lo = mid; else hi = mid;
  }
  const long double z = 0.5L * (lo + hi);
  if (o.colors != 0 && (o.colors < t->k || o.colors > SGC_MAX_K))
    return fail(SGC_ERR_INVALID, "options.colors must be 0 or in [|T|, " + std::to_string(SGC_MAX_K) + "]");
  const long double scale = inverse_colorful_probability(t->k, o.colors) / (long double)t->aut;
  long double sum = 0.0L, sum2 = 0.0L, half = 0.0L;
  int64_t n = 0;
  std::vector<uint64_t> seeds;
  std::vector<double> maps;
  while (n < cap) {
    const int64_t m = std::min<int64_t>(chunk, cap - n);
    seeds.resize((size_t)m);
    maps.resize((size_t)m);
    for (int64_t i = 0; i < m; ++i) seeds[(size_t)i] = first_seed + (uint64_t)(n + i);
    if ((rc = count_core(g, 1, &t, seeds.data(), (int32_t)m, &o, false, nullptr, maps.data())) != SGC_OK) return rc;
    for (double x : maps) {
      const long double e = (long double)x * scale;
      sum += e;
      sum2 += e * e;
    }
    n += m;
    const long double mean = sum / n;
    const long double var = n > 1 ? std::max(0.0L, (sum2 - sum * mean) / (n - 1)) : 0.0L;
    half = z * std::sqrt(var / n);
    if (n >= min_iter && n > 1 && half <= (long double)eps * mean) break;
  }
  const long double mean = n > 0 ? sum / n : 0.0L;
  *estimate = (double)mean;
  *n_used = n;
  if (rel_half_width) *rel_half_width = mean > 0 ? (double)(half / mean) : 0.0;
  return SGC_OK;
}

sgc_status sgc_autotune(const sgc_graph* g, const sgc_template* t, const sgc_options* opt, sgc_tune_entry* out,
                        int32_t cap, int32_t* n) {
  sgc_status rc = check_handles(g, t);
  if (rc != SGC_OK) return rc;
  if (!n || (cap > 0 && !out)) return fail(SGC_ERR_INVALID, "NULL argument");
  sgc_options o = resolve(opt);
  o.autotune = 1;
  if (o.precision != SGC_FP32 && o.precision != SGC_FP64) return fail(SGC_ERR_INVALID, "unknown precision");
  if (o.root >= t->k || o.root < -1) return fail(SGC_ERR_INVALID, "options.root out of range");
  *n = 0;
  if (t->k == 1) return SGC_OK;
  SGC_CUDA_TRY(cudaSetDevice(g->device));
  std::lock_guard<std::mutex> lock(g->mu);
  if (g->n_act == 0) return SGC_OK;
  DevicePool& pool = device_pool(g->device);
  std::lock_guard<std::mutex> pool_lock(pool.mu);
  cudaStream_t st = o.stream ? (cudaStream_t)o.stream : g->stream;
  size_t free_b = 0, total_b = 0;
  SGC_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const int64_t mem_limit = o.mem_limit > 0 ? o.mem_limit : (int64_t)((free_b + pool.bytes) * 0.9);
  const int bmax = pow2_floor(std::min(32, o.batch > 0 ? o.batch : 32));
  std::shared_ptr<PlanSet> plans;
  if ((rc = plan_batches(g, t, o, bmax, mem_limit, &plans)) != SGC_OK) return rc;
  if (!plans->tuned) {
    if (pool.last) SGC_CUDA_TRY(cudaEventSynchronize(pool.last));
    if ((rc = tune_plans(g, t, o, plans.get(), pool, st)) != SGC_OK) return rc;
  }
  *n = (int32_t)plans->report.size();
  for (int32_t i = 0; i < *n && i < cap; ++i) out[i] = plans->report[(size_t)i];
  return SGC_OK;
}

sgc_status sgc_estimate_from_maps(const sgc_template* t, int32_t colors, const double* maps, int64_t n,
                                  double* estimate) {
  if (!t || !estimate || (n > 0 && !maps)) return fail(SGC_ERR_INVALID, "NULL argument");
  if (n < 0) return fail(SGC_ERR_INVALID, "n must be >= 0");
  if (colors != 0 && (colors < t->k || colors > SGC_MAX_K))
    return fail(SGC_ERR_INVALID, "colors must be 0 or in [|T|, " + std::to_string(SGC_MAX_K) + "]");
  if (n == 0) {
    *estimate = 0.0;
    return SGC_OK;
  }
  long double s = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(maps[i] >= 0.0)) return fail(SGC_ERR_INVALID, "colorful maps must be non-negative numbers");
    s += (long double)maps[i];
  }
  *estimate = (double)(s / (long double)n / (long double)t->aut * inverse_colorful_probability(t->k, colors));
  return SGC_OK;
}

sgc_status sgc_profile_enable(const sgc_graph* g, int32_t on) {
  if (!g) return fail(SGC_ERR_INVALID, "graph is NULL");
  std::lock_guard<std::mutex> lock(g->mu);
  cudaSetDevice(g->device);
  for (auto& pe : g->prof.pending) {
    cudaEventSynchronize(pe.e1);
    cudaEventDestroy(pe.e0);
    cudaEventDestroy(pe.e1);
  }
  g->prof.pending.clear();
  g->prof.agg.clear();
  g->prof.on = on != 0;
  return SGC_OK;
}

sgc_status sgc_profile_read(const sgc_graph* g, sgc_op_profile* out, int32_t cap, int32_t* n) {
  if (!g || !n || (cap > 0 && !out)) return fail(SGC_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(g->mu);
  SGC_CUDA_TRY(cudaSetDevice(g->device));
  for (auto& pe : g->prof.pending) {
    SGC_CUDA_TRY(cudaEventSynchronize(pe.e1));
    float ms = 0.f;
    SGC_CUDA_TRY(cudaEventElapsedTime(&ms, pe.e0, pe.e1));
    g->prof.agg[pe.slot].ms += ms;
    cudaEventDestroy(pe.e0);
    cudaEventDestroy(pe.e1);
  }
  g->prof.pending.clear();
  *n = (int32_t)g->prof.agg.size();
  for (int32_t i = 0; i < *n && i < cap; ++i) {
    const OpProfile& a = g->prof.agg[i];
    out[i].kind = a.kind;
    out[i].t = a.t;
    out[i].a = a.a;
    out[i].p = a.p;
    out[i].batch = a.batch;
    out[i].passes = a.launches;
    out[i].kernels = a.kernels;
    out[i].ms = a.ms;
    out[i].bytes = a.bytes;
    out[i].flops = a.flops;
    out[i].gather_bytes = a.gather;
    out[i].k = a.k;
  }
  g->prof.agg.clear();
  return SGC_OK;
}

}  // extern "C"
