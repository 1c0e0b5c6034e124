// api.cpp - the C ABI of libsgc (include/sgc.h): argument checks, handles,
// and the host-side driver of sgc_count (batching colorings, workspace,
// result read-back and the k^k/k! estimator of Section 2.1).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "sgc_internal.h"

namespace sgc {

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
sgc_status plan_batches(const sgc_graph* g, const sgc_template* t, const sgc_options& o, int bmax, int64_t mem_limit,
                        std::shared_ptr<PlanSet>* out) {
  const std::string key = std::to_string(t->uid) + "/" + std::to_string(o.precision) + "/" + std::to_string(o.root) +
                          "/" + std::to_string(bmax);
  for (auto& kv : g->plan_cache)
    if (kv.first == key && kv.second->by_batch.at(kv.second->bfit).ws_bytes <= mem_limit) {
      *out = kv.second;
      return SGC_OK;
    }
  auto set = std::make_shared<PlanSet>();
  Plan p1;
  sgc_status rc = make_plan(g, t, o.precision, o.root, -1, 1, true, &p1);
  if (rc != SGC_OK) return rc;
  if (p1.ws_bytes > mem_limit)
    return fail(SGC_ERR_OOM, "one coloring needs " + std::to_string(p1.ws_bytes) + " bytes of device workspace, limit " +
                                 std::to_string(mem_limit));
  const int root = p1.root, policy = p1.policy;
  // Occupancy cap: a SpMM warp keeps a whole output row of `batch` colorings in
  // shared memory, so wide rows take fewer colorings per pass (at most ~8 KB
  // per warp keeps several blocks resident per SM).
  int64_t widest = 0;
  for (const PlanOp& op : p1.ops)
    if (op.kind == OP_SPMM) widest = std::max<int64_t>(widest, op.ld_out * p1.elem);
  while (bmax > 1 && widest * bmax > kSpmmRowBytesPerWarp) bmax /= 2;
  set->by_batch[1] = std::move(p1);
  set->bfit = 1;
  for (int b = 2; b <= bmax; b *= 2) {
    Plan pb;
    rc = make_plan(g, t, o.precision, root, policy, b, true, &pb);
    if (rc != SGC_OK) return rc;
    if (pb.ws_bytes > mem_limit) break;
    set->by_batch[b] = std::move(pb);
    set->bfit = b;
  }
  for (auto& kv : g->plan_cache)
    if (kv.first == key) {
      kv.second = set;
      *out = set;
      return SGC_OK;
    }
  if (g->plan_cache.size() >= 64) g->plan_cache.erase(g->plan_cache.begin());
  g->plan_cache.push_back({key, set});
  *out = set;
  return SGC_OK;
}

namespace {

sgc_status count_impl(const sgc_graph* g, const sgc_template* t, const uint64_t* seeds, int32_t n_iter,
                      const sgc_options* opt_in, bool device_io, double* estimate, double* maps_out) {
  sgc_status rc = check_handles(g, t);
  if (rc != SGC_OK) return rc;
  if (n_iter < 0) return fail(SGC_ERR_INVALID, "n_iter must be >= 0");
  if (n_iter > 0 && !seeds) return fail(SGC_ERR_INVALID, "seeds is NULL");
  if (device_io && n_iter > 0 && !maps_out) return fail(SGC_ERR_INVALID, "colorful_maps is NULL");
  const sgc_options o = resolve(opt_in);
  if (o.precision != SGC_FP32 && o.precision != SGC_FP64) return fail(SGC_ERR_INVALID, "unknown precision");
  if (o.root >= t->k || o.root < -1) return fail(SGC_ERR_INVALID, "options.root out of range");
  if (o.batch < 0) return fail(SGC_ERR_INVALID, "options.batch must be >= 0");
  SGC_CUDA_TRY(cudaSetDevice(g->device));
  std::lock_guard<std::mutex> lock(g->mu);
  DevicePool& pool = device_pool(g->device);
  std::lock_guard<std::mutex> pool_lock(pool.mu);
  cudaStream_t st = o.stream ? (cudaStream_t)o.stream : g->stream;
  const int k = t->k;
  if (estimate) *estimate = 0.0;
  if (n_iter == 0) return SGC_OK;

  std::vector<double> host_maps(device_io ? 0 : (size_t)n_iter);
  if (k == 1 || g->n_act == 0) {
    // one vertex: every vertex is a colorful map; no edges: nothing maps
    const double v = k == 1 ? (double)g->n : 0.0;
    if (device_io) {
      std::vector<double> tmp((size_t)n_iter, v);
      SGC_CUDA_TRY(cudaMemcpyAsync(maps_out, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      SGC_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
      std::fill(host_maps.begin(), host_maps.end(), v);
    }
  } else {
    size_t free_b = 0, total_b = 0;
    SGC_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const int64_t mem_limit = o.mem_limit > 0 ? o.mem_limit : (int64_t)((free_b + pool.bytes) * 0.9);
    const int bmax = pow2_floor(std::min(32, o.batch > 0 ? o.batch : std::max(1, (int)n_iter)));
    std::shared_ptr<PlanSet> plans;
    rc = plan_batches(g, t, o, bmax, mem_limit, &plans);
    if (rc != SGC_OK) return rc;
    const Plan& top = plans->by_batch.at(plans->bfit);
    // every batch size has its own plan and index tables (the SpMM form can
    // depend on the batch), each uploaded once and cached by content
    std::map<int, const uint32_t*> d_tabs_by_batch;
    for (auto& kv : plans->by_batch) {
      const uint32_t* d = nullptr;
      if ((rc = template_tables(t, kv.second, g->device, &d)) != SGC_OK) return rc;
      d_tabs_by_batch[kv.first] = d;
    }
    if ((rc = ensure_workspace(pool, top.ws_bytes)) != SGC_OK) return rc;
    if (!pool.last) SGC_CUDA_TRY(cudaEventCreateWithFlags(&pool.last, cudaEventDisableTiming));
    SGC_CUDA_TRY(cudaStreamWaitEvent(st, pool.last, 0));
    char* ws = static_cast<char*>(pool.ptr);
    Profiler* prof = g->prof.on ? &g->prof : nullptr;
    for (int32_t i = 0; i < n_iter;) {
      int b = plans->bfit;
      while (b > n_iter - i) b /= 2;
      const Plan& plan = plans->by_batch.at(b);
      char* d_seeds = ws + plan.bufs[plan.buf_seeds].offset;
      char* d_out = ws + plan.bufs[plan.buf_out].offset;
      SGC_CUDA_TRY(cudaMemcpyAsync(d_seeds, seeds + i, sizeof(uint64_t) * b,
                                   device_io ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      if ((rc = run_pass(g, plan, d_tabs_by_batch.at(b), ws, st, prof, &g->kernel_launches)) != SGC_OK) return rc;
      if (device_io) {
        SGC_CUDA_TRY(cudaMemcpyAsync(maps_out + i, d_out, sizeof(double) * b, cudaMemcpyDeviceToDevice, st));
      } else {
        SGC_CUDA_TRY(cudaMemcpyAsync(host_maps.data() + i, d_out, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
      }
      i += b;
    }
    SGC_CUDA_TRY(cudaEventRecord(pool.last, st));
    if (!device_io) SGC_CUDA_TRY(cudaStreamSynchronize(st));
    SGC_CUDA_TRY(cudaGetLastError());
  }
  if (!device_io) {
    if (maps_out) std::memcpy(maps_out, host_maps.data(), sizeof(double) * (size_t)n_iter);
    if (estimate) {
      long double scale = 1.0L;
      for (int i = 1; i <= k; ++i) scale *= (long double)k / (long double)i;  // k^k / k!
      long double s = 0;
      for (double m : host_maps) s += (long double)m;
      *estimate = (double)(s / (long double)n_iter / (long double)t->aut * scale);
    }
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
  if ((rc = make_plan(g, t, o.precision, o.root, -1, b, false, &p)) != SGC_OK) return rc;
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
  return count_impl(g, t, seeds, n_iter, opt, false, estimate, colorful_maps);
}

sgc_status sgc_count_device(const sgc_graph* g, const sgc_template* t, const uint64_t* d_seeds, int32_t n_iter,
                            const sgc_options* opt, double* d_colorful_maps) {
  return count_impl(g, t, d_seeds, n_iter, opt, true, nullptr, d_colorful_maps);
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
  }
  g->prof.agg.clear();
  return SGC_OK;
}

}  // extern "C"
