// noalloc.cu - sgc_count_device_static: counting with no device allocation.
//
// Some callers cannot call cudaMalloc while they count: code running inside
// a framework that owns all device memory through its own allocator, or a
// service that must not change its device-memory footprint (or risk an
// allocation failure) after start-up.  This entry point serves them for
// small problems.  All scratch of one call - count tables, SpMM partial rows,
// block partials, colorings, seeds, results and the plan's index tables -
// lives in one file-scope device array of kStaticWorkspaceBytes, so every GPU
// that loads this module holds that array until the process exits.  The
// graph and template handles are created beforehand (that allocates, once);
// the call itself allocates nothing.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress (host code cannot use the
// array's name as a device pointer) and keeps it for later calls; make that
// first call before any stream capture.  Every call shares the array, which
// keeps the last call's contents: the pass clears what must start at zero
// (scale states, heavy-row histograms) itself.  Calls that overlap on the GPU
// - on different streams, or from different threads - race on the array.
#include <algorithm>
#include <mutex>
#include <string>

#include "sgc_internal.h"

namespace sgc {
namespace {

constexpr size_t kStaticWorkspaceBytes = (size_t)SGC_STATIC_WORKSPACE_BYTES;

static __device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

std::mutex g_static_mu;
void* g_static_ptr[64] = {};

// device address of the array on the current device (looked up once per device)
sgc_status static_workspace(int device, char** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (device < 0 || device >= 64) return fail(SGC_ERR_UNSUPPORTED, "device ordinal above 63");
  if (!g_static_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_workspace);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static workspace)");
    g_static_ptr[device] = p;
  }
  *out = static_cast<char*>(g_static_ptr[device]);
  return SGC_OK;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// bytes of the array one pass of `plan` needs: workspace, then index tables
int64_t static_need(const Plan& plan) {
  return round_up(plan.ws_bytes, 256) + (int64_t)plan.tabs.size() * (int64_t)sizeof(uint32_t);
}

}  // namespace
}  // namespace sgc

using namespace sgc;

extern "C" sgc_status sgc_count_device_static(const sgc_graph* g, const sgc_template* t, const uint64_t* d_seeds,
                                              int32_t n_iter, const sgc_options* opt, double* d_colorful_maps) {
  if (!g) return fail(SGC_ERR_INVALID, "graph is NULL");
  if (!t) return fail(SGC_ERR_INVALID, "template is NULL");
  if (n_iter < 0) return fail(SGC_ERR_INVALID, "n_iter must be >= 0");
  if (n_iter > 0 && (!d_seeds || !d_colorful_maps)) return fail(SGC_ERR_INVALID, "seeds or colorful_maps is NULL");
  sgc_options o;
  sgc_options_init(&o);
  if (opt) o = *opt;
  if (o.precision != SGC_FP32 && o.precision != SGC_FP64) return fail(SGC_ERR_INVALID, "unknown precision");
  if (o.root >= t->k || o.root < -1) return fail(SGC_ERR_INVALID, "options.root out of range");
  if (o.batch < 0) return fail(SGC_ERR_INVALID, "options.batch must be >= 0");
  if (n_iter == 0) return SGC_OK;
  SGC_CUDA_TRY(cudaSetDevice(g->device));
  std::lock_guard<std::mutex> lock(g->mu);
  cudaStream_t st = o.stream ? (cudaStream_t)o.stream : g->stream;
  char* base = nullptr;
  sgc_status rc = static_workspace(g->device, &base);
  if (rc != SGC_OK) return rc;
  if (t->k == 1 || g->n_act == 0) {
    // no pass needed: every vertex is a map (k = 1) or nothing maps (no edges)
    const double v = t->k == 1 ? (double)g->n : 0.0;
    for (int32_t i = 0; i < n_iter; ++i)
      SGC_CUDA_TRY(cudaMemcpyAsync(d_colorful_maps + i, &v, sizeof(double), cudaMemcpyHostToDevice, st));
    SGC_CUDA_TRY(cudaStreamSynchronize(st));
    return SGC_OK;
  }
  // largest power-of-two batch (<= 32, <= n_iter or options.batch) whose pass fits
  int bmax = 1;
  const int want = std::min(32, o.batch > 0 ? o.batch : (int)n_iter);
  while (bmax * 2 <= want) bmax *= 2;
  Plan top;
  rc = make_plan(g, t, o.precision, o.root, -1, 1, true, &top, nullptr, o.colors, o.unpruned);
  if (rc != SGC_OK) return rc;
  if (static_need(top) > (int64_t)kStaticWorkspaceBytes)
    return fail(SGC_ERR_UNSUPPORTED, "this count needs " + std::to_string(static_need(top)) +
                                         " bytes of scratch for one coloring; the static workspace holds " +
                                         std::to_string(kStaticWorkspaceBytes) + " bytes (use sgc_count_device)");
  const int root = top.root, policy = top.policy;
  // the index tables depend on the batch (some SpMM forms key them by it), so each candidate
  // batch is sized with its own tables
  int bfit = 1;
  for (int b = 2; b <= bmax; b *= 2) {
    Plan pb;
    if ((rc = make_plan(g, t, o.precision, root, policy, b, true, &pb, nullptr,
                        o.colors, o.unpruned)) != SGC_OK) return rc;
    if (static_need(pb) > (int64_t)kStaticWorkspaceBytes) break;
    bfit = b;
  }
  for (int32_t i = 0; i < n_iter;) {
    int b = bfit;
    while (b > n_iter - i) b /= 2;
    Plan plan;
    for (;;) {
      if ((rc = make_plan(g, t, o.precision, root, policy, b, true, &plan, nullptr,
                          o.colors, o.unpruned)) != SGC_OK) return rc;
      if (static_need(plan) <= (int64_t)kStaticWorkspaceBytes) break;
      if (b == 1) return fail(SGC_ERR_INTERNAL, "static workspace plan grew beyond its size");
      b /= 2;  // a smaller pass needs less
    }
    char* ws = base;
    uint32_t* d_tabs = reinterpret_cast<uint32_t*>(base + round_up(plan.ws_bytes, 256));
    if (!plan.tabs.empty())
      SGC_CUDA_TRY(cudaMemcpyAsync(d_tabs, plan.tabs.data(), plan.tabs.size() * sizeof(uint32_t),
                                   cudaMemcpyHostToDevice, st));
    SGC_CUDA_TRY(cudaMemcpyAsync(ws + plan.bufs[plan.buf_seeds].offset, d_seeds + i, sizeof(uint64_t) * b,
                                 cudaMemcpyDeviceToDevice, st));
    if ((rc = run_pass(g, plan, d_tabs, ws, st, nullptr, &g->kernel_launches)) != SGC_OK) return rc;
    SGC_CUDA_TRY(cudaMemcpyAsync(d_colorful_maps + i, ws + plan.bufs[plan.buf_out].offset, sizeof(double) * b,
                                 cudaMemcpyDeviceToDevice, st));
    // the next pass rewrites the tables and the workspace: wait for this one
    // (the host copy source above must also stay valid until it is read)
    SGC_CUDA_TRY(cudaStreamSynchronize(st));
    i += b;
  }
  return SGC_OK;
}
