// graph.cu - graph handles: CSR validation on the device, removal of
// isolated vertices, renumbering by degree (highest first) and the
// neighbour-list segmentation of heavy rows used by SpMM and the histogram.
//
// The adjacency is the matrix A_G of Section 4.3 in CSR form.  Renumbering
// does not change any count (counts are invariant under relabelling), and an
// isolated vertex is in no embedding of a template with two or more vertices,
// so count tables only hold rows for vertices of degree >= 1.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "sgc_internal.h"

namespace sgc {
namespace {

enum : int32_t {
  BAD_ROWPTR = 1,
  BAD_COL = 2,
  SELF_LOOP = 4,
  UNSORTED = 8,
  ASYMMETRIC = 16,
};

// row_ptr must be non-decreasing and inside [0, nnz]
__global__ void k_check_rowptr(const int32_t* __restrict__ rp, int32_t n, int64_t nnz, int32_t* flags) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = rp[v], b = rp[v + 1];
    if (a < 0 || b < a || b > nnz) atomicOr(flags, BAD_ROWPTR);
  }
}

// One warp per row: range, self-loop, strictly ascending, and symmetry.
// Symmetry is checked from one side of each entry only: with key(x) =
// (deg x, x), an entry (v, u) with key(u) < key(v) is "searched" (v must be
// found, by binary search, in the shorter row u); otherwise it is "skipped".
// If every searched entry is found, mirroring maps searched entries one-to-one
// onto skipped ones (rows have no duplicates), so the adjacency is symmetric
// exactly when, in addition, both kinds are equally many (counts[0] ==
// counts[1], compared on the host).  The searches run in the shorter row of
// each pair, so hub rows are never searched from their many light neighbours.
//
// Rows longer than kWideRow are left to k_check_cols_wide (a block per row),
// so no warp walks a hub's whole neighbour list alone.
constexpr int32_t kWideRow = 2048;

__device__ __forceinline__ int32_t check_entry(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                               int32_t n, int64_t v, int32_t lo, int32_t dv, int32_t e,
                                               unsigned long long* searched, unsigned long long* skipped) {
  const int32_t u = ci[e];
  if (u < 0 || u >= n) return BAD_COL;
  int32_t f = 0;
  if (u == v) f |= SELF_LOOP;
  if (e > lo && ci[e - 1] >= u) f |= UNSORTED;
  int32_t a = rp[u], b = rp[u + 1] - 1;
  const int32_t du = b + 1 - a;
  if (du > dv || (du == dv && u >= v)) {
    ++*skipped;
    return f;
  }
  ++*searched;
  bool found = false;
  int guard = 0;
  while (a <= b && guard < 40) {
    const int32_t mid = a + ((b - a) >> 1);
    const int32_t x = ci[mid];
    if (x == v) { found = true; break; }
    if (x < v) a = mid + 1; else b = mid - 1;
    ++guard;
  }
  return found ? f : (f | ASYMMETRIC);
}

__device__ __forceinline__ void add_counts(unsigned long long* counts, unsigned long long searched,
                                           unsigned long long skipped) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    searched += __shfl_xor_sync(0xffffffffu, searched, o);
    skipped += __shfl_xor_sync(0xffffffffu, skipped, o);
  }
  if ((threadIdx.x & 31) == 0 && (searched | skipped)) {
    atomicAdd(counts, searched);
    atomicAdd(counts + 1, skipped);
  }
}

__global__ void k_check_cols_wide(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                  const int32_t* __restrict__ wide, int32_t n_wide, int32_t* flags,
                                  unsigned long long* counts) {
  unsigned long long searched = 0, skipped = 0;
  for (int32_t w = blockIdx.x; w < n_wide; w += gridDim.x) {
    const int64_t v = wide[w];
    const int32_t lo = rp[v], hi = rp[v + 1];
    int32_t f = 0;
    for (int32_t e = lo + threadIdx.x; e < hi; e += blockDim.x)
      f |= check_entry(rp, ci, n, v, lo, hi - lo, e, &searched, &skipped);
    if (f) atomicOr(flags, f);
  }
  add_counts(counts, searched, skipped);
}

__global__ void k_check_cols(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                             int32_t* flags, unsigned long long* counts) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long searched = 0, skipped = 0;
  for (int64_t v = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += nw) {
    const int32_t lo = rp[v], hi = rp[v + 1];
    const int32_t dv = hi - lo;
    if (dv > kWideRow) continue;
    int32_t f = 0;
    for (int32_t e = lo + lane; e < hi; e += 32) f |= check_entry(rp, ci, n, v, lo, dv, e, &searched, &skipped);
    if (f) atomicOr(flags, f);
  }
  add_counts(counts, searched, skipped);  // one pair of atomics per warp
}

// new row v copies old row orig[v] with neighbours renamed through inv.
// Column indices are range-checked here whatever the validation flags, so a
// malformed CSR is reported instead of read out of bounds later; an entry
// pointing at an isolated vertex (possible only without symmetry) is
// reported the same way.
//
// The first n_wide new rows (the longest, degree order) get a block each; the
// rest a warp each.
__device__ __forceinline__ void relabel_entry(const int32_t* __restrict__ old_ci, int32_t n,
                                              const int32_t* __restrict__ inv, int64_t src, int64_t dst,
                                              int32_t* __restrict__ new_ci, int32_t* flags) {
  const int32_t u = old_ci[src];
  int32_t w = 0;
  if (u < 0 || u >= n) {
    atomicOr(flags, BAD_COL);
  } else {
    w = inv[u];
    if (w < 0) { atomicOr(flags, ASYMMETRIC); w = 0; }
  }
  new_ci[dst] = w;
}

__global__ void k_relabel(const int32_t* __restrict__ old_rp, const int32_t* __restrict__ old_ci, int32_t n,
                          const int32_t* __restrict__ orig, const int32_t* __restrict__ inv,
                          const int32_t* __restrict__ new_rp, int32_t n_act, int32_t n_wide,
                          int32_t* __restrict__ new_ci, int32_t* flags) {
  if ((int32_t)blockIdx.x < n_wide) {  // one long row per block
    const int32_t v = blockIdx.x;
    const int32_t o = orig[v];
    const int32_t lo = old_rp[o], deg = old_rp[o + 1] - lo, dst = new_rp[v];
    for (int32_t j = threadIdx.x; j < deg; j += blockDim.x)
      relabel_entry(old_ci, n, inv, lo + j, dst + j, new_ci, flags);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)(gridDim.x - n_wide) * (blockDim.x >> 5);
  for (int64_t v = n_wide + (blockIdx.x - n_wide) * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n_act;
       v += nw) {
    const int32_t o = orig[v];
    const int32_t lo = old_rp[o], deg = old_rp[o + 1] - lo, dst = new_rp[v];
    for (int32_t j = lane; j < deg; j += 32) relabel_entry(old_ci, n, inv, lo + j, dst + j, new_ci, flags);
  }
}

int default_seg_len() {
  const char* s = std::getenv("SGC_SEG_LEN");
  if (s) {
    int v = std::atoi(s);
    if (v >= 32 && v <= (1 << 20)) return v;
  }
  return 256;
}

template <typename T>
void free_dev(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void destroy_graph(sgc_graph* g) {
  if (!g) return;
  free_dev(g->d_row_ptr);
  free_dev(g->d_col_idx);
  free_dev(g->d_orig);
  free_dev(g->d_seg_row);
  free_dev(g->d_seg_lo);
  free_dev(g->d_seg_hi);
  free_dev(g->d_heavy_seg);
  for (auto& pe : g->prof.pending) {
    cudaEventDestroy(pe.e0);
    cudaEventDestroy(pe.e1);
  }
  for (auto& x : g->exec_cache)
    if (x.exec) cudaGraphExecDestroy(x.exec);
  for (cudaStream_t s : g->lanes) cudaStreamDestroy(s);
  for (cudaEvent_t e : g->lane_events) cudaEventDestroy(e);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

template <typename T>
sgc_status upload(T** dst, const std::vector<T>& src, cudaStream_t st) {
  const size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
  cudaError_t e = cudaMalloc(dst, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(graph)");
  if (!src.empty()) {
    e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(graph)");
  }
  return SGC_OK;
}

// key[v] = maxd - degree (highest degree first; degree 0 last), vid[v] = v
__global__ void k_degree_keys(const int32_t* __restrict__ rp, int32_t n, int32_t maxd, uint32_t* __restrict__ key,
                              int32_t* __restrict__ vid) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    key[v] = (uint32_t)(maxd - (rp[v + 1] - rp[v]));
    vid[v] = (int32_t)v;
  }
}

// for the first n_act vertices of the new order: inv[orig[i]] = i and deg[i] = degree of orig[i]
__global__ void k_order_maps(const int32_t* __restrict__ orig, const int32_t* __restrict__ rp, int32_t n_act,
                             int32_t* __restrict__ inv, int32_t* __restrict__ deg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_act;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = orig[i];
    inv[v] = (int32_t)i;
    deg[i] = rp[v + 1] - rp[v];
  }
}

// Reverse Cuthill-McKee order of the rows of degree 1..thr (Section 4.3 names
// RCM as the locality pre-processing of the adjacency matrix), after the rows
// of degree > thr in degree order (highest first, ties by id) and before the
// isolated vertices (by id).  Breadth-first search over the light rows only:
// each component starts at its unvisited row of lowest degree (ties by id),
// a row's unvisited light neighbours are queued by increasing degree (ties by
// id), and the whole light sequence is then reversed.  Neighbours of the
// heavy rows are not expanded through them, so a hub does not pull its
// thousands of otherwise unrelated neighbours together.  Column indices
// outside [0, n) are skipped here (validation or relabelling reports them).
void rcm_order(int32_t n, const std::vector<int32_t>& rp, const int32_t* ci, int32_t thr,
               std::vector<int32_t>* orig) {
  orig->clear();
  orig->reserve((size_t)n);
  std::vector<int32_t> deg((size_t)n);
  int32_t maxd = 0;
  for (int32_t v = 0; v < n; ++v) {
    deg[(size_t)v] = rp[(size_t)v + 1] - rp[(size_t)v];
    maxd = std::max(maxd, deg[(size_t)v]);
  }
  // counting sort by degree: descending for the heavy prefix, ascending for the start list
  std::vector<int64_t> cnt((size_t)maxd + 2, 0);
  for (int32_t v = 0; v < n; ++v) ++cnt[(size_t)deg[(size_t)v] + 1];
  for (size_t d = 1; d < cnt.size(); ++d) cnt[d] += cnt[d - 1];
  std::vector<int32_t> by_deg((size_t)n);  // ascending degree, ties by id
  for (int32_t v = 0; v < n; ++v) by_deg[(size_t)cnt[(size_t)deg[(size_t)v]]++] = v;
  for (int32_t d = maxd; d > thr; --d) {
    // the vertices of degree d sit in by_deg[start of d .. end of d) in id order
    const int64_t hi = cnt[(size_t)d], lo = d > 0 ? cnt[(size_t)d - 1] : 0;
    for (int64_t i = lo; i < hi; ++i) orig->push_back(by_deg[(size_t)i]);
  }
  std::vector<uint8_t> seen((size_t)n, 0);
  for (int32_t v = 0; v < n; ++v) seen[(size_t)v] = deg[(size_t)v] == 0 || deg[(size_t)v] > thr;
  const size_t light0 = orig->size();
  std::vector<std::pair<int32_t, int32_t>> nb;
  for (int32_t s : by_deg) {
    if (seen[(size_t)s]) continue;
    seen[(size_t)s] = 1;
    size_t head = orig->size();
    orig->push_back(s);
    while (head < orig->size()) {
      const int32_t x = (*orig)[head++];
      nb.clear();
      for (int32_t e = rp[(size_t)x]; e < rp[(size_t)x + 1]; ++e) {
        const int32_t w = ci[e];
        if (w < 0 || w >= n || seen[(size_t)w]) continue;
        seen[(size_t)w] = 1;
        nb.emplace_back(deg[(size_t)w], w);
      }
      std::sort(nb.begin(), nb.end());
      for (const auto& dw : nb) orig->push_back(dw.second);
    }
  }
  std::reverse(orig->begin() + (std::ptrdiff_t)light0, orig->end());
  for (int32_t v = 0; v < n; ++v)
    if (deg[(size_t)v] == 0) orig->push_back(v);
}

// Build the handle from device CSR (d_rp, d_ci) and the host copy of row_ptr.
sgc_status build_graph(int32_t n, int64_t nnz, const int32_t* d_rp, const int32_t* d_ci,
                       const std::vector<int32_t>& h_rp, const int32_t* h_ci, uint32_t flags, cudaStream_t st,
                       sgc_graph* g) {
  int dev = 0, sms = 0;
  SGC_CUDA_TRY(cudaGetDevice(&dev));
  SGC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  g->device = dev;
  g->num_sms = sms;
  SGC_CUDA_TRY(cudaDeviceGetAttribute(&g->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  g->n = n;
  g->nnz = nnz;
  // row_ptr is always checked (host side): everything below indexes with it
  if (h_rp[0] != 0 || (int64_t)h_rp[n] != nnz)
    return fail(SGC_ERR_INVALID, "row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
  for (int32_t v = 0; v < n; ++v)
    if (h_rp[v + 1] < h_rp[v]) return fail(SGC_ERR_INVALID, "row_ptr must be non-decreasing");
  if (flags & SGC_GRAPH_VALIDATE) {
    SGC_TRACE_SCOPE("graph.validate");
    if (nnz % 2 != 0) return fail(SGC_ERR_INVALID, "an undirected simple graph has an even nnz");
    // flags word, then the searched / skipped entry counts of the symmetry check
    int32_t* d_flags = nullptr;
    SGC_CUDA_TRY(cudaMalloc(&d_flags, 3 * sizeof(unsigned long long)));
    unsigned long long* d_counts = reinterpret_cast<unsigned long long*>(d_flags) + 1;
    int32_t h_flags = 0;
    unsigned long long h_counts[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(d_flags, 0, 3 * sizeof(unsigned long long), st);
    // rows longer than kWideRow, checked a block per row
    std::vector<int32_t> wide;
    for (int32_t v = 0; v < n; ++v)
      if (h_rp[v + 1] - h_rp[v] > kWideRow) wide.push_back(v);
    int32_t* d_wide = nullptr;
    if (e == cudaSuccess && !wide.empty()) {
      e = cudaMalloc(&d_wide, wide.size() * sizeof(int32_t));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_wide, wide.data(), wide.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && n > 0) {
      k_check_rowptr<<<std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(d_rp, n, nnz, d_flags);
      k_check_cols<<<std::min<int64_t>((n + 7) / 8, 65536), 256, 0, st>>>(d_rp, d_ci, n, d_flags, d_counts);
      if (!wide.empty())
        k_check_cols_wide<<<std::min<int64_t>((int64_t)wide.size(), 65536), 256, 0, st>>>(
            d_rp, d_ci, n, d_wide, (int32_t)wide.size(), d_flags, d_counts);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_flags, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_counts, d_counts, sizeof(h_counts), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_flags);
    if (d_wide) cudaFree(d_wide);
    if (e != cudaSuccess) return cuda_fail(e, "graph validation");
    if (!(h_flags & (BAD_ROWPTR | BAD_COL)) && h_counts[0] != h_counts[1]) h_flags |= ASYMMETRIC;
    if (h_flags) {
      std::string why;
      if (h_flags & BAD_ROWPTR) why += " row_ptr out of range;";
      if (h_flags & BAD_COL) why += " column index out of range;";
      if (h_flags & SELF_LOOP) why += " self-loop;";
      if (h_flags & UNSORTED) why += " row not strictly ascending (unsorted or duplicate);";
      if (h_flags & ASYMMETRIC) why += " adjacency not symmetric;";
      return fail(SGC_ERR_INVALID, "invalid CSR:" + why);
    }
  }
  // degree order, highest first, ties by original id; degree-0 vertices dropped.
  // On the device: key = maxd - degree, a stable radix sort of (key, vertex)
  // pairs (ties keep id order), then the inverse map, the sorted degrees and
  // the new row_ptr by an exclusive scan.  The host only needs the degrees of
  // the heavy prefix (for the segments) and of the wide prefix (relabelling).
  // SGC_GRAPH_ORDER_RCM: the same prefix of long rows, the rest in reverse
  // Cuthill-McKee order, computed on the host (rcm_order) and uploaded.
  SGC_TRACE_SCOPE("graph.order");
  int32_t maxd = 0, n_iso = 0, n_heavy_h = 0, n_wide_h = 0;
  g->seg_len = default_seg_len();
  for (int32_t v = 0; v < n; ++v) {
    const int32_t d = h_rp[v + 1] - h_rp[v];
    maxd = std::max(maxd, d);
    n_iso += d == 0;
    n_heavy_h += d > g->seg_len;
    n_wide_h += d > kWideRow;
  }
  const int32_t n_act = n - n_iso;
  g->n_act = n_act;
  g->max_deg = maxd;
  int key_bits = 1;
  while (key_bits < 31 && ((int64_t)1 << key_bits) <= maxd) ++key_bits;
  // device buffers: keys in/out, vertices in/out (the sorted vertices become d_orig)
  uint32_t *d_key = nullptr, *d_key_s = nullptr;
  int32_t *d_vid = nullptr, *d_inv = nullptr, *d_flags = nullptr;
  void* d_tmp = nullptr;
  size_t tmp_sort = 0, tmp_scan = 0;
  cudaError_t e = cudaSuccess;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n + 255) / 256, 65536));
  auto dev_fail = [&](cudaError_t err, const char* what) {
    cudaFree(d_key);
    cudaFree(d_key_s);
    cudaFree(d_vid);
    cudaFree(d_inv);
    cudaFree(d_flags);
    cudaFree(d_tmp);
    return cuda_fail(err, what);
  };
  if (n > 0) {
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_sort, d_key, d_key_s, d_vid, g->d_orig, n, 0, key_bits, st);
    cub::DeviceScan::ExclusiveSum(nullptr, tmp_scan, (const int32_t*)nullptr, (int32_t*)nullptr, n_act + 1, st);
  }
  const size_t tmp_bytes = std::max<size_t>({tmp_sort, tmp_scan, 16});
  if ((e = cudaMalloc(&d_key, sizeof(uint32_t) * std::max(n, 1))) != cudaSuccess ||
      (e = cudaMalloc(&d_key_s, sizeof(uint32_t) * std::max(n, 1))) != cudaSuccess ||
      (e = cudaMalloc(&d_vid, sizeof(int32_t) * ((size_t)std::max(n, 1) + 1))) != cudaSuccess ||
      (e = cudaMalloc(&g->d_orig, sizeof(int32_t) * std::max(n, 1))) != cudaSuccess ||
      (e = cudaMalloc(&d_inv, sizeof(int32_t) * std::max(n, 1))) != cudaSuccess ||
      (e = cudaMalloc(&g->d_row_ptr, sizeof(int32_t) * ((size_t)n_act + 1))) != cudaSuccess ||
      (e = cudaMalloc(&d_tmp, tmp_bytes)) != cudaSuccess)
    return dev_fail(e, "cudaMalloc(graph order)");
  if (n > 0 && (flags & SGC_GRAPH_ORDER_RCM)) {
    std::vector<int32_t> h_ci_copy;
    if (!h_ci && nnz > 0) {
      h_ci_copy.resize((size_t)nnz);
      if ((e = cudaMemcpyAsync(h_ci_copy.data(), d_ci, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost,
                               st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return dev_fail(e, "reading col_idx for the RCM order");
      h_ci = h_ci_copy.data();
    }
    std::vector<int32_t> order;
    rcm_order(n, h_rp, h_ci, std::min(g->seg_len, kWideRow), &order);
    if ((e = cudaMemcpyAsync(g->d_orig, order.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)  // `order` is released on return
      return dev_fail(e, "uploading the RCM order");
    g->ordering = 1;
  } else if (n > 0) {
    k_degree_keys<<<nb, 256, 0, st>>>(d_rp, n, maxd, d_key, d_vid);
    e = cub::DeviceRadixSort::SortPairs(d_tmp, tmp_sort, d_key, d_key_s, d_vid, g->d_orig, n, 0, key_bits, st);
    if (e != cudaSuccess) return dev_fail(e, "sorting the vertices by degree");
  }
  if (n > 0) {
    // d_vid now takes the degrees in the new order (n_act of them, then a 0 for the scan's total)
    if ((e = cudaMemsetAsync(d_inv, 0xFF, sizeof(int32_t) * n, st)) != cudaSuccess)
      return dev_fail(e, "graph order");
    k_order_maps<<<nb, 256, 0, st>>>(g->d_orig, d_rp, n_act, d_inv, d_vid);
    if ((e = cudaMemsetAsync(d_vid + n_act, 0, sizeof(int32_t), st)) != cudaSuccess) return dev_fail(e, "graph order");
    e = cub::DeviceScan::ExclusiveSum(d_tmp, tmp_scan, d_vid, g->d_row_ptr, n_act + 1, st);
    if (e != cudaSuccess) return dev_fail(e, "row_ptr scan");
  } else {
    if ((e = cudaMemsetAsync(g->d_row_ptr, 0, sizeof(int32_t), st)) != cudaSuccess) return dev_fail(e, "graph order");
  }
  // the heavy prefix's degrees and row starts, for the segments
  const int32_t n_pref = std::max(n_heavy_h, std::min(n_wide_h, 65536));
  std::vector<int32_t> pref_deg((size_t)n_pref), pref_rp((size_t)n_pref + 1);
  if (n_pref > 0) {
    if ((e = cudaMemcpyAsync(pref_deg.data(), d_vid, sizeof(int32_t) * n_pref, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(pref_rp.data(), g->d_row_ptr, sizeof(int32_t) * ((size_t)n_pref + 1),
                             cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return dev_fail(e, "reading the heavy rows");
  }
  // heavy rows are a prefix; cut their neighbour lists into seg_len pieces
  std::vector<int32_t> seg_row, seg_lo, seg_hi, heavy_seg(1, 0);
  const int32_t n_heavy = n_heavy_h;
  for (int32_t r = 0; r < n_heavy; ++r) {
    const int32_t lo = pref_rp[(size_t)r], hi = pref_rp[(size_t)r + 1];
    for (int32_t s = lo; s < hi; s += g->seg_len) {
      seg_row.push_back(r);
      seg_lo.push_back(s);
      seg_hi.push_back(std::min(hi, s + g->seg_len));
    }
    heavy_seg.push_back((int32_t)seg_row.size());
  }
  g->n_heavy = n_heavy;
  g->n_seg = (int32_t)seg_row.size();
  sgc_status rc;
  if ((rc = upload(&g->d_seg_row, seg_row, st)) != SGC_OK || (rc = upload(&g->d_seg_lo, seg_lo, st)) != SGC_OK ||
      (rc = upload(&g->d_seg_hi, seg_hi, st)) != SGC_OK || (rc = upload(&g->d_heavy_seg, heavy_seg, st)) != SGC_OK) {
    dev_fail(cudaSuccess, "");
    return rc;
  }
  SGC_TRACE_SCOPE("graph.relabel");  // waits for the CSR copy to the device too
  int32_t h_flags = 0;
  e = cudaMalloc(&g->d_col_idx, std::max<int64_t>(nnz, 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_flags, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_flags, 0, sizeof(int32_t), st);
  if (e == cudaSuccess && n_act > 0) {
    const int32_t n_wide = std::min(n_wide_h, 65536);  // rows in degree order: the long ones are a prefix
    const int64_t light_blocks = std::min<int64_t>((n_act - n_wide + 7) / 8, 65536);
    k_relabel<<<n_wide + std::max<int64_t>(light_blocks, 1), 256, 0, st>>>(
        d_rp, d_ci, n, g->d_orig, d_inv, g->d_row_ptr, n_act, n_wide, g->d_col_idx, d_flags);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_flags, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_key);
  cudaFree(d_key_s);
  cudaFree(d_vid);
  cudaFree(d_inv);
  cudaFree(d_tmp);
  if (d_flags) cudaFree(d_flags);
  if (e != cudaSuccess) return cuda_fail(e, "graph relabel");
  if (h_flags & BAD_COL) return fail(SGC_ERR_INVALID, "invalid CSR: column index out of range");
  if (h_flags & ASYMMETRIC) return fail(SGC_ERR_INVALID, "invalid CSR: adjacency not symmetric");
  return SGC_OK;
}

}  // namespace

// Host CSR: copy to the device, then build.  Device CSR: read row_ptr back for
// the host-side ordering, then build.  The raw copy is released either way.
sgc_status graph_create_impl(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, bool on_device,
                             uint32_t flags, cudaStream_t user_stream, sgc_graph** out) {
  SGC_TRACE_SCOPE("graph.create");
  if (!out) return fail(SGC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 0 || nnz < 0 || nnz > INT32_MAX) return fail(SGC_ERR_INVALID, "n and nnz must be in [0, 2^31)");
  if (!row_ptr || (nnz > 0 && !col_idx)) return fail(SGC_ERR_INVALID, "row_ptr/col_idx is NULL");
  sgc_graph* g = new sgc_graph();
  cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete g;
    return cuda_fail(e, "cudaStreamCreateWithFlags");
  }
  cudaStream_t st = g->stream;
  std::vector<int32_t> h_rp((size_t)n + 1);
  int32_t* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  sgc_status rc = SGC_OK;
  if (on_device) {
    if (user_stream) e = cudaStreamSynchronize(user_stream);
    if (e == cudaSuccess)
      e = cudaMemcpy(h_rp.data(), row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "reading device row_ptr");
    if (rc == SGC_OK) rc = build_graph(n, nnz, row_ptr, col_idx, h_rp, nullptr, flags, st, g);
  } else {
    std::copy(row_ptr, row_ptr + n + 1, h_rp.begin());
    e = cudaMalloc(&d_rp, sizeof(int32_t) * ((size_t)n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_ci, sizeof(int32_t) * std::max<size_t>((size_t)nnz, 1));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_rp, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz > 0)
      e = cudaMemcpyAsync(d_ci, col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = e == cudaErrorMemoryAllocation ? fail(SGC_ERR_OOM, "device memory for the graph")
                                                              : cuda_fail(e, "uploading the graph");
    if (rc == SGC_OK) rc = build_graph(n, nnz, d_rp, d_ci, h_rp, col_idx, flags, st, g);
    cudaStreamSynchronize(st);
    if (d_rp) cudaFree(d_rp);
    if (d_ci) cudaFree(d_ci);
  }
  if (rc != SGC_OK) {
    cudaStreamSynchronize(st);
    destroy_graph(g);
    return rc;
  }
  *out = g;
  return SGC_OK;
}

void graph_destroy_impl(sgc_graph* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  cudaStreamSynchronize(g->stream);
  for (cudaStream_t s : g->lanes) cudaStreamSynchronize(s);
  destroy_graph(g);
}

}  // namespace sgc
