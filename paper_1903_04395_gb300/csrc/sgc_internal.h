// sgc_internal.h - shared declarations of libsgc's host planner, executor and
// kernels.  Not part of the public ABI (include/sgc.h is).
#pragma once

#include <cstdint>
#include <array>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sgc.h"

namespace sgc {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
sgc_status fail(sgc_status st, const std::string& msg);
sgc_status cuda_fail(cudaError_t e, const char* what);

#define SGC_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return ::sgc::cuda_fail(_e, #expr); \
  } while (0)

// ---------------------------------------------------------------- tracing
// Every traced phase is an NVTX range (visible to ncu --nvtx and Nsight); with
// SGC_TRACE set in the environment its host wall time also goes to stderr.
struct TraceScope {
  const char* name;
  long long t0_ns;
  bool on;
  explicit TraceScope(const char* n);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;
};
#define SGC_CAT2(a, b) a##b
#define SGC_CAT(a, b) SGC_CAT2(a, b)
#define SGC_TRACE_SCOPE(name) ::sgc::TraceScope SGC_CAT(sgc_trace_scope_, __LINE__)(name)

// ------------------------------------------------ color-set index (Eq. 1)
// Columns of a count table for sub-templates of size h are the h-subsets of
// the k colors, numbered by Eq. 1: I(C) = sum_i binom(c_i, i) with the colors
// ascending and i counted from 1 (the combinatorial number system, colex
// order).
struct ColorIndex {
  int k = 0;
  uint64_t binom[SGC_MAX_K + 2][SGC_MAX_K + 2] = {};
  explicit ColorIndex(int k_);
  uint64_t nsets(int h) const { return (h < 0 || h > k) ? 0 : binom[k][h]; }
  // rank of a subset given as a bit mask over colors 0..k-1
  uint32_t rank_mask(uint32_t mask) const;
  // subset (bit mask) of size h with rank r
  uint32_t unrank_mask(uint64_t r, int h) const;
};

// ---------------------------------------------------------------- profile
// Per-op device time measured with CUDA events recorded on the launching
// stream around every op of every pass while profiling is on.
struct OpProfile {
  int kind = 0, t = 0, a = 0, p = 0, batch = 0, k = 0;  // k = colors of the op's plan
  int64_t launches = 0;   // passes recorded
  int64_t kernels = 0;    // kernel launches of those passes
  double ms = 0, bytes = 0, flops = 0;  // summed time; algorithmic bytes / flops per pass
  double gather = 0;                    // SpMM: gathered neighbour-row bytes per pass
};

struct PendingEvent {
  int slot;
  cudaEvent_t e0, e1;
};

struct Profiler {
  bool on = false;
  bool by_index = false;   // one slot per op index of the plan (autotuner) instead of per op kind
  std::vector<OpProfile> agg;
  std::vector<PendingEvent> pending;
};

struct PlanSet;

// A recorded launch sequence of one counting call, replayed with one launch.
struct ExecEntry {
  std::string key;
  cudaGraphExec_t exec = nullptr;
  void* ws = nullptr;                 // workspace the graph was recorded on
  int64_t kernels = 0;                // kernel nodes in the graph
  std::vector<std::shared_ptr<PlanSet>> plans;  // keeps the plans (and their keys) alive
};

}  // namespace sgc

struct sgc_graph {
  int device = 0;
  int num_sms = 0;
  int smem_optin = 0;     // bytes of shared memory a block may opt into
  int32_t n = 0;          // vertices as given
  int32_t n_act = 0;      // vertices with degree > 0, renumbered (by degree, desc, or RCM)
  int64_t nnz = 0;
  int32_t max_deg = 0;
  int32_t seg_len = 0;    // neighbour-list segment length for heavy rows
  int32_t n_heavy = 0;    // rows 0..n_heavy-1 have degree > seg_len
  int32_t n_seg = 0;      // segments covering the heavy rows
  int32_t ordering = 0;   // 0 = rows by degree, 1 = heavy prefix by degree + reverse Cuthill-McKee
  int32_t* d_row_ptr = nullptr;   // n_act + 1
  int32_t* d_col_idx = nullptr;   // nnz, new numbering
  int32_t* d_orig = nullptr;      // n_act: original id of each new vertex
  int32_t* d_seg_row = nullptr;   // n_seg: heavy row of each segment
  int32_t* d_seg_lo = nullptr;    // n_seg: first CSR entry of each segment
  int32_t* d_seg_hi = nullptr;    // n_seg: one past the last CSR entry
  int32_t* d_heavy_seg = nullptr; // n_heavy + 1: first segment of each heavy row
  cudaStream_t stream = nullptr;
  mutable std::mutex mu;                  // serialises calls on this handle
  mutable sgc::Profiler prof;
  mutable int64_t kernel_launches = 0;    // kernels enqueued by calls on this handle
  mutable std::vector<std::pair<std::string, std::shared_ptr<sgc::PlanSet>>> plan_cache;
  mutable std::vector<cudaStream_t> lanes;       // side streams for templates counted side by side
  mutable std::vector<cudaEvent_t> lane_events;  // fork (0) and join (1..) events of those streams
  mutable std::vector<sgc::ExecEntry> exec_cache;
};

struct sgc_template {
  int64_t uid = 0;   // unique per created template (plan cache key)
  int32_t k = 0;
  std::vector<int32_t> parent;
  std::vector<std::vector<int32_t>> adj;
  uint64_t aut = 0;
  // device copies of the plan index tables, keyed by (device, root, policy)
  mutable std::mutex mu;
  mutable std::vector<std::pair<std::array<uint64_t, 3>, uint32_t*>> tab_cache;  // (device, hash, words)
};

namespace sgc {

// ------------------------------------------------------------------- plan
enum OpKind : int32_t {
  OP_COLOR = 0,      // colors of every (vertex, coloring)
  OP_HIST = 1,       // P for a single-vertex passive child: neighbour color histogram
  OP_SPMM = 2,       // P = A * M_p
  OP_EMA = 4,        // eMA over the split table (a single-vertex active child needs none)
  OP_FINAL_LEAF = 5, // last step, single-vertex active child, fused with the vertex sum
  OP_FINAL = 6,      // last step, general, fused with the vertex sum
  OP_FINAL_SUM = 7,  // root table summed over all its color sets (more colors than template
                     // vertices, or after an unpruned combine)
  OP_UNPRUNED = 8,   // ablation: a combine in Algorithm 1's order, the neighbour sum taken again
                     // for every color set and split (no SpMM)
};

struct PlanBuffer {
  std::string name;
  int64_t bytes = 0;
  int64_t offset = 0;
  int first = 0, last = 0;  // op indices of first and last use
};

struct PlanOp {
  OpKind kind;
  int out = -1;       // buffer written
  int in_a = -1;      // active table buffer (EMA, FINAL)
  int in_p = -1;      // passive table (SPMM input) or P buffer (GATHER, EMA, FINAL)
  int t = 0, a = 0, p = 0;   // sub-template sizes
  int64_t cols_out = 0, ld_out = 0;
  int64_t cols_a = 0, ld_a = 0;
  int64_t cols_p = 0, ld_p = 0;
  int64_t nsplit = 0;        // binom(t, p)
  bool spmm_buckets = false; // SpMM: sum neighbour rows per neighbour color, resolve once per row
  int spmm_variant = 0;      // direct SpMM loop: 0 chunked, 1 next-neighbour prefetch, 3 / 4 ring
                             // of 2 / 4 asynchronous row copies, 5 / 6 compile-time batch with
                             // the 32-bit / lane-major 16-bit position table, 8 / 9 compile-time
                             // batch with 8 / 12 entries per lane in flight, 10 private
                             // accumulator columns, 11 unrolled (8-bit positions, one 16-byte
                             // load per lane and neighbour), 12 wide (16-bit positions, one
                             // 16-byte load per lane, neighbour and eight entries), 14 one column
                             // at a time (a thread per row and P column walks the row's neighbours:
                             // the pruned sums without the row-wise SpMM), 13 grouped
                             // (a warp per row and coloring sums the rows of each neighbour color
                             // in registers and scatters each color's sum once; chunks of up to 512
                             // columns), 15 the same with chunks of up to 256 columns;
                             // bucketed: 0 shared-memory buckets, 2 register buckets, 7 shared-
                             // memory buckets with a compile-time batch
  int spmm_pos_bytes = 0;    // direct: 0 = 32-bit position table read through L1; 1 or 2 =
                             // packed entries staged in shared memory
  int shape = 0;             // launch shape code (kSpmm* / eMA rows), see op_shape_candidates
  int ema_rows = 0;          // eMA: rows staged per block (32 * rows_per_lane, or 16..1)
  int ema_reg_k = 0;         // eMA: > 0 = the register form for K = ema_reg_k relative colors
  int ema_sched = 0;         // eMA: > 0 = the scheduled form (one coloring per pass) staging this many rows
  int ema_upg = 1;           // scheduled eMA: warps sharing one group of 32 outputs
  bool final_reg = false;    // last step: compile-time complement indices (k_final_reg)
  bool ema_final = false;    // eMA (register form, symmetric) fused with the last step that
                             // follows it: writes the last step's partials, not its table
  bool final_fused = false;  // last step done by the preceding fused eMA (only the sum remains)
  int ema_rpl = 1;           // eMA: rows per lane
  int ema_vrpl = 0;          // eMA over vertex tiles (batch >= 4) with 1 or 2 rows per lane; 0 = rows
                             // staged column-major (ema_rows)
  bool ema_sym = false;      // eMA of a table with itself (same buffer, |A| - 1 == |T_p|): each
                             // unordered split once, doubled
  int64_t tab_off = -1;      // offset (uint32 words) of this op's index table
  int64_t tab2_off = -1;     // OP_UNPRUNED: the neighbour position table
  int state_out = -1, state_a = -1, state_p = -1;  // scale-state slots (FP32)
  double alg_bytes = 0;      // algorithmic HBM bytes of one pass (tables read / written once)
  double alg_flops = 0;      // multiply + add count of one pass
  double gather_bytes = 0;   // SpMM / histogram: neighbour-row bytes gathered in one pass
};

struct Plan {
  int k = 0, root = 0, batch = 1, precision = SGC_FP32, policy = 0;  // k = number of colors
  int t_size = 0;            // template vertices (<= k)
  int elem = 4;              // bytes per table entry
  int64_t rows = 0;          // n_act * batch
  std::vector<PlanBuffer> bufs;
  std::vector<PlanOp> ops;
  std::vector<uint32_t> tabs;  // all index tables, concatenated
  int n_states = 0;
  int n_tables = 0, n_spmm = 0, n_ema = 0;
  int64_t ws_bytes = 0;
  // per-coloring algorithmic traffic (bytes) and eMA FMAs
  double est_bytes = 0, est_spmm_bytes = 0, est_fma = 0, est_cost = 0;
  // fixed buffers
  int buf_colors = -1, buf_seeds = -1, buf_out = -1, buf_states = -1, buf_partials = -1;
  int buf_scratch = -1, buf_hist_heavy = -1;
  // neighbours grouped by color, per coloring (grouped SpMM form only): ids, colors, kept counts
  int buf_gids = -1, buf_gcols = -1, buf_gkept = -1;
  int final_blocks = 0;
  int64_t scratch_width = 0;
};

// Launch-shape codes an autotuner may pick per op (0 keeps the planner's choice);
// eMA: the rows a block stages.
// SpMM: the direct form with its chunked loop, the direct form with a
// next-neighbour prefetch, the bucketed form (buckets in shared memory),
// register buckets (one coloring per pass), or the direct form with its
// position table packed into 1- or 2-byte entries and staged in shared memory.
// The direct form can also stream neighbour rows through a ring of 2 or 4
// shared-memory slots filled by asynchronous copies (batch >= 4), or run with
// the batch as a compile-time constant (immediate offsets, shuffled ids) with
// the 32-bit position table or a lane-major 16-bit one, or with 8 / 12 entries
// per lane in flight (11 / 12), or with one private accumulator column per
// lane (13, conflict-free adds), or unrolled over a compile-time bound on a
// lane's entries with one 16-byte position load per neighbour (14), or in
// chunks of eight 16-bit positions per 16-byte load for any width (15);
// likewise the bucketed form (10).
constexpr int kShapeSpmmDirect = 1, kShapeSpmmPrefetch = 2, kShapeSpmmBuckets = 3, kShapeSpmmRegBuckets = 4,
              kShapeSpmmPacked = 5, kShapeSpmmRing2 = 6, kShapeSpmmRing4 = 7, kShapeSpmmDirectB = 8,
              kShapeSpmmDirectBLane = 9, kShapeSpmmBucketsB = 10, kShapeSpmmDirectB8 = 11,
              kShapeSpmmDirectB12 = 12, kShapeSpmmDirectBPriv = 13, kShapeSpmmUnrolled = 14,
              kShapeSpmmWide = 15, kShapeSpmmGrouped = 16, kShapeSpmmGrouped8 = 17, kShapeSpmmStaged = 18,
              kShapeSpmmStaged8 = 19;
// private accumulator columns (shape 13) are tried while a warp's fit in this
constexpr int64_t kSpmmPrivMaxBytes = 16 * 1024;
constexpr int64_t kSpmmPackedMaxBytes = 24 * 1024;
// eMA shape codes for the vertex-tile kernel (1 or 2 rows per lane) and the
// register form (FP32, the (K, a-1, p, symmetric) shapes compiled in)
constexpr int kShapeEmaVertex1 = 101, kShapeEmaVertex2 = 102, kShapeEmaReg = 103, kShapeEmaSched = 104,
              kShapeEmaSched2 = 105;
// the scheduled eMA (shape 104, one coloring per pass, kEmaSchedWarps warps per block): rows a block
// stages (8, 6, 4 or 2 within 200 KB; 0 = does not fit) and shares of each group of 32 outputs' rounds
constexpr int kEmaSchedWarps = 16;
// rows per block of the scheduled eMA: the most of 8, 6, 4, 2 (12 too for two blocks) whose
// block fits in at most 200 KB (blocks = 1) or in half of an SM's shared memory (blocks = 2: two
// blocks per SM, one staging its rows while the other computes); 0 when none fits
int ema_sched_rows(int64_t ct, int64_t ld_a, int64_t ld_p, bool sym, int elem, int64_t smem_cap, int* upg,
                   int blocks = 1);
// words of one staged row: M_a row, P row (unless the table is combined with itself), 4 zero words
inline int64_t ema_sched_rw(int64_t ld_a, int64_t ld_p, bool sym) { return ld_a + (sym ? 0 : ld_p) + 4; }
inline int64_t ema_sched_smem(int rows, int64_t ct, int64_t ld_a, int64_t ld_p, bool sym, int elem, int upg) {
  const int64_t G = (ct + 31) / 32;
  return (int64_t)rows * ema_sched_rw(ld_a, ld_p, sym) * elem + (upg > 1 ? G * upg * 32 * rows * elem : 0) + 16;
}
// whether the register-form eMA is compiled in for K relative colors, an active
// child of a vertices (a - 1 colors besides the root's) and a passive child of p
bool ema_reg_compiled(int K, int a_minus_1, int p, bool sym);
// whether the last step's compile-time form is compiled in for K relative colors and a passive child of p
bool final_reg_compiled(int K, int p);
// whether the fused symmetric register eMA + last step is compiled in (K, a - 1 = p)
bool ema_final_compiled(int K, int p);
// entries per lane of the lane-major position table of the batch-specialised
// direct form (L lanes per coloring; a multiple of 4 so a lane reads 4 at once)
inline int64_t spmm_lane_nsp(int64_t w_in, int L) { return ((w_in + L - 1) / L + 3) / 4 * 4; }
// whether the unrolled direct SpMM (shape 14) takes this op: 4, 8 or 16 colorings, at most 16
// entries per lane and neighbour, positions below 255
// chunks of eight entries per lane of the wide direct SpMM (shape 15)
inline int64_t spmm_wide_nch(int batch, int64_t w_in) {
  const int L = 32 / batch;
  return ((w_in + L - 1) / L + 7) / 8;
}
inline bool spmm_unrolled_fits(int batch, int64_t w_in, int64_t ld_out) {
  if (batch != 4 && batch != 8 && batch != 16) return false;
  const int L = 32 / batch;
  return (w_in + L - 1) / L <= 16 && ld_out < 255;
}
// whether the grouped SpMM (shape 16) takes this op: at most 4 colorings per pass (a warp
// per row and coloring reads the coloring's entries at a stride of `batch`), positions in 16
// bits, and at least two warps' output rows in shared memory
inline bool spmm_grouped_fits(int batch, int64_t ld_out, int elem, int64_t smem_cap) {
  return batch <= 4 && ld_out < 65535 && 2 * ld_out * elem <= smem_cap;
}
// the grouped SpMM's kernel variants: 13 and 15 (neighbour rows in registers, chunks of 512 or
// 256 columns), 16 and 17 (the staged form: rows copied into a ring of shared-memory slots)
inline bool spmm_variant_grouped(int v) { return v == 13 || v == 15 || v == 16 || v == 17; }
// the staged form: chunks of 128 nr4 columns (the fewest chunks, at most 1,024 columns), a ring
// of 3 (variant 16) or 2 (17: less shared memory per warp, more warps per SM) chunk slots per
// warp, and rows of 16-bit positions at a pitch of whole 16-byte pieces
inline int spmm_staged_nr4(int64_t w_in, int variant) {
  (void)variant;
  return w_in <= 256 ? 2 : w_in <= 512 ? 4 : 8;
}
inline int spmm_staged_rs(int variant) { return variant == 17 ? 2 : 3; }
inline int64_t spmm_staged_pitch(int64_t w_in) { return (w_in + 7) / 8 * 8; }
// a warp's shared memory: its output row, the chunk ring, rs + 1 chunks of positions
inline int64_t spmm_staged_warp_bytes(int64_t w_in, int64_t ld_out, int variant) {
  const int64_t ch = 128 * spmm_staged_nr4(w_in, variant), rs = spmm_staged_rs(variant);
  return 4 * (ld_out + rs * ch + (rs + 1) * ch / 2);
}
// whether the staged form takes this op: FP32, one coloring per pass, rows wider than 128
// columns, positions in 16 bits, and at least two warps in shared memory
inline bool spmm_staged_fits(int batch, int64_t w_in, int64_t ld_out, int elem, int64_t smem_cap, int variant) {
  return batch == 1 && elem == 4 && w_in > 128 && ld_out < 65535 &&
         2 * spmm_staged_warp_bytes(w_in, ld_out, variant) <= smem_cap;
}
// entries per [c_v][c_u] row of the packed position table (rows of whole words)
inline int64_t spmm_packed_ld(int64_t w_in, int eb) { return (w_in * eb + 3) / 4 * 4 / eb; }

// Plan the DP for template t on graph g.  root < 0 and policy < 0 let the
// cost model choose; batch is the number of colorings per pass.  Index tables
// are only built when build_tabs is set.  `shapes`, when given, holds one
// launch-shape code per op index (0 = default); codes that do not fit the
// op (shared memory, form) are ignored.  colors = number of colors (0: |T|).
// unpruned: 1 = the ablation plan of Algorithm 1's loop order (OP_UNPRUNED ops); 2 = the
// pruned plan with every SpMM taken one passive column at a time (thread per row and column).
sgc_status make_plan(const sgc_graph* g, const sgc_template* t, int precision, int root, int policy, int batch,
                     bool build_tabs, Plan* out, const std::vector<int>* shapes = nullptr, int colors = 0,
                     int unpruned = 0);

// The launch shapes worth timing for op `i` of plan p (empty: nothing to choose).
std::vector<int> op_shape_candidates(const sgc_graph* g, const Plan& p, int i);

uint64_t automorphisms(const sgc_template* t);

int pow2_floor(int x);
long double inverse_colorful_probability(int t, int colors);
sgc_options resolve(const sgc_options* opt);
struct PlanSet;
// Plans for every power-of-two batch up to bmax (capped for SpMM occupancy) whose
// workspace fits mem_limit, cached on the graph; the caller holds g->mu.
sgc_status plan_batches(const sgc_graph* g, const sgc_template* t, const sgc_options& o, int bmax, int64_t mem_limit,
                        std::shared_ptr<PlanSet>* out);
// Device copy of a plan's index tables, cached on the template by content.
sgc_status template_tables(const sgc_template* t, const Plan& plan, int device, const uint32_t** out);

sgc_status graph_create_impl(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, bool on_device,
                             uint32_t flags, cudaStream_t user_stream, sgc_graph** out);
void graph_destroy_impl(sgc_graph* g);

// -------------------------------------------------------------- kernels
struct ScaleState {
  int32_t e;          // table value = count * 2^-e  (FP32 path)
  uint32_t max_bits;  // bits of the largest stored value (non-negative float)
};

// Executes one pass of `plan` for plan.batch colorings whose seeds are in
// the workspace; writes plan.batch doubles (colorful maps) to the out buffer.
// With a profiler, CUDA events bracket every op.  *kernels counts launches.
sgc_status run_pass(const sgc_graph* g, const Plan& plan, const uint32_t* d_tabs, char* ws,
                    cudaStream_t stream, Profiler* prof, int64_t* kernels);

// Shared memory per warp of the bucketed SpMM form: one bucket row per color.
inline int64_t spmm_bucket_bytes(int batch, int k, int64_t w_in, int elem) {
  return (int64_t)batch * k * w_in * elem;
}
constexpr int64_t kSpmmBucketMaxBytes = 4 * 1024;  // keeps ~48 warps per SM resident
constexpr int64_t kSpmmRowBytesPerWarp = 8 * 1024;  // batch cap for wide SpMM output rows

// Plans for the powers of two up to `btop` colorings per pass (same root and
// cut order), cached per graph; `bfit` is the one count calls use.
struct PlanSet {
  std::map<int, Plan> by_batch;
  int btop = 1;  // the most colorings per pass that fit (the autotuner starts there)
  int bfit = 1;
  bool tuned = false;                 // by_batch[bfit] (and the next smaller) carry timed shapes
  std::vector<sgc_tune_entry> report; // what the autotuner measured
};

}  // namespace sgc
