/*
 * sgc.h - C ABI of libsgc, a GB300 (sm_103a) implementation of color-coding
 * counting of non-induced tree templates (Chen et al., "A GraphBLAS Approach
 * for Subgraph Counting", HPDC'19).
 *
 * One iteration of the method (Section 2.1) colors every vertex uniformly at
 * random with k = |T| colors, counts the colorful embeddings of the template
 * T by a dynamic program over sub-templates, and scales the count by
 * k^k / k! (the inverse of the probability that a fixed copy is colorful).
 * Each DP step for a sub-template T_s with active child T_a and passive child
 * T_p is
 *     P   = A * M_p                                   (SpMM, Eq. 2 and Section 4.5)
 *     M_s(v, I(C)) = sum over splits C = C_a + C_p of
 *                    M_a(v, I(C_a)) * P(v, I(C_p))    (eMA, Section 4.5)
 * with color sets indexed by Eq. 1.  The last step reduces over vertices.
 *
 * Conventions for every function below:
 *   - Return an sgc_status; SGC_OK is 0.  On failure sgc_last_error() gives a
 *     message (thread-local, valid until the next call on that thread).
 *   - Host pointers are only read during the call; inputs are copied.
 *   - Handles are opaque, owned by the library, and released by the matching
 *     *_destroy function (NULL is accepted and ignored).
 *   - All device work runs on the GPU that was current when the graph was
 *     created.  Calls on the same graph handle are serialised internally.
 *   - There is no CPU fallback: if no CUDA device is usable, calls that need
 *     one return SGC_ERR_CUDA.
 */
#ifndef SGC_H
#define SGC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sgc_status {
  SGC_OK = 0,
  SGC_ERR_INVALID = 1,     /* bad argument: malformed CSR, not a tree, k out of range ... */
  SGC_ERR_OOM = 2,         /* device or host memory exhausted, or above options.mem_limit */
  SGC_ERR_CUDA = 3,        /* a CUDA runtime error (message has the CUDA error string) */
  SGC_ERR_TIMEOUT = 4,     /* a bounded wait ran out (server wait, device-side spin limit) */
  SGC_ERR_OVERFLOW = 5,    /* a result is not representable (not expected for k <= 16) */
  SGC_ERR_INTERNAL = 6,    /* a device-side consistency check failed */
  SGC_ERR_UNSUPPORTED = 7  /* valid request outside what this build supports */
} sgc_status;

/* Arithmetic of the count tables.  FP64 tables hold exact integers while
 * every count stays below 2^53.  FP32 tables hold counts divided by a
 * per-table power of two chosen on the device so nothing overflows; products
 * are summed in FP32 inside SpMM and eMA and the final vertex reduction is
 * FP64. */
typedef enum sgc_precision { SGC_FP32 = 0, SGC_FP64 = 1 } sgc_precision;

/* Largest number of colors (and template vertices) supported: 18, so that every color set of
 * the relative-color tables (subsets of the other k - 1 = 17 colors, at most C(17, 8) = 24310 per
 * row) has a 16-bit index. */
#define SGC_MAX_K 18

typedef struct sgc_graph sgc_graph;
typedef struct sgc_template sgc_template;

/* Graph creation flags. */
#define SGC_GRAPH_VALIDATE 1u   /* check CSR invariants on the device (recommended) */
#define SGC_GRAPH_ORDER_RCM 2u  /* renumber the rows of degree <= 256 in reverse Cuthill-McKee order
                                   (Section 4.3's locality pre-processing) instead of by degree;
                                   computed on the host, O(nnz log d) */

typedef struct sgc_options {
  int32_t precision;   /* sgc_precision; default SGC_FP32 */
  int32_t batch;       /* colorings evaluated together in one device pass; 0 = automatic */
  int64_t mem_limit;   /* device workspace bytes this call may use; 0 = 90% of free memory */
  void* stream;        /* cudaStream_t to run on; NULL = the graph's own stream */
  int32_t root;        /* template vertex used as the DP root; -1 = cost-model choice */
  int32_t use_graph;   /* 1 (default) = record the call's whole launch sequence - every pass of
                          every template - as one CUDA graph, cache it on the graph handle and
                          replay it with one launch; 0 = launch op by op.  Profiling (below)
                          always launches op by op. */
  int32_t autotune;    /* 1 = before the first count of a template on a graph, time every
                          candidate launch shape of each SpMM and eMA op (and the two largest
                          batch sizes) on that graph and keep the fastest; cached with the
                          plan.  0 (default) = the planner's shapes. */
  int32_t spmm_shape;  /* force the SpMM launch shape: 1 direct, 2 direct with next-neighbour
                          prefetch, 3 bucketed, 4 register buckets (one coloring per pass: use
                          batch = 1), 5 direct with a packed position table in shared memory,
                          6 / 7 direct with neighbour rows streamed through a ring of 2 / 4
                          asynchronous copies (batch >= 4), 8 / 9 direct specialised for the
                          batch (9: with a lane-major 16-bit position table; 11 / 12: with 8 / 12
                          entries per lane in flight; 13: with a private accumulator column per
                          lane; 14: unrolled, one 16-byte position load per lane and neighbour,
                          4..16 colorings; 15: 16-bit positions, one 16-byte load per lane,
                          neighbour and eight entries, any width), 10 bucketed specialised for the
                          batch, 16 grouped (1, 2 or 4 colorings per pass: a warp per row and
                          coloring sums the rows of each neighbour color in registers and adds each
                          color's sum into the output row once; columns in chunks of up to 512),
                          17 grouped in chunks of up to 256 columns, 18 grouped with the
                          neighbour rows copied into a ring of 3 shared-memory chunks of up to
                          1,024 columns per warp (FP32, one coloring per pass, rows wider than 128
                          columns), 19 the same with a ring of 2 chunks (more warps per SM); ops
                          it does not fit keep theirs.  0 (default) = planner or
                          autotuner.  Results do not depend on it beyond FP32 summation order. */
  int32_t ema_rows;    /* force the eMA shape: 64, 32, 16, 8, 4, 2 or 1 rows staged column-major per
                          block, or 101 / 102 = whole vertex rows copied asynchronously in tiles,
                          1 / 2 rows per lane (4..32 colorings per pass), or 103 = every operand in
                          registers (FP32; the shapes compiled in: 10 colors with 3-color active and
                          passive children, and the 7-, 8- and 11-color trees' combines with narrow
                          rows; the default where it applies at 8 or more colorings per pass), or
                          104 = scheduled (one coloring per pass: up to 8 rows staged by bulk copies
                          in at most 200 KB, each output's split terms in rounds that read distinct
                          shared-memory banks), or 105 = scheduled with up to 12 rows in half of
                          an SM's shared memory, so that two blocks share an SM (one stages its
                          rows while the other computes; the default where each block gets at least
                          as many rows as one block alone would);
                          ops it does not fit keep theirs; 0 (default) = planner or autotuner */
  int32_t colors;      /* number of colors k (Section 2.1: k >= |T|): 0 (default) = |T|, else
                          |T| <= colors <= SGC_MAX_K.  A map is colorful when its |T| images have
                          distinct colors; the estimate divides by k! / ((k - |T|)! k^|T|). */
  int32_t unpruned;    /* ablations, same results: 1 = without the pruning (Eq. 2, Section 4.2):
                          every combine in Algorithm 1's loop order, the neighbour sum taken again
                          for each color set and split (no SpMM); 2 = pruned as in Section 4.2
                          (each neighbour sum once per passive color set) but one column at a time,
                          a thread per vertex and column walking its neighbours, instead of the
                          row-wise SpMM of Section 4.5.  0 (default) = pruned, SpMM + eMA. */
} sgc_options;

/* Fill *opt with the defaults described above. */
void sgc_options_init(sgc_options* opt);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char* sgc_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t sgc_version(void);

/* ---------------------------------------------------------------- graphs -- */

/*
 * Create a graph from a host CSR adjacency (Section 4.3: the adjacency
 * matrix A_G with A(i,j) = 1 for an edge).
 *   n        vertices, 0 <= n < 2^31
 *   nnz      stored entries = 2 * |E|
 *   row_ptr  n+1 int32, row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz
 *   col_idx  nnz int32 in [0, n); each row strictly ascending (no
 *            duplicates), no self-loops, and the matrix symmetric
 *   flags    SGC_GRAPH_VALIDATE checks all of the above (SGC_ERR_INVALID)
 * The library copies the CSR to the device, drops isolated vertices (they
 * are in no embedding of a template with k >= 2) and renumbers the rest by
 * degree, highest first; with SGC_GRAPH_ORDER_RCM only the rows longer than
 * 256 stay first by degree and the others follow in reverse Cuthill-McKee
 * order (neighbouring rows get nearby numbers, so the SpMM's gathers reuse
 * cached rows).  Counts do not depend on vertex numbering: colors are drawn
 * from the original ids.
 */
sgc_status sgc_graph_create(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                            uint32_t flags, sgc_graph** out);

/* Same as sgc_graph_create, from device-resident CSR arrays (read on
 * `stream`, a cudaStream_t or NULL; the caller keeps ownership). */
sgc_status sgc_graph_create_device(int32_t n, int64_t nnz, const int32_t* d_row_ptr,
                                   const int32_t* d_col_idx, uint32_t flags, void* stream,
                                   sgc_graph** out);

typedef struct sgc_graph_stats {
  int32_t n;          /* vertices as given */
  int32_t n_active;   /* vertices with degree > 0 (rows of every count table) */
  int64_t nnz;        /* stored adjacency entries */
  int32_t max_degree;
  int32_t n_heavy;    /* rows whose neighbour list is split across warps in SpMM */
  int32_t n_segments; /* neighbour-list segments of those rows */
  int32_t device;     /* CUDA device ordinal */
  int64_t kernel_launches; /* kernels enqueued so far by calls on this handle */
  int32_t ordering;   /* 0 = rows by degree, 1 = reverse Cuthill-McKee (SGC_GRAPH_ORDER_RCM) */
} sgc_graph_stats;

sgc_status sgc_graph_stats_get(const sgc_graph* g, sgc_graph_stats* out);
void sgc_graph_destroy(sgc_graph* g);

/* ------------------------------------------------------------- templates -- */

/*
 * Create a tree template from a parent array (Section 2.1, item 2).
 *   k       vertices, 1 <= k <= SGC_MAX_K
 *   parent  k int32; exactly one entry is -1 (the given root), every other
 *           entry is a vertex in [0, k), and the edges form one tree.
 * The DP root and the order in which child edges are cut are chosen per
 * count call by a cost model after Lemma 1 (or fixed by options.root);
 * results do not depend on that choice.
 */
sgc_status sgc_template_create(int32_t k, const int32_t* parent, sgc_template** out);

/* |Aut(T)|, the number of automorphisms of the (unrooted) template. */
sgc_status sgc_template_automorphisms(const sgc_template* t, uint64_t* aut);
void sgc_template_destroy(sgc_template* t);

typedef struct sgc_plan_info {
  int32_t root;            /* DP root used */
  int32_t n_tables;        /* distinct sub-template count tables (isomorphic ones shared) */
  int32_t n_spmm;          /* SpMM passes (one per distinct passive sub-template) */
  int32_t n_ema;           /* eMA steps, including the final one */
  int32_t batch;           /* colorings per device pass */
  int64_t workspace_bytes; /* device workspace for one pass of `batch` colorings */
  double est_bytes;        /* algorithmic HBM bytes per coloring (tables read/written once) */
  double est_spmm_bytes;   /* of which SpMM (CSR + gathers counted once + outputs) */
  double est_fma;          /* eMA multiply-adds per coloring */
} sgc_plan_info;

/* Describe the plan sgc_count would use for this graph, template and options. */
sgc_status sgc_plan_get(const sgc_graph* g, const sgc_template* t, const sgc_options* opt,
                        sgc_plan_info* out);

/* -------------------------------------------------------------- counting -- */

/*
 * Run n_iter color-coding iterations, one per seed.
 *   seeds          n_iter host uint64 coloring seeds.  Vertex v (original
 *                  numbering) gets color floor(hi32(x) * k / 2^32) where x is
 *                  output number v of the SplitMix64 stream keyed by the seed
 *                  (Steele, Lea and Flood 2014): x = mix(seed + (v+1) * 0x9E3779B97F4A7C15).
 *   opt            NULL for defaults
 *   estimate       out (host, may be NULL): mean over iterations of
 *                  maps_i / |Aut(T)| * k^k / k!  (with opt->colors = k > |T|:
 *                  maps_i / |Aut(T)| * (k - |T|)! k^|T| / k!)
 *   colorful_maps  out (host, n_iter doubles, may be NULL): for each coloring
 *                  the number of colorful injective edge-preserving maps
 *                  T -> G, i.e. sum_v N(v, T, all colors) = |Aut(T)| * colorful copies.
 *                  Exact in SGC_FP64 while every count is below 2^53.
 * Blocks until the results are on the host.
 */
sgc_status sgc_count(const sgc_graph* g, const sgc_template* t, const uint64_t* seeds, int32_t n_iter,
                     const sgc_options* opt, double* estimate, double* colorful_maps);

/*
 * Device-resident form of sgc_count for pipelines that keep everything on
 * the GPU: seeds and colorful_maps are device pointers (n_iter each), the
 * work is enqueued on opt->stream (or the graph's stream) and the call
 * returns without synchronising.  The workspace stays owned by the graph;
 * do not destroy the graph before the stream has finished.
 */
sgc_status sgc_count_device(const sgc_graph* g, const sgc_template* t, const uint64_t* d_seeds,
                            int32_t n_iter, const sgc_options* opt, double* d_colorful_maps);

/*
 * Count several templates on one graph in one call.  Every coloring of every
 * template is an independent iteration of the estimator of Section 2.1 (the
 * iteration count of Section 5.1 is per template).  For template j,
 * seeds[j * n_iter + i] (host) is the seed of its coloring i, and the results
 * are colorful_maps[j * n_iter + i] and estimates[j] (host, either may be
 * NULL), each equal to what sgc_count returns for that template and those
 * seeds.  The passes of different templates run side by side on up to four
 * streams (templates assigned longest first to the least loaded stream, fewer
 * streams when their workspaces do not fit opt->mem_limit); with
 * opt->use_graph the whole call - every pass of every template - is one CUDA
 * graph launch, recorded on the first call and replayed on later calls with
 * the same templates, n_iter and options (new seeds each time).
 * Blocks until the results are on the host.
 */
sgc_status sgc_count_many(const sgc_graph* g, int32_t n_templates, const sgc_template* const* templates,
                          const uint64_t* seeds, int32_t n_iter, const sgc_options* opt, double* estimates,
                          double* colorful_maps);

/* One op of a tuned plan: the launch shapes timed and the one kept. */
typedef struct sgc_tune_entry {
  int32_t kind;              /* as sgc_op_profile.kind */
  int32_t t, a, p;           /* sub-template sizes */
  int32_t batch;             /* colorings per pass of the plan tuned */
  int32_t n_candidates;
  int32_t chosen;            /* index of the kept shape in shapes[] */
  int32_t shapes[8];         /* SpMM: 1 direct, 2 direct with prefetch, 3 bucketed, 4 register buckets,
                                5 direct with packed positions, 6 / 7 direct with a copy ring,
                                8 / 9 / 11 / 12 / 13 / 14 / 15 direct specialised for the batch, 10
                                bucketed specialised, 16 / 17 grouped;
                                eMA: rows staged per block, or 101 / 102 vertex tiles */
  double ms[8];              /* device time of the op, one pass, per shape */
} sgc_tune_entry;

/*
 * Launch shapes of the SpMM (Eq. 2, Section 4.5) and eMA (Section 4.5) steps
 * only change how the same sums are scheduled; FP64 results are identical and
 * FP32 results differ by summation order only.
 * Run the autotuner for template t on graph g under *opt (as sgc_count with
 * opt->autotune = 1 would before its first pass) and copy up to `cap` entries of
 * its report to out; *n = entries available.  The batch sizes compared are
 * reported with kind = -1, shapes[] = batch sizes and ms[] = time per coloring.
 */
sgc_status sgc_autotune(const sgc_graph* g, const sgc_template* t, const sgc_options* opt, sgc_tune_entry* out,
                        int32_t cap, int32_t* n);

/* ---------------------------------------------------- iteration count -- */

/*
 * Colorings for an (eps, delta)-approximation of the copy count in the worst
 * case: the lemma after Lemma 1 (Section 5.1) performs O(e^k log(1/delta) /
 * eps^2) iterations; this returns ceil(e^k ln(1/delta) / eps^2), i.e. that
 * bound with constant 1 (the paper gives none).  0 < eps, 0 < delta < 1,
 * 1 <= k <= SGC_MAX_K; -1 on bad arguments.
 */
int64_t sgc_iterations_bound(int32_t k, double eps, double delta);

/*
 * Count colorings of template t until the estimate meets a relative
 * (eps, delta) target empirically: after every chunk of colorings (seeds
 * first_seed, first_seed + 1, ..., chunk = opt->batch or 32), with n colorings
 * so far, mean m and sample standard deviation s of the per-coloring estimates
 * (maps_i / |Aut(T)| * k^k / k!, Section 2.1), it stops once n >= min_iter and
 * z * s / sqrt(n) <= eps * m, z the standard normal quantile at 1 - delta / 2
 * (a normal-approximation confidence interval of half-width eps * m), or once
 * n reaches max_iter (0: sgc_iterations_bound(k, eps, delta)).
 *   estimate        out: m
 *   n_used          out: n
 *   rel_half_width  out (may be NULL): z * s / (sqrt(n) * m), 0 when m = 0
 * Colorings are counted as by sgc_count with *opt (precision, batch, ...).
 */
sgc_status sgc_estimate(const sgc_graph* g, const sgc_template* t, double eps, double delta, uint64_t first_seed,
                        int64_t min_iter, int64_t max_iter, const sgc_options* opt, double* estimate,
                        int64_t* n_used, double* rel_half_width);

/*
 * The color-coding estimate of Section 2.1 from per-coloring colorful maps
 * (as sgc_count returns them, e.g. gathered from several processes that each
 * counted their own seeds): the mean over the n colorings of
 * maps_i / |Aut(T)| / P(colorful), with P(colorful) = k! / k^k for k = |T|
 * colors, or k! / ((k - |T|)! k^|T|) for colors = k > |T| (0 = |T|).
 *   maps      n host doubles, each >= 0
 *   estimate  out (host); 0 when n = 0
 */
sgc_status sgc_estimate_from_maps(const sgc_template* t, int32_t colors, const double* maps, int64_t n,
                                  double* estimate);

/* --------------------------------------------------------------- serving -- */

/*
 * A counting server over one device-resident graph with continuous batching
 * (the paper has no counterpart; it serves many color-coding queries on one
 * graph).  Requests (template, colorings) queue on the host; a scheduler thread
 * admits them - of the first 8 queued, the shortest by the planner's cost model
 * that fits; the oldest is overtaken at most 8 times - whenever their device
 * workspace fits in the free part of `mem_budget` bytes
 * (allocated once, at creation) and one of `max_inflight` execution slots is
 * free.  Each admitted request runs its DP passes on its own stream, so requests
 * overlap on the GPU; the stream's priority follows the request's estimated
 * device time (shorter requests get higher priorities).  Results are those of sgc_count for the same seeds and
 * precision (FP32 within the FP32 tolerance: a request's batch size may differ).
 * The graph and every submitted template must outlive the server.
 */
typedef struct sgc_server sgc_server;

sgc_status sgc_server_create(const sgc_graph* g, int64_t mem_budget, int32_t max_inflight, sgc_server** out);

/* Queue n colorings (host seeds, copied) of template t; *ticket identifies the request. */
sgc_status sgc_server_submit(sgc_server* s, const sgc_template* t, const uint64_t* seeds, int32_t n,
                             int32_t precision, uint64_t* ticket);

/*
 * Wait up to timeout_ms (< 0: no limit) for a request.  On SGC_OK the request is
 * retired and estimate, maps[n] (colorful maps per coloring) and latency_ms
 * (submission to completion) are written where non-NULL.  SGC_ERR_TIMEOUT leaves
 * the request pending (wait again); a request that failed returns its error
 * (SGC_ERR_OOM when its workspace exceeds the whole budget) and is retired.
 */
sgc_status sgc_server_wait(sgc_server* s, uint64_t ticket, int32_t timeout_ms, double* estimate, double* maps,
                           double* latency_ms);

typedef struct sgc_server_stats {
  int64_t completed;       /* requests finished successfully */
  int64_t failed;          /* requests that failed or were cancelled */
  int64_t pending;         /* queued, not admitted yet */
  int32_t inflight;        /* admitted, running */
  int32_t peak_inflight;   /* most requests running at once */
  int64_t peak_bytes;      /* most budget bytes in use at once */
  int64_t kernel_launches; /* kernels enqueued by the server */
  double latency_p50_ms;   /* over completed requests, submission to completion */
  double latency_p99_ms;
  double queue_p50_ms;     /* submission to admission */
  double span_s;           /* first submission to last completion */
} sgc_server_stats;

sgc_status sgc_server_stats_get(sgc_server* s, sgc_server_stats* out);

/* Cancel queued requests, wait for running ones, release everything. */
void sgc_server_destroy(sgc_server* s);

/*
 * Counting without any device allocation (the paper has no counterpart:
 * this serves callers that cannot call cudaMalloc while they count, such as
 * code whose device memory is owned by another framework's allocator or a
 * service whose device-memory footprint must stay fixed after start-up).
 * Same arguments and results as sgc_count_device, but every byte of scratch
 * - count tables, partial rows and sums, colorings, the plan's index tables -
 * comes from one static device array of SGC_STATIC_WORKSPACE_BYTES, held by
 * every GPU that loads the library until the process exits.
 *   - Requests whose single-coloring scratch exceeds that size fail with
 *     SGC_ERR_UNSUPPORTED (use sgc_count_device); larger batches are split.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make it before any stream capture.
 *   - All calls share the array: calls that overlap on the GPU race.  Each
 *     call waits for its own work before returning.
 *   - The graph and template handles are created beforehand (that allocates).
 */
#define SGC_STATIC_WORKSPACE_BYTES (64u << 20)
sgc_status sgc_count_device_static(const sgc_graph* g, const sgc_template* t, const uint64_t* d_seeds,
                                   int32_t n_iter, const sgc_options* opt, double* d_colorful_maps);

/* ------------------------------------------------------------ profiling -- */

/* Device time of one kind of DP op, aggregated over the passes recorded
 * since profiling was enabled or last read.  Times come from CUDA events
 * recorded on the launching stream immediately before and after the op. */
typedef struct sgc_op_profile {
  int32_t kind;      /* 0 coloring, 1 neighbour color histogram, 2 SpMM, 4 eMA,
                        5 final step (single-vertex active child), 6 final step */
  int32_t t, a, p;   /* sub-template sizes |T_s|, |T_a|, |T_p| */
  int32_t batch;     /* colorings per pass */
  int64_t passes;    /* passes recorded */
  int64_t kernels;   /* kernel launches in those passes */
  double ms;         /* summed device time */
  double bytes;      /* algorithmic bytes of one pass: every table read or written once,
                        CSR read once per column tile */
  double flops;      /* multiplies + adds of one pass (eMA and final step) */
  double gather_bytes; /* SpMM and histogram: bytes of the neighbour rows gathered in one pass
                          (every stored entry's row once, nnz * row bytes), served by L2 and HBM */
  int32_t k;           /* colors of the count the op belongs to (ops of different templates with the
                          same sizes are kept apart) */
} sgc_op_profile;

/* Turn event recording around every op on (1) or off (0); turning it on
 * discards earlier records.  Adds two event records per op to each pass. */
sgc_status sgc_profile_enable(const sgc_graph* g, int32_t on);

/* Wait for the recorded events, then copy up to `cap` aggregated entries to
 * `out` (host) and their number to *n; records are cleared. */
sgc_status sgc_profile_read(const sgc_graph* g, sgc_op_profile* out, int32_t cap, int32_t* n);

#ifdef __cplusplus
}
#endif

#endif /* SGC_H */
