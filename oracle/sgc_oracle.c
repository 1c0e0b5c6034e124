/*
 * sgc_oracle.c - TEST INFRASTRUCTURE ONLY.  The exact CPU oracle for
 * color-coding tree counting ("A GraphBLAS Approach for Subgraph Counting",
 * Chen et al., HPDC'19).  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this code; the CUDA library never does,
 * and the two share no source.
 *
 * What it computes, following the paper's Section 2.1 (color coding):
 *
 *   1. Random coloring: vertex v gets color
 *        c(v) = floor(hi32(x_v) * k / 2^32),  x_v = SplitMix64 output number v
 *      of the stream keyed by the coloring seed (SplitMix64 as published by
 *      Steele, Lea and Flood, OOPSLA 2014).  The paper only asks for a
 *      uniform color in [0, k); this counter-based draw is the reading used
 *      everywhere in this project.  Explicit colors can be passed instead.
 *   2. Template partitioning (Section 2.1, item 2): a root rho is chosen, the
 *      edge (rho, tau) to rho's first remaining child is cut; the active child
 *      keeps rho, the passive child is the subtree rooted at tau; recurse
 *      until single vertices.  Children are taken in ascending vertex order.
 *   3. Dynamic programming (Section 2.1, item 3), with the sum over color-set
 *      splits made explicit:
 *        N(v, {x}, {c})  = [c(v) == c]
 *        N(v, T_s, C_s)  = sum over C_a subset C_s, |C_a| = |T_a|, C_p = C_s \ C_a
 *                          of N(v, T_a, C_a) * sum_{u in N(v)} N(u, T_p, C_p)
 *      Color sets index the columns of the count tables M_s (n rows,
 *      C(k,|T_s|) columns) by Eq. 1: I(C) = sum_i binom(c_i, i) over the
 *      colors sorted ascending, i = 1..h.
 *      - "pruned" mode evaluates the neighbour sum once per passive column
 *        into a buffer (Eq. 2 and the pre-computed neighbour traversal of
 *        Section 4.2), i.e. P = A * M_p, and then does the split sums.
 *      - "literal" mode keeps the loop order of the paper's Algorithm 1
 *        (vertex, color set, split, neighbour) with no hoisting; it is only
 *        meant for small inputs and pins Eq. 2.
 *   4. maps = sum_v N(v, T, {0..k-1}): the number of colorful injective
 *      edge-preserving maps T -> G.  copies = maps / |Aut(T)|, and the
 *      estimate of the number of (non-induced) copies is
 *      copies * k^k / k! (Section 2.1, item 1).  With k > |T| colors
 *      (Section 2.1 allows k >= |T|) the maps sum the root table over every
 *      |T|-subset of colors, and the estimate scales by the inverse of the
 *      probability k! / ((k - |T|)! k^|T|) that a fixed copy is colorful.
 *
 * All counts are exact unsigned integers of ORACLE_WORDS 64-bit words: 128
 * bits by default, 192 bits when compiled with -DORACLE_WIDE (a second
 * library the Python side falls back to when a count needs more than 128
 * bits; the paper's Section 7.4 only says floats are used to avoid overflow,
 * and exact counts of 15-vertex trees on R-MAT graphs of 2^16 vertices
 * already exceed 2^128).  Every add and multiply is overflow-checked and an
 * overflow makes the call return ORACLE_OVERFLOW.
 * The largest value seen in any count table, neighbour-sum buffer or the
 * final sum is reported so callers know whether a double-precision
 * computation of the same quantity is exact (all values below 2^53).
 *
 * OpenMP parallelises over vertices; the integer results do not depend on
 * the number of threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ---------------- the count type: exact unsigned, overflow-checked ------- */

#ifdef ORACLE_WIDE
#define ORACLE_WORDS 3
typedef struct { uint64_t w[3]; } cnt_t;  /* little-endian 64-bit limbs */

static inline cnt_t cnt_small(uint64_t x) { cnt_t r = {{x, 0, 0}}; return r; }

/* r = a + b; returns 1 on overflow past 192 bits */
static inline int cnt_add(cnt_t a, cnt_t b, cnt_t* r) {
  u128 c = 0;
  for (int i = 0; i < 3; ++i) {
    c += (u128)a.w[i] + b.w[i];
    r->w[i] = (uint64_t)c;
    c >>= 64;
  }
  return c != 0;
}

/* r = a * b; returns 1 when the exact product needs more than 192 bits */
static inline int cnt_mul(cnt_t a, cnt_t b, cnt_t* r) {
  uint64_t t[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 3; ++i) {
    u128 c = 0;
    for (int j = 0; j < 3; ++j) {
      c += (u128)a.w[i] * b.w[j] + t[i + j];
      t[i + j] = (uint64_t)c;
      c >>= 64;
    }
    t[i + 3] = (uint64_t)c;
  }
  r->w[0] = t[0]; r->w[1] = t[1]; r->w[2] = t[2];
  return (t[3] | t[4] | t[5]) != 0;
}

static inline int cnt_gt(cnt_t a, cnt_t b) {
  for (int i = 2; i >= 0; --i) if (a.w[i] != b.w[i]) return a.w[i] > b.w[i];
  return 0;
}

static inline void cnt_put(cnt_t x, uint64_t* out) { for (int i = 0; i < 3; ++i) out[i] = x.w[i]; }
#else
#define ORACLE_WORDS 2
typedef u128 cnt_t;

static inline cnt_t cnt_small(uint64_t x) { return (cnt_t)x; }
static inline int cnt_add(cnt_t a, cnt_t b, cnt_t* r) { return __builtin_add_overflow(a, b, r); }
static inline int cnt_mul(cnt_t a, cnt_t b, cnt_t* r) { return __builtin_mul_overflow(a, b, r); }
static inline int cnt_gt(cnt_t a, cnt_t b) { return a > b; }
static inline void cnt_put(cnt_t x, uint64_t* out) { out[0] = (uint64_t)x; out[1] = (uint64_t)(x >> 64); }
#endif

#define ORACLE_OK 0
#define ORACLE_OVERFLOW 1
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

#define ORACLE_MAXK 20

/* ---------------- coloring (SplitMix64, published definition) ----------- */

static uint64_t oracle_splitmix64(uint64_t seed, uint64_t j) {
  uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int oracle_color(uint64_t seed, int32_t n, int32_t k, uint8_t* colors) {
  if (n < 0 || k < 1 || k > ORACLE_MAXK) return ORACLE_EINVAL;
  for (int32_t v = 0; v < n; ++v) {
    uint64_t x = oracle_splitmix64(seed, (uint64_t)v);
    colors[v] = (uint8_t)(((x >> 32) * (uint64_t)k) >> 32);
  }
  return ORACLE_OK;
}

/* ---------------- binomials and the Eq. 1 color-set index --------------- */

static uint64_t binom_tab[ORACLE_MAXK + 2][ORACLE_MAXK + 2];

static void init_binom(void) {
  for (int a = 0; a <= ORACLE_MAXK + 1; ++a) {
    for (int b = 0; b <= ORACLE_MAXK + 1; ++b) {
      if (b == 0) binom_tab[a][b] = 1;
      else if (a == 0) binom_tab[a][b] = 0;
      else binom_tab[a][b] = binom_tab[a - 1][b - 1] + binom_tab[a - 1][b];
    }
  }
}

static uint64_t binom(int a, int b) {
  if (b < 0 || a < 0 || b > a) return 0;
  return binom_tab[a][b];
}

/* Eq. 1: colors c[0] < c[1] < ... < c[h-1]; index = sum binom(c_i, i), i 1-based */
static int64_t colorset_index(const int* c, int h) {
  int64_t idx = 0;
  for (int i = 0; i < h; ++i) idx += (int64_t)binom(c[i], i + 1);
  return idx;
}

/* inverse of Eq. 1: fill c[0..h-1] ascending */
static void colorset_unindex(int64_t idx, int h, int k, int* c) {
  int top = k - 1;
  for (int i = h; i >= 1; --i) {
    int x = top;
    while ((int64_t)binom(x, i) > idx) --x;
    c[i - 1] = x;
    idx -= (int64_t)binom(x, i);
    top = x - 1;
  }
}

int64_t oracle_colorset_index(const int32_t* colors, int32_t h) {
  int c[ORACLE_MAXK];
  if (h < 0 || h > ORACLE_MAXK) return -1;
  init_binom();
  for (int i = 0; i < h; ++i) c[i] = colors[i];
  return colorset_index(c, h);
}

int oracle_colorset_unindex(int64_t idx, int32_t h, int32_t k, int32_t* colors) {
  int c[ORACLE_MAXK];
  if (h < 0 || h > k || k > ORACLE_MAXK) return ORACLE_EINVAL;
  init_binom();
  if (idx < 0 || idx >= (int64_t)binom(k, h)) return ORACLE_EINVAL;
  colorset_unindex(idx, h, k, c);
  for (int i = 0; i < h; ++i) colors[i] = c[i];
  return ORACLE_OK;
}

/* ---------------- count tables ------------------------------------------- */

typedef struct {
  int32_t size;   /* |T_s| */
  int64_t ncols;  /* binom(k, size) */
  cnt_t* m;       /* n x ncols, row-major: m[v * ncols + I] */
} table;

typedef struct {
  int32_t n, k;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const uint8_t* colors;
  int mode; /* 0 pruned, 1 literal */
  /* template, rooted */
  int32_t nchild[ORACLE_MAXK];
  int32_t child[ORACLE_MAXK][ORACLE_MAXK];
  int32_t subsize[ORACLE_MAXK];
  int status;
  cnt_t max_seen;
} dp_ctx;

static void note_max(dp_ctx* ctx, const cnt_t* a, int64_t len) {
  cnt_t mx = cnt_small(0);
  for (int64_t i = 0; i < len; ++i) if (cnt_gt(a[i], mx)) mx = a[i];
  if (cnt_gt(mx, ctx->max_seen)) ctx->max_seen = mx;
}

/* leaf table of a single template vertex: N(v,{x},{c}) = [c(v) == c] */
static int make_leaf(dp_ctx* ctx, table* out) {
  out->size = 1;
  out->ncols = ctx->k;
  out->m = (cnt_t*)calloc((size_t)ctx->n * (size_t)ctx->k, sizeof(cnt_t));
  if (!out->m && ctx->n > 0) return ORACLE_ENOMEM;
  for (int32_t v = 0; v < ctx->n; ++v) out->m[(int64_t)v * ctx->k + ctx->colors[v]] = cnt_small(1);
  if (ctx->n > 0) note_max(ctx, out->m, (int64_t)ctx->n * ctx->k);
  return ORACLE_OK;
}

/*
 * Split list for |T_s| = t, |T_a| = a: for every color set C_s (by index I_s)
 * all pairs (I(C_a), I(C_s \ C_a)) with |C_a| = a, enumerated by bitmask over
 * the positions of C_s.
 */
typedef struct { int64_t nsplit; int64_t* ia; int64_t* ip; } splits;

static int make_splits(int k, int t, int a, splits* s) {
  int64_t cs = (int64_t)binom(k, t);
  s->nsplit = (int64_t)binom(t, a);
  s->ia = (int64_t*)malloc((size_t)(cs * s->nsplit) * sizeof(int64_t));
  s->ip = (int64_t*)malloc((size_t)(cs * s->nsplit) * sizeof(int64_t));
  if (!s->ia || !s->ip) { free(s->ia); free(s->ip); return ORACLE_ENOMEM; }
  int c[ORACLE_MAXK], ca[ORACLE_MAXK], cp[ORACLE_MAXK];
  for (int64_t is = 0; is < cs; ++is) {
    colorset_unindex(is, t, k, c);
    int64_t j = 0;
    for (uint32_t mask = 0; mask < (1u << t); ++mask) {
      if (__builtin_popcount(mask) != a) continue;
      int na = 0, np = 0;
      for (int i = 0; i < t; ++i) {
        if (mask & (1u << i)) ca[na++] = c[i]; else cp[np++] = c[i];
      }
      s->ia[is * s->nsplit + j] = colorset_index(ca, na);
      s->ip[is * s->nsplit + j] = colorset_index(cp, np);
      ++j;
    }
  }
  return ORACLE_OK;
}

/* combine active child table `ma` and passive child table `mp` into `out` */
static int combine(dp_ctx* ctx, const table* ma, const table* mp, table* out) {
  const int32_t n = ctx->n, k = ctx->k;
  const int t = ma->size + mp->size;
  splits s;
  int rc = make_splits(k, t, ma->size, &s);
  if (rc != ORACLE_OK) return rc;
  out->size = t;
  out->ncols = (int64_t)binom(k, t);
  out->m = (cnt_t*)calloc((size_t)n * (size_t)out->ncols + 1, sizeof(cnt_t));
  if (!out->m) { free(s.ia); free(s.ip); return ORACLE_ENOMEM; }
  const int64_t ca = ma->ncols, cp = mp->ncols, cs = out->ncols, ns = s.nsplit;
  int ovf = 0;

  if (ctx->mode == 0) {
    /* pruned: P(v, I_p) = sum_{u in N(v)} M_p(u, I_p), once per passive column */
    cnt_t* P = (cnt_t*)calloc((size_t)n * (size_t)cp + 1, sizeof(cnt_t));
    if (!P) { free(s.ia); free(s.ip); return ORACLE_ENOMEM; }
#pragma omp parallel for schedule(dynamic, 256) reduction(| : ovf)
    for (int32_t v = 0; v < n; ++v) {
      for (int64_t ip = 0; ip < cp; ++ip) {
        cnt_t acc = cnt_small(0);
        for (int32_t e = ctx->row_ptr[v]; e < ctx->row_ptr[v + 1]; ++e) {
          int32_t u = ctx->col_idx[e];
          ovf |= cnt_add(acc, mp->m[(int64_t)u * cp + ip], &acc);
        }
        P[(int64_t)v * cp + ip] = acc;
      }
    }
    if (n > 0) note_max(ctx, P, (int64_t)n * cp);
#pragma omp parallel for schedule(dynamic, 256) reduction(| : ovf)
    for (int32_t v = 0; v < n; ++v) {
      for (int64_t is = 0; is < cs; ++is) {
        cnt_t acc = cnt_small(0);
        for (int64_t j = 0; j < ns; ++j) {
          cnt_t prod;
          ovf |= cnt_mul(ma->m[(int64_t)v * ca + s.ia[is * ns + j]], P[(int64_t)v * cp + s.ip[is * ns + j]], &prod);
          ovf |= cnt_add(acc, prod, &acc);
        }
        out->m[(int64_t)v * cs + is] = acc;
      }
    }
    free(P);
  } else {
    /* literal: vertex -> color set -> split -> neighbour, no hoisting */
#pragma omp parallel for schedule(dynamic, 64) reduction(| : ovf)
    for (int32_t v = 0; v < n; ++v) {
      for (int64_t is = 0; is < cs; ++is) {
        cnt_t acc = cnt_small(0);
        for (int64_t j = 0; j < ns; ++j) {
          const cnt_t a_val = ma->m[(int64_t)v * ca + s.ia[is * ns + j]];
          const int64_t ip = s.ip[is * ns + j];
          for (int32_t e = ctx->row_ptr[v]; e < ctx->row_ptr[v + 1]; ++e) {
            int32_t u = ctx->col_idx[e];
            cnt_t prod;
            ovf |= cnt_mul(a_val, mp->m[(int64_t)u * cp + ip], &prod);
            ovf |= cnt_add(acc, prod, &acc);
          }
        }
        out->m[(int64_t)v * cs + is] = acc;
      }
    }
  }
  free(s.ia);
  free(s.ip);
  if (ovf) return ORACLE_OVERFLOW;
  if (n > 0) note_max(ctx, out->m, (int64_t)n * cs);
  return ORACLE_OK;
}

/* table of the sub-template made of x and the subtrees of its children j.. */
static int subtemplate_table(dp_ctx* ctx, int32_t x, int32_t j, table* out) {
  if (j == ctx->nchild[x]) return make_leaf(ctx, out);
  table ta, tp;
  int rc = subtemplate_table(ctx, x, j + 1, &ta);           /* active child, keeps x */
  if (rc != ORACLE_OK) return rc;
  rc = subtemplate_table(ctx, ctx->child[x][j], 0, &tp);    /* passive child, rooted at tau */
  if (rc != ORACLE_OK) { free(ta.m); return rc; }
  rc = combine(ctx, &ta, &tp, out);
  free(ta.m);
  free(tp.m);
  return rc;
}

static int32_t subtree_size(dp_ctx* ctx, int32_t x) {
  int32_t s = 1;
  for (int32_t j = 0; j < ctx->nchild[x]; ++j) s += subtree_size(ctx, ctx->child[x][j]);
  return ctx->subsize[x] = s;
}

/* parent array -> rooted children lists (ascending order) for root `root` */
static int root_template(dp_ctx* ctx, int32_t k, const int32_t* parent, int32_t root) {
  int32_t adj[ORACLE_MAXK][ORACLE_MAXK], deg[ORACLE_MAXK];
  int32_t nroot = 0;
  memset(deg, 0, sizeof(deg));
  for (int32_t i = 0; i < k; ++i) {
    if (parent[i] < 0) { ++nroot; if (parent[i] != -1) return ORACLE_EINVAL; continue; }
    if (parent[i] >= k || parent[i] == i) return ORACLE_EINVAL;
    adj[i][deg[i]++] = parent[i];
    adj[parent[i]][deg[parent[i]]++] = i;
  }
  if (nroot != 1) return ORACLE_EINVAL;
  if (root < 0) { for (int32_t i = 0; i < k; ++i) if (parent[i] == -1) root = i; }
  if (root >= k) return ORACLE_EINVAL;
  /* BFS from root; children sorted ascending because adjacency is scanned per vertex */
  int32_t seen[ORACLE_MAXK], queue[ORACLE_MAXK], head = 0, tail = 0;
  memset(seen, 0, sizeof(seen));
  seen[root] = 1;
  queue[tail++] = root;
  for (int32_t i = 0; i < k; ++i) ctx->nchild[i] = 0;
  while (head < tail) {
    int32_t x = queue[head++];
    int32_t tmp[ORACLE_MAXK], nt = 0;
    for (int32_t e = 0; e < deg[x]; ++e) if (!seen[adj[x][e]]) tmp[nt++] = adj[x][e];
    for (int32_t a = 1; a < nt; ++a)
      for (int32_t b = a; b > 0 && tmp[b - 1] > tmp[b]; --b) { int32_t q = tmp[b]; tmp[b] = tmp[b - 1]; tmp[b - 1] = q; }
    for (int32_t e = 0; e < nt; ++e) {
      seen[tmp[e]] = 1;
      ctx->child[x][ctx->nchild[x]++] = tmp[e];
      queue[tail++] = tmp[e];
    }
  }
  if (tail != k) return ORACLE_EINVAL; /* not connected: not a tree */
  subtree_size(ctx, root);
  return root;
}


/*
 * Colorful maps of the tree `parent` (t vertices, parent[root] = -1) into the
 * graph (CSR, n vertices) under `colors` (values in [0, ncolors), ncolors >= t:
 * Section 2.1 draws colors from k >= |T|).  A map is colorful when its t
 * images have t distinct colors; the DP runs over color sets of the ncolors
 * colors and the result sums the root table over every t-subset:
 *   maps = sum_v sum_{C, |C| = t} N(v, T, C).
 *   mode: 0 = pruned (neighbour sums hoisted, Eq. 2), 1 = literal (Algorithm 1 order)
 *   root: template vertex used as the DP root, or -1 for parent's root
 *   maps_out[ORACLE_WORDS]: maps, 64-bit words, least significant first
 *   max_out[ORACLE_WORDS]:  largest value held in any table, buffer or the final sum
 *   per_vertex:  NULL, or n x ORACLE_WORDS uint64 receiving sum_C N(v, T, C)
 * Returns ORACLE_OK, ORACLE_OVERFLOW, ORACLE_EINVAL or ORACLE_ENOMEM.
 */
int oracle_count_colors(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t t, int32_t ncolors,
                        const int32_t* parent, const uint8_t* colors, int32_t mode, int32_t root,
                        uint64_t* maps_out, uint64_t* max_out, uint64_t* per_vertex) {
  if (n < 0 || t < 1 || t > ORACLE_MAXK || ncolors < t || ncolors > ORACLE_MAXK || (mode != 0 && mode != 1))
    return ORACLE_EINVAL;
  for (int32_t v = 0; v < n; ++v) if (colors[v] >= ncolors) return ORACLE_EINVAL;
  init_binom();
  dp_ctx ctx;
  memset(&ctx, 0, sizeof(ctx));
  ctx.n = n; ctx.k = ncolors; ctx.row_ptr = row_ptr; ctx.col_idx = col_idx;
  ctx.colors = colors; ctx.mode = mode;
  int32_t r = root_template(&ctx, t, parent, root);
  if (r < 0) return ORACLE_EINVAL;
  table full;
  int rc = subtemplate_table(&ctx, r, 0, &full);
  if (rc != ORACLE_OK) return rc;
  /* full.ncols == binom(ncolors, t): 1 when ncolors == t */
  cnt_t maps = cnt_small(0);
  int ovf = 0;
  for (int32_t v = 0; v < n; ++v) {
    cnt_t row = cnt_small(0);
    for (int64_t i = 0; i < full.ncols; ++i) ovf |= cnt_add(row, full.m[(int64_t)v * full.ncols + i], &row);
    ovf |= cnt_add(maps, row, &maps);
    if (cnt_gt(row, ctx.max_seen)) ctx.max_seen = row;
    if (per_vertex) cnt_put(row, per_vertex + ORACLE_WORDS * (int64_t)v);
  }
  free(full.m);
  if (ovf) return ORACLE_OVERFLOW;
  if (cnt_gt(maps, ctx.max_seen)) ctx.max_seen = maps;
  cnt_put(maps, maps_out);
  if (max_out) cnt_put(ctx.max_seen, max_out);
  return ORACLE_OK;
}

/*
 * |Aut(T)|: every injective edge-preserving map of a k-vertex tree into
 * itself is an automorphism, and with the identity coloring c(i) = i every
 * such map is colorful, so |Aut(T)| is the DP's maps count of T in T.
 */
/* k colors for a k-vertex tree (Section 2.1 with k = |T|) */
int oracle_count(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t k, const int32_t* parent,
                 const uint8_t* colors, int32_t mode, int32_t root, uint64_t* maps_out, uint64_t* max_out,
                 uint64_t* per_vertex) {
  return oracle_count_colors(n, row_ptr, col_idx, k, k, parent, colors, mode, root, maps_out, max_out, per_vertex);
}

int oracle_automorphisms(int32_t k, const int32_t* parent, uint64_t* aut_out) {
  if (k < 1 || k > ORACLE_MAXK) return ORACLE_EINVAL;
  int32_t deg[ORACLE_MAXK + 1];
  int32_t rp[ORACLE_MAXK + 1], ci[2 * ORACLE_MAXK];
  uint8_t col[ORACLE_MAXK];
  memset(deg, 0, sizeof(deg));
  for (int32_t i = 0; i < k; ++i) {
    if (parent[i] >= 0 && parent[i] < k) { deg[i]++; deg[parent[i]]++; }
  }
  rp[0] = 0;
  for (int32_t i = 0; i < k; ++i) rp[i + 1] = rp[i] + deg[i];
  int32_t fill[ORACLE_MAXK];
  for (int32_t i = 0; i < k; ++i) fill[i] = rp[i];
  for (int32_t i = 0; i < k; ++i) {
    if (parent[i] >= 0 && parent[i] < k) {
      ci[fill[i]++] = parent[i];
      ci[fill[parent[i]]++] = i;
    }
  }
  for (int32_t i = 0; i < k; ++i) col[i] = (uint8_t)i;
  uint64_t maps[ORACLE_WORDS];
  int rc = oracle_count(k, rp, ci, k, parent, col, 0, -1, maps, NULL, NULL);
  if (rc != ORACLE_OK) return rc;
  for (int i = 1; i < ORACLE_WORDS; ++i) if (maps[i] != 0) return ORACLE_OVERFLOW;
  *aut_out = maps[0];
  return ORACLE_OK;
}

static int oracle_threads_impl(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* 64-bit words of every count this build returns (2, or 3 with -DORACLE_WIDE) */
int oracle_words(void) { return ORACLE_WORDS; }

/* OpenMP threads used by later calls (n >= 1); the previous setting is returned */
int oracle_set_threads(int n) {
  int old = oracle_threads_impl();
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
  return old;
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
