/*
 * sgcgen.c - seeded synthetic inputs for the subgraph-counting tests and
 * benchmarks: simple undirected graphs in CSR form and tree templates as
 * parent arrays.
 *
 * This file holds input generation only.  It contains none of the counting
 * method's arithmetic (no coloring, no color-set index, no dynamic program),
 * so both the CPU oracle and the CUDA library can be fed from it without
 * sharing any of the method's code.
 *
 * Random numbers come from the SplitMix64 generator (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): the j-th
 * output of the stream with key `seed` is mix(seed + (j+1)*0x9E3779B97F4A7C15)
 * with the published 64-bit finaliser below.  Everything is integer
 * arithmetic, so x86-64 and aarch64 produce identical graphs.
 *
 * Generators:
 *   - R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): 2^scale * ef edge
 *     samples, quadrant probabilities a,b,c,(d) given as 32-bit fixed-point
 *     thresholds, no noise and no vertex permutation; symmetrised, self-loops
 *     and duplicates removed.
 *   - Erdos-Renyi G(n, m): m distinct unordered non-loop pairs.
 *   - Pruefer-sequence random labelled trees (uniform over labelled trees),
 *     decoded smallest-leaf-first and rooted at vertex 0 by BFS.
 *
 * CSR outputs are malloc'd here and released with sgcgen_free().  Rows are
 * sorted ascending, there are no self-loops and no duplicate entries, and
 * the adjacency is symmetric.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SGCGEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gen_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* j-th SplitMix64 output of the stream keyed by `seed`. */
static inline uint64_t gen_draw(uint64_t seed, uint64_t j) {
  return gen_mix(seed + (j + 1) * SGCGEN_GAMMA);
}

/* uniform integer in [0, bound) from the high 32 bits of a draw */
static inline uint32_t gen_below(uint64_t r, uint32_t bound) {
  return (uint32_t)(((r >> 32) * (uint64_t)bound) >> 32);
}

void sgcgen_free(void* p) { free(p); }

uint64_t sgcgen_splitmix64_draw(uint64_t seed, uint64_t j) { return gen_draw(seed, j); }

/* ---- LSD radix sort of 64-bit keys (16-bit digits), stable ------------- */
static int radix_sort_u64(uint64_t* keys, int64_t n, int nbits) {
  if (n <= 1) return 0;
  uint64_t* tmp = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
  if (!tmp) return -1;
  int64_t* count = (int64_t*)malloc(65536 * sizeof(int64_t));
  if (!count) { free(tmp); return -1; }
  uint64_t* src = keys;
  uint64_t* dst = tmp;
  int passes = 0;
  for (int shift = 0; shift < nbits; shift += 16) {
    memset(count, 0, 65536 * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) count[(src[i] >> shift) & 0xFFFF]++;
    int64_t run = 0;
    for (int d = 0; d < 65536; ++d) { int64_t c = count[d]; count[d] = run; run += c; }
    for (int64_t i = 0; i < n; ++i) dst[count[(src[i] >> shift) & 0xFFFF]++] = src[i];
    uint64_t* t = src; src = dst; dst = t;
    ++passes;
  }
  if (passes & 1) memcpy(keys, src, (size_t)n * sizeof(uint64_t));
  free(tmp);
  free(count);
  return 0;
}

/*
 * Build a symmetric CSR from `m` undirected pairs packed as (u << 32 | v)
 * (u != v, any order, duplicates allowed).  Consumes `pairs` (freed).
 */
static int csr_from_pairs(uint64_t* pairs, int64_t m, int32_t n,
                          int32_t** row_ptr_out, int32_t** col_idx_out, int64_t* nnz_out) {
  uint64_t* keys = (uint64_t*)malloc((size_t)(2 * m + 1) * sizeof(uint64_t));
  if (!keys) { free(pairs); return -1; }
  for (int64_t i = 0; i < m; ++i) {
    uint64_t u = pairs[i] >> 32, v = pairs[i] & 0xFFFFFFFFULL;
    keys[2 * i] = (u << 32) | v;
    keys[2 * i + 1] = (v << 32) | u;
  }
  free(pairs);
  int64_t nk = 2 * m;
  /* sort by (row, col): column digits first, then row digits */
  if (radix_sort_u64(keys, nk, 64) != 0) { free(keys); return -1; }
  int64_t w = 0;
  for (int64_t i = 0; i < nk; ++i) {
    if (w > 0 && keys[w - 1] == keys[i]) continue;
    keys[w++] = keys[i];
  }
  int32_t* row_ptr = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t* col_idx = (int32_t*)malloc((size_t)(w > 0 ? w : 1) * sizeof(int32_t));
  if (!row_ptr || !col_idx) { free(keys); free(row_ptr); free(col_idx); return -1; }
  for (int64_t i = 0; i < w; ++i) {
    row_ptr[(keys[i] >> 32) + 1]++;
    col_idx[i] = (int32_t)(keys[i] & 0xFFFFFFFFULL);
  }
  for (int32_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
  free(keys);
  *row_ptr_out = row_ptr;
  *col_idx_out = col_idx;
  *nnz_out = w;
  return 0;
}

/*
 * R-MAT graph with 2^scale vertices and 2^scale*edge_factor edge samples;
 * sample i picks one quadrant per level, level l using draw i*scale + l.
 * thr_a, thr_ab, thr_abc are cumulative probabilities a, a+b, a+b+c scaled
 * to 2^32.  Returns 0 on success.
 */
int sgcgen_rmat(int32_t scale, int64_t edge_factor, uint64_t thr_a, uint64_t thr_ab,
                uint64_t thr_abc, uint64_t seed, int32_t** row_ptr, int32_t** col_idx,
                int64_t* nnz) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return -2;
  int32_t n = (int32_t)1 << scale;
  int64_t samples = (int64_t)n * edge_factor;
  uint64_t* pairs = (uint64_t*)malloc((size_t)samples * sizeof(uint64_t));
  if (!pairs) return -1;
  int64_t m = 0;
  for (int64_t i = 0; i < samples; ++i) {
    uint64_t u = 0, v = 0;
    for (int32_t l = 0; l < scale; ++l) {
      uint64_t r = gen_draw(seed, (uint64_t)i * (uint64_t)scale + (uint64_t)l) >> 32;
      uint64_t bit = (uint64_t)1 << (scale - 1 - l);
      if (r < thr_a) {
      } else if (r < thr_ab) {
        v |= bit;
      } else if (r < thr_abc) {
        u |= bit;
      } else {
        u |= bit;
        v |= bit;
      }
    }
    if (u == v) continue;
    pairs[m++] = (u << 32) | v;
  }
  return csr_from_pairs(pairs, m, n, row_ptr, col_idx, nnz);
}

/* open-addressing set of nonzero 64-bit keys */
typedef struct { uint64_t* slot; uint64_t mask; } keyset;

static int keyset_insert(keyset* s, uint64_t key) {
  uint64_t h = gen_mix(key) & s->mask;
  while (s->slot[h] != 0) {
    if (s->slot[h] == key) return 0;
    h = (h + 1) & s->mask;
  }
  s->slot[h] = key;
  return 1;
}

/*
 * Erdos-Renyi G(n, m): draw j gives the ordered pair (hi32 -> u, lo32 -> v)
 * scaled to [0, n); loops and repeats are skipped until m distinct unordered
 * pairs are accepted.
 */
int sgcgen_er(int32_t n, int64_t m, uint64_t seed, int32_t** row_ptr, int32_t** col_idx,
              int64_t* nnz) {
  if (n < 2 || m < 0 || m > (int64_t)n * (n - 1) / 2) return -2;
  uint64_t cap = 16;
  while (cap < (uint64_t)(2 * m + 16)) cap <<= 1;
  keyset s;
  s.slot = (uint64_t*)calloc(cap, sizeof(uint64_t));
  s.mask = cap - 1;
  uint64_t* pairs = (uint64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
  if (!s.slot || !pairs) { free(s.slot); free(pairs); return -1; }
  int64_t got = 0;
  for (uint64_t j = 0; got < m; ++j) {
    uint64_t r = gen_draw(seed, j);
    uint64_t u = ((r >> 32) * (uint64_t)n) >> 32;
    uint64_t v = ((r & 0xFFFFFFFFULL) * (uint64_t)n) >> 32;
    if (u == v) continue;
    uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
    /* +1 keeps the key nonzero for the empty-slot convention */
    if (keyset_insert(&s, ((lo << 32) | hi) + 1)) pairs[got++] = (lo << 32) | hi;
  }
  free(s.slot);
  return csr_from_pairs(pairs, m, n, row_ptr, col_idx, nnz);
}

/* CSR from an explicit list of undirected edges (eu[i], ev[i]). */
int sgcgen_from_edges(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                      int32_t** row_ptr, int32_t** col_idx, int64_t* nnz) {
  if (n < 0 || m < 0) return -2;
  uint64_t* pairs = (uint64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
  if (!pairs) return -1;
  int64_t w = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (eu[i] < 0 || ev[i] < 0 || eu[i] >= n || ev[i] >= n) { free(pairs); return -2; }
    if (eu[i] == ev[i]) continue;
    pairs[w++] = ((uint64_t)eu[i] << 32) | (uint64_t)ev[i];
  }
  return csr_from_pairs(pairs, w, n, row_ptr, col_idx, nnz);
}

/*
 * Uniform random labelled tree on k vertices from a Pruefer sequence of
 * length k-2 (entry i = draw i scaled to [0,k)).  Decoding joins, for each
 * sequence entry x in turn, the smallest current leaf to x; the last two
 * remaining vertices are joined at the end.  The tree is rooted at vertex 0
 * and returned as a parent array (parent[0] = -1) built by BFS.
 */
int sgcgen_pruefer_tree(int32_t k, uint64_t seed, int32_t* parent) {
  if (k < 1 || k > 64) return -2;
  int32_t eu[64], ev[64], deg[64], seq[64];
  int32_t ne = 0;
  if (k == 1) { parent[0] = -1; return 0; }
  for (int32_t i = 0; i < k; ++i) deg[i] = 1;
  for (int32_t i = 0; i < k - 2; ++i) {
    seq[i] = (int32_t)gen_below(gen_draw(seed, (uint64_t)i), (uint32_t)k);
    deg[seq[i]]++;
  }
  for (int32_t i = 0; i < k - 2; ++i) {
    int32_t leaf = 0;
    while (deg[leaf] != 1) ++leaf;
    eu[ne] = leaf; ev[ne] = seq[i]; ++ne;
    deg[leaf]--; deg[seq[i]]--;
  }
  int32_t a = -1, b = -1;
  for (int32_t i = 0; i < k; ++i) {
    if (deg[i] == 1) { if (a < 0) a = i; else b = i; }
  }
  eu[ne] = a; ev[ne] = b; ++ne;
  /* BFS from 0 */
  int32_t queue[64], head = 0, tail = 0;
  for (int32_t i = 0; i < k; ++i) parent[i] = -2;
  parent[0] = -1;
  queue[tail++] = 0;
  while (head < tail) {
    int32_t x = queue[head++];
    for (int32_t e = 0; e < ne; ++e) {
      int32_t y = -1;
      if (eu[e] == x) y = ev[e]; else if (ev[e] == x) y = eu[e];
      if (y >= 0 && parent[y] == -2) { parent[y] = x; queue[tail++] = y; }
    }
  }
  for (int32_t i = 0; i < k; ++i) if (parent[i] == -2) return -3;
  return 0;
}
