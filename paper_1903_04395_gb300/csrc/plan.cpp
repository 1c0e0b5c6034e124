// plan.cpp - host-side planning for libsgc.
//
// * Eq. 1 color-set index (ColorIndex).
// * |Aut(T)| by canonical forms of rooted trees (AHU encoding).
// * Template partitioning (Section 2.1, item 2): a root rho is chosen and the
//   edge (rho, tau) to one child is cut; the active child keeps rho, the
//   passive child is the subtree at tau; recurse to single vertices.  Each
//   sub-template is identified by its rooted canonical form, so isomorphic
//   sub-templates (for example the equal legs of a spider) share one count
//   table and one SpMM.  Root and cut order are chosen by a cost model built
//   on Lemma 1: per step alpha*|E|*C(k,|T_p|) + beta*|V|*C(k,|T_s|)*C(|T_s|,|T_p|).
// * Index tables for the eMA split sums (Algorithm 4's eMA over all splits of
//   a color set) and the final vertex reduction.
// * Workspace layout: every buffer's lifetime in op order and a first-fit
//   placement in one device arena.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "sgc_internal.h"

namespace sgc {

ColorIndex::ColorIndex(int k_) : k(k_) {
  for (int a = 0; a <= SGC_MAX_K + 1; ++a) {
    binom[a][0] = 1;
    for (int b = 1; b <= a; ++b) binom[a][b] = binom[a - 1][b - 1] + (b <= a - 1 ? binom[a - 1][b] : 0);
  }
}

uint32_t ColorIndex::rank_mask(uint32_t mask) const {
  // walk the colors upward; the i-th present color c contributes binom(c, i)
  uint64_t r = 0;
  int i = 0;
  for (int c = 0; c < k; ++c) {
    if (mask >> c & 1u) {
      ++i;
      r += (c >= i) ? binom[c][i] : 0;
    }
  }
  return (uint32_t)r;
}

uint32_t ColorIndex::unrank_mask(uint64_t r, int h) const {
  uint32_t mask = 0;
  int c = k - 1;
  for (int i = h; i >= 1; --i) {
    // largest c with binom(c, i) <= r
    while (c >= i && binom[c][i] > r) --c;
    if (c < i) c = i - 1;  // binom(i-1, i) = 0
    mask |= 1u << c;
    r -= (c >= i) ? binom[c][i] : 0;
    --c;
  }
  return mask;
}

namespace {

struct Rooted {
  int k = 0, root = 0;
  std::vector<std::vector<int>> children;
  std::vector<int> size;
  std::vector<std::string> canon;  // canonical form of the full subtree at each vertex
};

void root_tree(const sgc_template* t, int root, Rooted* R) {
  R->k = t->k;
  R->root = root;
  R->children.assign(t->k, {});
  R->size.assign(t->k, 1);
  R->canon.assign(t->k, "");
  std::vector<int> order, par(t->k, -2);
  order.push_back(root);
  par[root] = -1;
  for (size_t h = 0; h < order.size(); ++h) {
    int x = order[h];
    for (int y : t->adj[x]) {
      if (par[y] != -2) continue;
      par[y] = x;
      R->children[x].push_back(y);
      order.push_back(y);
    }
  }
  for (int h = (int)order.size() - 1; h >= 0; --h) {
    int x = order[h];
    std::vector<std::string> cs;
    for (int y : R->children[x]) {
      R->size[x] += R->size[y];
      cs.push_back(R->canon[y]);
    }
    std::sort(cs.begin(), cs.end());
    std::string s = "(";
    for (auto& c : cs) s += c;
    s += ")";
    R->canon[x] = s;
  }
}

// automorphisms of the rooted subtree at x
uint64_t rooted_aut(const Rooted& R, int x) {
  uint64_t a = 1;
  std::map<std::string, int> groups;
  for (int y : R.children[x]) {
    a *= rooted_aut(R, y);
    groups[R.canon[y]]++;
  }
  for (auto& kv : groups)
    for (int i = 2; i <= kv.second; ++i) a *= (uint64_t)i;
  return a;
}

}  // namespace

uint64_t automorphisms(const sgc_template* t) {
  const int k = t->k;
  if (k <= 2) return k == 2 ? 2 : 1;
  // centre(s): peel leaves
  std::vector<int> deg(k), alive(k, 1), leaves;
  for (int i = 0; i < k; ++i) {
    deg[i] = (int)t->adj[i].size();
    if (deg[i] <= 1) leaves.push_back(i);
  }
  int remaining = k;
  while (remaining > 2) {
    std::vector<int> next;
    for (int x : leaves) {
      alive[x] = 0;
      --remaining;
      for (int y : t->adj[x])
        if (alive[y] && --deg[y] == 1) next.push_back(y);
    }
    leaves = next;
  }
  std::vector<int> centres;
  for (int i = 0; i < k; ++i)
    if (alive[i]) centres.push_back(i);
  if (centres.size() == 1) {
    Rooted R;
    root_tree(t, centres[0], &R);
    return rooted_aut(R, centres[0]);
  }
  // two centres joined by an edge: split it
  int c1 = centres[0], c2 = centres[1];
  Rooted R;
  root_tree(t, c1, &R);
  // in the tree rooted at c1, c2 is a child; the c1-side excludes c2's subtree
  uint64_t a2 = rooted_aut(R, c2);
  uint64_t a1 = 1;
  std::map<std::string, int> groups;
  std::vector<std::string> cs;
  for (int y : R.children[c1]) {
    if (y == c2) continue;
    a1 *= rooted_aut(R, y);
    groups[R.canon[y]]++;
    cs.push_back(R.canon[y]);
  }
  for (auto& kv : groups)
    for (int i = 2; i <= kv.second; ++i) a1 *= (uint64_t)i;
  std::sort(cs.begin(), cs.end());
  std::string side1 = "(";
  for (auto& c : cs) side1 += c;
  side1 += ")";
  return a1 * a2 * (side1 == R.canon[c2] ? 2 : 1);
}

namespace {

struct Cls {
  std::string key;
  int size = 1;
  int a = -1, p = -1;  // active / passive child classes; -1 for a single vertex
};

struct Builder {
  const Rooted& R;
  int policy;
  std::vector<std::vector<int>> order;  // children of x in cut order
  std::vector<Cls> cls;
  std::map<std::string, int> memo;

  Builder(const Rooted& r, int pol) : R(r), policy(pol) {
    order = R.children;
    for (auto& ch : order) {
      std::sort(ch.begin(), ch.end(), [&](int u, int v) {
        if (R.size[u] != R.size[v]) return policy == 0 ? R.size[u] > R.size[v] : R.size[u] < R.size[v];
        if (R.canon[u] != R.canon[v]) return R.canon[u] < R.canon[v];
        return u < v;
      });
    }
  }

  std::string key_of(int x, int j) const {
    std::vector<std::string> cs;
    for (size_t i = j; i < order[x].size(); ++i) cs.push_back(R.canon[order[x][i]]);
    std::sort(cs.begin(), cs.end());
    std::string s = "(";
    for (auto& c : cs) s += c;
    return s + ")";
  }

  // class of the sub-template made of x and its children order[x][j..]
  int build(int x, int j) {
    std::string key = key_of(x, j);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    Cls c;
    c.key = key;
    if (j < (int)order[x].size()) {
      c.a = build(x, j + 1);
      c.p = build(order[x][j], 0);
      c.size = cls[c.a].size + cls[c.p].size;
    }
    cls.push_back(c);
    memo[key] = (int)cls.size() - 1;
    return (int)cls.size() - 1;
  }
};

int64_t pad_ld(int64_t cols, int elem) {
  const int64_t v = 16 / elem;  // 16-byte rows
  return (cols + v - 1) / v * v;
}

struct TabKey {  // (kind, t, a, eMA rows) of an index table
  int kind, t, a, rows;
  bool operator<(const TabKey& o) const {
    if (kind != o.kind) return kind < o.kind;
    if (t != o.t) return t < o.t;
    if (a != o.a) return a < o.a;
    return rows < o.rows;
  }
};

// eMA block shape: rows staged per block so that both input rows fit in
// shared memory as [column][row] with row stride rows+1; 64 rows (two per
// lane) when possible.
// Rows an eMA block stages: the most that keep a block within 72 KB of shared
// memory (three blocks per SM), else the most that fit at all.
void ema_shape(int64_t ca, int64_t cp, int elem, int smem_cap, int* rows, int* rpl) {
  const int64_t per = (ca + cp) * elem;
  const int cands[] = {64, 32, 16, 8, 4, 2, 1};
  for (int64_t cap : {std::min<int64_t>(72 * 1024, smem_cap), (int64_t)smem_cap}) {
    for (int r : cands) {
      if (per * (r + 1) <= cap) {
        *rows = r;
        *rpl = r == 64 ? 2 : 1;
        return;
      }
    }
  }
  *rows = 0;
  *rpl = 1;
}

}  // namespace

// Where entry j of a neighbour u's row lands in v's SpMM output row (relative
// colors, Eq. 1 ranks), for c(v) = cv and c(u) = cu; all ones when nowhere.
static uint32_t spmm_position(const ColorIndex& cr, int k, int p, int cv, int cu, uint64_t j) {
  if (cu == cv) return 0xFFFFFFFFu;
  const int K = k - 1;
  const uint32_t rel_u = cr.unrank_mask(j, p - 1);
  uint32_t abs_set = 1u << cu;
  for (int x = 0; x < K; ++x)
    if (rel_u >> x & 1u) abs_set |= 1u << (x < cu ? x : x + 1);
  if (abs_set >> cv & 1u) return 0xFFFFFFFFu;
  uint32_t rel_v = 0;
  for (int y = 0; y < k; ++y)
    if (abs_set >> y & 1u) rel_v |= 1u << (y < cv ? y : y - 1);
  return cr.rank_mask(rel_v);
}

// Index tables.  All count tables are stored in relative-color form (see
// make_plan): a row of vertex v is indexed by subsets of the K = k-1 colors
// other than c(v), relabelled 0..K-1 by skipping c(v), and ranked by Eq. 1
// over those K labels.  `ci` ranks subsets of k colors, `cr` of K colors.
static int64_t build_table(const ColorIndex& cr, int k, OpKind kind, int t, int a, std::vector<uint32_t>* tabs,
                           std::map<TabKey, int64_t>* cache, int ema_rows = 0, int64_t ema_ca = 0) {
  TabKey key{(int)kind, t, a, ema_rows};
  auto it = cache->find(key);
  if (it != cache->end()) return it->second;
  const int K = k - 1;
  // align each table to 4 words (the scheduled eMA's to 32: its rounds are 128-byte lines)
  const size_t align = (kind == OP_EMA + 300 || kind == OP_EMA + 400) ? 32 : 4;
  while (tabs->size() % align) tabs->push_back(0);
  int64_t off = (int64_t)tabs->size();
  if (kind == OP_SPMM) {
    // [c_v][c_u][j]: a neighbour u of color c_u holds, at index j, the count for the
    // (p-1)-subset S of the colors other than c_u (relative to c_u).  Its set S + {c_u}
    // lands at this index of v's row (relative to c_v), or nowhere (~0) when c_v is in
    // S + {c_u}: v's P row only keeps sets without c(v).
    const int p = t;
    const uint64_t w_in = cr.nsets(p - 1);
    for (int cv = 0; cv < k; ++cv)
      for (int cu = 0; cu < k; ++cu)
        for (uint64_t j = 0; j < w_in; ++j) tabs->push_back(spmm_position(cr, k, p, cv, cu, j));
  } else if (kind == OP_SPMM + 400) {
    // the same positions in 16-bit entries, lane-major for a = L lanes per coloring:
    // row [c_v][c_u] holds, for each lane jl < L, the entries j = jl + L q (q < nsp,
    // spmm_lane_nsp, padding all ones) contiguously, so a lane reads four at once
    const int p = t, L = a;
    const uint64_t w_in = cr.nsets(p - 1);
    const int64_t nsp = spmm_lane_nsp((int64_t)w_in, L);
    std::vector<uint16_t> h((size_t)(k * k * L * nsp), 0xFFFFu);
    for (int cv = 0; cv < k; ++cv)
      for (int cu = 0; cu < k; ++cu)
        for (uint64_t j = 0; j < w_in; ++j) {
          const uint32_t pos = spmm_position(cr, k, p, cv, cu, j);
          if (pos == 0xFFFFFFFFu) continue;
          const int64_t jl = (int64_t)j % L, q = (int64_t)j / L;
          h[(size_t)(((int64_t)(cv * k + cu) * L + jl) * nsp + q)] = (uint16_t)pos;
        }
    for (size_t i = 0; i < h.size(); i += 2) tabs->push_back((uint32_t)h[i] | (uint32_t)h[i + 1] << 16);
  } else if (kind == OP_SPMM + 600) {
    // unrolled direct SpMM: for each (c_v, c_u) pair and lane position jl < L = 32 / a
    // (a = batch), 16 bytes: byte q = the position of entry j = jl + L q (0xFF = dropped
    // or beyond the row), one 16-byte load per lane and neighbour
    const int p = t, L = 32 / a;
    const uint64_t w_in = cr.nsets(p - 1);
    for (int cv = 0; cv < k; ++cv)
      for (int cu = 0; cu < k; ++cu)
        for (int jl = 0; jl < L; ++jl)
          for (int wd = 0; wd < 4; ++wd) {
            uint32_t w = 0;
            for (int i = 0; i < 4; ++i) {
              const uint64_t j = (uint64_t)jl + (uint64_t)L * (uint64_t)(4 * wd + i);
              const uint32_t pos = j < w_in ? spmm_position(cr, k, p, cv, cu, j) : 0xFFFFFFFFu;
              w |= (pos < 0xFFu ? pos : 0xFFu) << (8 * i);
            }
            tabs->push_back(w);
          }
  } else if (kind == OP_SPMM + 700) {
    // wide direct SpMM: for each (c_v, c_u) pair and lane position jl < L = 32 / a
    // (a = batch), nch chunks of 8 16-bit positions: entry q of the lane's list is
    // j = jl + L q (0xFFFF = dropped or beyond the row)
    const int p = t, L = 32 / a;
    const uint64_t w_in = cr.nsets(p - 1);
    const int64_t nch = spmm_wide_nch(a, (int64_t)w_in);
    for (int cv = 0; cv < k; ++cv)
      for (int cu = 0; cu < k; ++cu)
        for (int jl = 0; jl < L; ++jl)
          for (int64_t c = 0; c < nch; ++c)
            for (int wd = 0; wd < 4; ++wd) {
              uint32_t w = 0;
              for (int i = 0; i < 2; ++i) {
                const uint64_t j = (uint64_t)jl + (uint64_t)L * (uint64_t)(8 * c + 2 * wd + i);
                const uint32_t pos = j < w_in ? spmm_position(cr, k, p, cv, cu, j) : 0xFFFFFFFFu;
                w |= (pos < 0xFFFFu ? pos : 0xFFFFu) << (16 * i);
              }
              tabs->push_back(w);
            }
  } else if (kind == OP_SPMM + 800) {
    // grouped SpMM: 16-bit positions [c_v][c_u][j] for every entry j < w_in of a
    // neighbour's row (0xFFFF = dropped), two per word
    const int p = t;
    const uint64_t w_in = cr.nsets(p - 1);
    std::vector<uint16_t> h((size_t)(k * k * w_in) + 1, 0xFFFFu);
    for (int cv = 0; cv < k; ++cv)
      for (int cu = 0; cu < k; ++cu)
        for (uint64_t j = 0; j < w_in; ++j) {
          const uint32_t pos = spmm_position(cr, k, p, cv, cu, j);
          if (pos != 0xFFFFFFFFu) h[(size_t)((int64_t)(cv * k + cu) * (int64_t)w_in + (int64_t)j)] = (uint16_t)pos;
        }
    for (size_t i = 0; i + 1 < h.size(); i += 2) tabs->push_back((uint32_t)h[i] | (uint32_t)h[i + 1] << 16);
  } else if (kind == OP_SPMM + 900) {
    // staged grouped SpMM: the same 16-bit positions with rows [c_v][c_u] at a pitch of
    // whole 16-byte pieces (8 entries; 0xFFFF past the row), so a row's chunks are copied as is
    const int p = t;
    const uint64_t w_in = cr.nsets(p - 1);
    const uint64_t wp = (uint64_t)spmm_staged_pitch((int64_t)w_in);
    std::vector<uint16_t> h((size_t)(k * k * wp), 0xFFFFu);
    for (int cv = 0; cv < k; ++cv)
      for (int cu = 0; cu < k; ++cu)
        for (uint64_t j = 0; j < w_in; ++j) {
          const uint32_t pos = spmm_position(cr, k, p, cv, cu, j);
          if (pos != 0xFFFFFFFFu) h[(size_t)((int64_t)(cv * k + cu) * (int64_t)wp + (int64_t)j)] = (uint16_t)pos;
        }
    for (size_t i = 0; i < h.size(); i += 2) tabs->push_back((uint32_t)h[i] | (uint32_t)h[i + 1] << 16);
  } else if (kind == OP_SPMM + 500) {
    // unpruned combine: [c_v][I_p][c_u] -> the index, in the passive table row of a
    // neighbour u of color c_u, of the p-set I_p (relative to c_v) minus c_u, or ~0
    // when c_u is not in the set (that neighbour adds nothing to this split)
    const int p = t;
    const uint64_t w = cr.nsets(p);
    for (int cv = 0; cv < k; ++cv)
      for (uint64_t ip = 0; ip < w; ++ip) {
        const uint32_t rel_v = cr.unrank_mask(ip, p);
        uint32_t abs_set = 0;
        for (int x = 0; x < K; ++x)
          if (rel_v >> x & 1u) abs_set |= 1u << (x < cv ? x : x + 1);
        for (int cu = 0; cu < k; ++cu) {
          if (!(abs_set >> cu & 1u)) {
            tabs->push_back(0xFFFFFFFFu);
            continue;
          }
          const uint32_t rest = abs_set & ~(1u << cu);
          uint32_t rel_u = 0;
          for (int y = 0; y < k; ++y)
            if (rest >> y & 1u) rel_u |= 1u << (y < cu ? y : y - 1);
          tabs->push_back(cr.rank_mask(rel_u));
        }
      }
  } else if (kind == OP_SPMM + 300) {
    // the same positions packed into a-byte entries (a = 1 or 2; all ones = nowhere)
    // for a table staged in shared memory: rows [c_v][c_u] of spmm_packed_ld entries
    const int p = t, eb = a;
    const uint64_t w_in = cr.nsets(p - 1);
    const int64_t ld = spmm_packed_ld((int64_t)w_in, eb);
    std::vector<uint8_t> bytes((size_t)(k * k * ld * eb), 0xFF);
    for (int cv = 0; cv < k; ++cv)
      for (int cu = 0; cu < k; ++cu)
        for (uint64_t j = 0; j < w_in; ++j) {
          const uint32_t pos = spmm_position(cr, k, p, cv, cu, j);
          if (pos == 0xFFFFFFFFu) continue;
          const size_t at = (size_t)(((int64_t)(cv * k + cu) * ld + (int64_t)j) * eb);
          bytes[at] = (uint8_t)(pos & 0xffu);
          if (eb == 2) bytes[at + 1] = (uint8_t)(pos >> 8);
        }
    for (size_t i = 0; i < bytes.size(); i += 4)
      tabs->push_back((uint32_t)bytes[i] | (uint32_t)bytes[i + 1] << 8 | (uint32_t)bytes[i + 2] << 16 |
                      (uint32_t)bytes[i + 3] << 24);
  } else if (kind == OP_SPMM + 100) {
    // bucketed SpMM: [c_v][S][t] for the p-subsets S of v's relative colors and the
    // t-th (ascending) element of S: its absolute color c | (the index, relative to c,
    // of S minus that element) << 8.  P(v, S) = sum_t bucket[c_t][j_t], where
    // bucket[c] sums the rows of v's neighbours of color c.
    const int p = t;
    const uint64_t w_out = cr.nsets(p);
    for (int cv = 0; cv < k; ++cv)
      for (uint64_t s = 0; s < w_out; ++s) {
        const uint32_t rel_v = cr.unrank_mask(s, p);
        uint32_t abs_set = 0;
        for (int x = 0; x < K; ++x)
          if (rel_v >> x & 1u) abs_set |= 1u << (x < cv ? x : x + 1);
        for (int c = 0; c < k; ++c) {
          if (!(abs_set >> c & 1u)) continue;
          const uint32_t rest = abs_set & ~(1u << c);
          uint32_t rel_c = 0;
          for (int y = 0; y < k; ++y)
            if (rest >> y & 1u) rel_c |= 1u << (y < c ? y : y - 1);
          tabs->push_back((uint32_t)c | (cr.rank_mask(rel_c) << 8));
        }
      }
  } else if (kind == OP_EMA || kind == OP_EMA + 200) {
    // [j][S]: the j-th split of the (t-1)-subset S of the K relative colors into an
    // (a-1)-subset A (active child, minus the root's own color) and S \ A (passive
    // child), stored as two word offsets into the eMA block's shared memory, which
    // holds the active rows as [I(A)][row] and then the P rows as [I(S \ A)][row],
    // row stride ema_rows + 1.  The symmetric form (a table times itself, |A| = |S \ A|)
    // keeps only the splits with I(A) < I(S \ A); the kernel doubles the sum.
    const bool sym = kind == OP_EMA + 200;
    const int tt = t - 1, aa = a - 1;
    const uint64_t ct = cr.nsets(tt);
    const uint64_t ns = sym ? cr.binom[tt][aa] / 2 : cr.binom[tt][aa];
    const uint32_t rs = (uint32_t)ema_rows + 1;
    std::vector<uint32_t> tab(2 * ns * ct);
    for (uint64_t s = 0; s < ct; ++s) {
      const uint32_t m = cr.unrank_mask(s, tt);
      uint64_t j = 0;
      for (uint32_t sub = m;; sub = (sub - 1) & m) {
        if (__builtin_popcount(sub) == aa) {
          const uint32_t ia = cr.rank_mask(sub), ip = cr.rank_mask(m & ~sub);
          if (!sym || ia < ip) {
            tab[2 * (j * ct + s)] = ia * rs;
            tab[2 * (j * ct + s) + 1] = ((uint32_t)ema_ca + ip) * rs;
            ++j;
          }
        }
        if (sub == 0) break;
      }
    }
    tabs->insert(tabs->end(), tab.begin(), tab.end());
  } else if (kind == OP_EMA + 300 || kind == OP_EMA + 400) {
    // scheduled eMA (k_ema_s, one coloring per pass): outputs in groups of 32 (lane = output), each
    // group's split terms (I(A), I(S \ A)) ordered in rounds so that in every round the 32 lanes read
    // active columns in 32 distinct shared-memory banks and passive columns in 32 distinct banks
    // (the passive row starts `ema_rows` words after the active one: ema_rows carries that offset
    // here; lanes reading the same word share its bank); an idle slot is all ones.  Layout: per group (round offset, rounds), then the rounds,
    // 32 words each (I(A) | I(S \ A) << 16).  OP_EMA + 400: the symmetric form (each unordered split
    // once).  Greedy: every round, lanes with the most terms left pick first, each its first term
    // whose two banks are still free.
    const bool sym = kind == OP_EMA + 400;
    const int tt = t - 1, aa = a - 1;
    const uint32_t pofs = (uint32_t)ema_rows;
    const uint64_t ct = cr.nsets(tt);
    const int64_t G = ((int64_t)ct + 31) / 32;
    std::vector<std::vector<uint32_t>> lists(32);
    std::vector<uint32_t> body;
    std::vector<uint32_t> hdr(2 * (size_t)G);
    for (int64_t gi = 0; gi < G; ++gi) {
      size_t left = 0;
      for (int l = 0; l < 32; ++l) {
        lists[l].clear();
        const uint64_t S = (uint64_t)gi * 32 + (uint64_t)l;
        if (S >= ct) continue;
        const uint32_t m = cr.unrank_mask(S, tt);
        for (uint32_t sub = m;; sub = (sub - 1) & m) {
          if (__builtin_popcount(sub) == aa) {
            const uint32_t ia = cr.rank_mask(sub), ip = cr.rank_mask(m & ~sub);
            if (!sym || ia < ip) lists[l].push_back(ia | ip << 16);
          }
          if (sub == 0) break;
        }
        left += lists[l].size();
      }
      hdr[2 * gi] = (uint32_t)(body.size() / 32);
      uint32_t rounds = 0;
      std::vector<int> order(32);
      while (left > 0) {
        for (int l = 0; l < 32; ++l) order[l] = l;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return lists[x].size() > lists[y].size(); });
        // a bank taken by one word stays free for that same word (lanes reading one word broadcast)
        uint32_t word_a[32], word_p[32];
        for (int l = 0; l < 32; ++l) word_a[l] = word_p[l] = 0xFFFFFFFFu;
        uint32_t slot[32];
        for (int l = 0; l < 32; ++l) slot[l] = 0xFFFFFFFFu;
        for (int l : order) {
          auto& L = lists[l];
          for (size_t i = 0; i < L.size(); ++i) {
            const uint32_t wa = L[i] & 0xFFFFu, wp = pofs + (L[i] >> 16);
            const uint32_t ba = wa & 31u, bp = wp & 31u;
            if ((word_a[ba] != 0xFFFFFFFFu && word_a[ba] != wa) || (word_p[bp] != 0xFFFFFFFFu && word_p[bp] != wp))
              continue;
            word_a[ba] = wa;
            word_p[bp] = wp;
            slot[l] = L[i];
            L.erase(L.begin() + (int64_t)i);
            --left;
            break;
          }
        }
        body.insert(body.end(), slot, slot + 32);
        ++rounds;
      }
      hdr[2 * gi + 1] = rounds;
    }
    tabs->insert(tabs->end(), hdr.begin(), hdr.end());
    while ((tabs->size() - (size_t)off) % 32) tabs->push_back(0);  // rounds start on a 128-byte line
    for (int64_t gi = 0; gi < G; ++gi) (*tabs)[(size_t)off + 2 * gi] += (uint32_t)((tabs->size() - (size_t)off) / 32);
    tabs->insert(tabs->end(), body.begin(), body.end());
  } else if (kind == OP_FINAL) {
    // [I_p]: rank of the complement (among all K relative colors) of the p-subset I_p,
    // an (a-1)-subset: the active child's index for the full color set
    const int p = k - a;
    const uint32_t full = (1u << K) - 1;
    for (uint64_t s = 0; s < cr.nsets(p); ++s) tabs->push_back(cr.rank_mask(full & ~cr.unrank_mask(s, p)));
  }
  (*cache)[key] = off;
  return off;
}

static void place_buffers(Plan* P) {
  // first-fit in address order over buffers sorted by first use
  std::vector<int> idx(P->bufs.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    if (P->bufs[a].first != P->bufs[b].first) return P->bufs[a].first < P->bufs[b].first;
    return P->bufs[a].bytes > P->bufs[b].bytes;
  });
  std::vector<int> placed;
  int64_t top = 0;
  for (int i : idx) {
    PlanBuffer& b = P->bufs[i];
    const int64_t need = (b.bytes + 255) / 256 * 256;
    // collect busy ranges overlapping in time
    std::vector<std::pair<int64_t, int64_t>> busy;
    for (int j : placed) {
      const PlanBuffer& o = P->bufs[j];
      if (o.last < b.first || b.last < o.first) continue;
      busy.push_back({o.offset, o.offset + (o.bytes + 255) / 256 * 256});
    }
    std::sort(busy.begin(), busy.end());
    int64_t off = 0;
    for (auto& r : busy) {
      if (off + need <= r.first) break;
      off = std::max(off, r.second);
    }
    b.offset = off;
    top = std::max(top, off + need);
    placed.push_back(i);
  }
  P->ws_bytes = top;
}

static int add_buf(Plan* P, const std::string& name, int64_t bytes, int op) {
  PlanBuffer b;
  b.name = name;
  b.bytes = std::max<int64_t>(bytes, 16);
  b.first = b.last = op;
  P->bufs.push_back(b);
  return (int)P->bufs.size() - 1;
}

static void use_buf(Plan* P, int buf, int op) {
  if (buf < 0) return;
  P->bufs[buf].first = std::min(P->bufs[buf].first, op);
  P->bufs[buf].last = std::max(P->bufs[buf].last, op);
}

int ema_sched_rows(int64_t ct, int64_t ld_a, int64_t ld_p, bool sym, int elem, int64_t smem_cap, int* upg,
                   int blocks) {
  const int64_t G = (ct + 31) / 32;
  // fewer groups than warps: each group's rounds in W / gcd(G, W) shares, so that the G * shares
  // units divide evenly among the W warps
  const int64_t W = kEmaSchedWarps;
  int64_t gcd = W, x = G % W;
  for (int64_t y = W; x != 0;) {
    const int64_t r = y % x;
    y = x;
    x = r;
    gcd = y;
  }
  *upg = G < W ? (int)(W / gcd) : 1;
  if (ema_sched_rw(ld_a, ld_p, sym) >= 65535) return 0;  // every word of a row has a 16-bit index
  // at most 200 KB of the block's shared memory (under ncu a launch of this kernel that asked for
  // 218 of the 227 KB failed; the plain run of the same program did not); two blocks share an
  // SM's 228 KB less 1 KB reserved per block, and take up to 12 rows each (the 15-vertex tree's
  // (8, 3, 5) combine on R-MAT 21: 25.7 ms at 12 rows and two blocks, 27.5 at 8 rows and one
  // block, 28.1 at 16 rows and one block)
  const int64_t cap = blocks == 2 ? (smem_cap + 1024) / 2 - 1024 : std::min<int64_t>(smem_cap, 200 * 1024);
  for (int r : {12, 8, 6, 4, 2})
    if ((blocks == 2 || r <= 8) && ema_sched_smem(r, ct, ld_a, ld_p, sym, elem, *upg) <= cap) return r;
  return 0;
}

static int64_t smem_cap_of(const sgc_graph* g) { return g->smem_optin > 0 ? g->smem_optin : 227 * 1024; }

// Direct SpMM loop used when no tuned shape says otherwise and the unrolled
// form (11, below) does not apply: 5 = specialised for the batch (20-30%
// faster than the runtime-batch loops on R-MAT 20), 0 = chunked with a runtime
// batch, 1 = next-neighbour prefetch; SGC_SPMM_DIRECT selects 0, 1 or 5 and
// also turns the unrolled default off.
static int default_spmm_variant() {
  static const int v = [] {
    const char* e = std::getenv("SGC_SPMM_DIRECT");
    const int x = e ? std::atoi(e) : 5;
    return x == 0 || x == 1 ? x : 5;
  }();
  return v;
}

// The last step's compile-time form where it is compiled in; SGC_FINAL_TABLE=1
// keeps the table-driven kernel (same results; read when a plan is made).
static bool final_reg_enabled() {
  const char* e = std::getenv("SGC_FINAL_TABLE");
  return !(e && std::atoi(e) == 1);
}

// Bucketed SpMM rows the autotuner may try (the planner's own limit is
// kSpmmBucketMaxBytes): up to 24 KB per warp still keeps 9 warps per SM.
constexpr int64_t kSpmmBucketTuneMaxBytes = 24 * 1024;

// The register-bucket SpMM (one coloring per pass): a row's w_in columns over
// at most 8 warps of 32, 64 or 128 columns, k <= 16 buckets in registers, and
// the rows of a block's buckets in shared memory.
static bool reg_buckets_fit(int batch, int k, int64_t w_in, int elem, const sgc_graph* g) {
  if (batch != 1 || k > 16 || w_in > 1024) return false;
  const int64_t ns = w_in <= 32 ? 1 : w_in <= 512 ? 2 : 4;
  const int64_t wpr = (w_in + 32 * ns - 1) / (32 * ns);
  const int64_t rows = 8 / wpr;
  const int64_t smem_cap = g->smem_optin > 0 ? g->smem_optin : 227 * 1024;
  return rows * k * w_in * elem <= smem_cap;
}

// Bytes of the direct form's packed position table (entries of 1 byte when
// every position and the all-ones marker fit, else 2), or 0 when it is too
// large to stage in shared memory beside the accumulators.
static int64_t spmm_packed_bytes(int k, int64_t w_in, int64_t ld_out) {
  if (ld_out >= 65535) return 0;
  const int eb = ld_out < 255 ? 1 : 2;
  const int64_t bytes = (int64_t)k * k * spmm_packed_ld(w_in, eb) * eb;
  return bytes <= kSpmmPackedMaxBytes ? bytes : 0;
}

// The vertex-tile eMA: batch 4..32, one buffer of (32 / batch) * rpl whole
// vertex rows (both tables unless symmetric) in shared memory.
static bool ema_vertex_fits(int batch, int rpl, int64_t ld_a, int64_t ld_p, bool sym, int elem, int64_t smem_cap) {
  if (batch < 4 || batch > 32) return false;
  auto vs = [&](int64_t ld) { const int64_t x = ld * batch; return x + ((batch - x % 32) % 32 + 32) % 32; };
  const int64_t v = (32 / batch) * rpl;
  return (v * vs(ld_a) + (sym ? 0 : v * vs(ld_p))) * elem <= smem_cap;
}

static int64_t spmm_cols_per_lane(int batch, int64_t cols_p) {
  const int lanes_per_col = 32 / batch;
  return (cols_p + lanes_per_col - 1) / lanes_per_col;
}

// The ablation plan: Algorithm 1's loop order (vertex, color set, split,
// neighbour) with no hoisted neighbour sums - one OP_UNPRUNED op per combine
// reading both children's tables (a single-vertex child's all-ones table is
// implied) - then the root table summed (OP_FINAL_SUM).  Same colors, tables
// and results as the pruned plan; work |E| C(k,t) C(t,p) per step instead of
// |E| C(k,p) + |V| C(k,t) C(t,p) (Lemma 1).
static void plan_unpruned(const sgc_graph* g, const Builder& B, int k, int tk, int batch, bool build_tabs,
                          Plan* P) {
  const int K = k - 1;
  ColorIndex cr(K);
  const int elem = P->elem;
  const int64_t rows = P->rows;
  const double nv = (double)g->n_act, nnz = (double)g->nnz;
  const double bw = 6.0e12;
  std::map<TabKey, int64_t> tcache;
  std::vector<int> table_buf(B.cls.size(), -1), table_state(B.cls.size(), -1);
  std::vector<int64_t> table_ld(B.cls.size(), 1), table_w(B.cls.size(), 1);
  int n_states = 0;
  PlanOp color_op{};
  color_op.kind = OP_COLOR;
  color_op.out = P->buf_colors;
  color_op.alg_bytes = nv * 4 + nv * batch + 8.0 * batch;
  P->ops.push_back(color_op);
  int root_cls = -1;
  for (size_t c = 0; c < B.cls.size(); ++c) {
    const Cls& C = B.cls[c];
    if (C.size == tk) root_cls = (int)c;
    if (C.a < 0) continue;
    const Cls& A = B.cls[C.a];
    const Cls& Pc = B.cls[C.p];
    PlanOp op{};
    op.kind = OP_UNPRUNED;
    op.t = C.size;
    op.a = A.size;
    op.p = Pc.size;
    const int idx = (int)P->ops.size();
    op.in_a = A.a < 0 ? -1 : table_buf[C.a];
    op.state_a = A.a < 0 ? -1 : table_state[C.a];
    op.ld_a = table_ld[C.a];
    op.cols_a = table_w[C.a];
    op.in_p = Pc.a < 0 ? -1 : table_buf[C.p];
    op.state_p = Pc.a < 0 ? -1 : table_state[C.p];
    op.ld_p = table_ld[C.p];
    op.cols_p = (int64_t)cr.nsets(Pc.size);  // p-sets of the split (relative to c_v)
    op.cols_out = (int64_t)cr.nsets(C.size - 1);
    op.ld_out = pad_ld(op.cols_out, elem);
    op.nsplit = (int64_t)cr.binom[C.size - 1][Pc.size];
    op.tab_off = build_tabs ? build_table(cr, k, OP_EMA, C.size, A.size, &P->tabs, &tcache, 0, 0) : 0;
    op.tab2_off = build_tabs ? build_table(cr, k, (OpKind)(OP_SPMM + 500), Pc.size, 0, &P->tabs, &tcache) : 0;
    op.state_out = table_state[c] = n_states++;
    op.out = table_buf[c] = add_buf(P, "U" + std::to_string(c), rows * op.ld_out * elem, idx);
    table_w[c] = op.cols_out;
    table_ld[c] = op.ld_out;
    op.alg_bytes = (double)elem * nv * batch * (double)op.cols_out;
    op.alg_flops = 2.0 * nnz * batch * (double)op.cols_out * (double)op.nsplit;
    P->est_cost += nnz * (double)op.cols_out * (double)op.nsplit * elem / bw;
    P->n_ema++;
    if (op.in_a >= 0) use_buf(P, op.in_a, idx);
    if (op.in_p >= 0) use_buf(P, op.in_p, idx);
    P->ops.push_back(op);
  }
  PlanOp op{};
  op.kind = OP_FINAL_SUM;
  op.t = tk;
  op.in_p = table_buf[root_cls];
  op.state_p = table_state[root_cls];
  op.cols_p = table_w[root_cls];
  op.ld_p = table_ld[root_cls];
  op.out = P->buf_partials;
  op.alg_bytes = (double)elem * nv * batch * (double)op.cols_p;
  use_buf(P, op.in_p, (int)P->ops.size());
  P->ops.push_back(op);
  P->n_states = n_states;
}

// `colors` = number of colors k >= |T| (0: k = |T|).  Section 2.1 draws colors
// from k >= |T|; with k > |T| the root table keeps every (|T|-1)-subset of the
// other colors and the last op sums its entries (OP_FINAL_SUM) instead of
// evaluating the single full color set.
static void plan_for(const sgc_graph* g, const sgc_template* t, int precision, int root, int policy,
                     int batch, bool build_tabs, Plan* P, const std::vector<int>* shapes = nullptr,
                     int colors = 0, int unpruned = 0) {
  Rooted R;
  root_tree(t, root, &R);
  Builder B(R, policy);
  B.build(root, 0);
  const int tk = t->k;                          // template vertices
  const int k = colors > tk ? colors : tk;      // colors
  const int K = k - 1;
  ColorIndex cr(K);

  P->k = k;
  P->t_size = tk;
  P->root = root;
  P->policy = policy;
  P->batch = batch;
  P->precision = precision;
  P->elem = precision == SGC_FP64 ? 8 : 4;
  P->rows = (int64_t)g->n_act * batch;
  P->bufs.clear();
  P->ops.clear();
  P->tabs.clear();
  P->buf_gids = P->buf_gcols = P->buf_gkept = -1;
  const int64_t rows = P->rows;
  const int elem = P->elem;
  const double nv = (double)g->n_act, nnz = (double)g->nnz;
  // widths: a table of a sub-template of size t keeps the (t-1)-subsets of the
  // other colors; P of a passive child of size p keeps its p-subsets
  auto w_table = [&](int size) { return (int64_t)cr.nsets(size - 1); };
  auto w_p = [&](int size) { return (int64_t)cr.nsets(size); };

  // fixed buffers; lifetimes are stretched to the whole pass below
  P->buf_seeds = add_buf(P, "seeds", 8LL * batch, 0);
  P->buf_colors = add_buf(P, "colors", rows, 0);
  P->buf_out = add_buf(P, "out", 8LL * batch, 0);
  P->final_blocks = (4 * std::max(1, g->num_sms) + 31) / 32 * 32;  // multiple of 32: see k_final
  P->buf_partials = add_buf(P, "partials", 8LL * batch * P->final_blocks, 0);

  if (unpruned == 1) {
    plan_unpruned(g, B, k, tk, batch, build_tabs, P);
    P->buf_states = add_buf(P, "states", 8LL * std::max(1, P->n_states), 0);
    P->scratch_width = 0;
    P->buf_scratch = add_buf(P, "spmm_scratch", 16, 0);
    P->buf_hist_heavy = add_buf(P, "hist_heavy", 16, 0);
    const int last = (int)P->ops.size() - 1;
    for (int b : {P->buf_seeds, P->buf_colors, P->buf_out, P->buf_partials, P->buf_states, P->buf_scratch,
                  P->buf_hist_heavy}) {
      P->bufs[b].first = 0;
      P->bufs[b].last = last;
    }
    place_buffers(P);
    return;
  }
  std::vector<int> table_buf(B.cls.size(), -1), pbuf(B.cls.size(), -1);
  std::vector<int> table_state(B.cls.size(), -1), p_state(B.cls.size(), -1);
  std::vector<int64_t> table_w(B.cls.size(), 0), table_ld(B.cls.size(), 0);
  std::map<TabKey, int64_t> tcache;
  int n_states = 0;
  P->n_spmm = P->n_ema = 0;
  P->n_tables = 0;
  P->est_bytes = P->est_spmm_bytes = P->est_fma = P->est_cost = 0;
  int64_t max_spmm_width = 0;
  const double bw = 6.0e12, fma_rate = 4.0e12, gather_factor = 0.25;

  PlanOp color_op{};
  color_op.kind = OP_COLOR;
  color_op.out = P->buf_colors;
  color_op.alg_bytes = nv * 4 + nv * batch + 8.0 * batch;
  P->ops.push_back(color_op);
  P->est_bytes += nv * 5;

  // classes were created in post-order: inputs precede users
  for (size_t c = 0; c < B.cls.size(); ++c) {
    const Cls& C = B.cls[c];
    if (C.a < 0) continue;  // single vertex: implied by the colors
    const Cls& A = B.cls[C.a];
    const Cls& Pc = B.cls[C.p];
    // ---- P for the passive child
    if (pbuf[C.p] < 0) {
      PlanOp op{};
      op.p = Pc.size;
      op.cols_out = w_p(Pc.size);
      op.ld_out = pad_ld(op.cols_out, elem);
      op.state_out = p_state[C.p] = n_states++;
      const int idx = (int)P->ops.size();
      op.out = pbuf[C.p] = add_buf(P, "P" + std::to_string(c), rows * op.ld_out * elem, idx);
      if (Pc.a < 0) {
        op.kind = OP_HIST;
        op.in_p = P->buf_colors;
        op.alg_bytes = 4 * (nv + 1) + 4 * nnz + nv * batch + (double)elem * nv * batch * (double)op.cols_out;
        op.gather_bytes = nnz * (double)batch;  // one color byte per stored entry and coloring
        double by = nnz * 4 + nnz * 1 + nv * (double)op.cols_out * elem;
        P->est_bytes += by;
        P->est_spmm_bytes += by;
        P->est_cost += by / bw;
      } else {
        op.kind = OP_SPMM;
        op.in_p = table_buf[C.p];
        op.cols_p = table_w[C.p];
        op.ld_p = table_ld[C.p];
        op.state_p = table_state[C.p];
        op.spmm_buckets = spmm_bucket_bytes(batch, k, op.cols_p, elem) <= kSpmmBucketMaxBytes;
        op.spmm_variant = op.spmm_buckets ? 7 : default_spmm_variant();
        if (op.spmm_buckets && batch >= 8 && op.ld_out < 65535) {
          // narrow rows at 8+ colorings per pass: the direct form with the lane-major table
          // measured faster than the buckets (R-MAT 20 spider, p = 2: 3.4 vs 4.1 ms)
          op.spmm_buckets = false;
          op.spmm_variant = 6;
        }
        if ((batch == 4 || batch == 8) && spmm_unrolled_fits(batch, op.cols_p, op.ld_out) &&
            !std::getenv("SGC_SPMM_DIRECT")) {
          // the unrolled direct form where it fits: fastest of all shapes on the R-MAT 20 spider
          // at 8 colorings (p = 3: 7.5 vs 8.1 ms; p = 2: 2.6 vs 3.4 ms) and at 4 (p = 2)
          op.spmm_buckets = false;
          op.spmm_variant = 11;
        }
        if (batch == 1 && spmm_grouped_fits(batch, op.ld_out, elem, smem_cap_of(g)) && !std::getenv("SGC_SPMM_DIRECT")) {
          // one coloring per pass: the grouped form, measured fastest or within 2% of the fastest on
          // every SpMM of the 12-, 13- and 15-vertex trees on R-MAT 21 (narrow rows 1.4-3x faster)
          op.spmm_buckets = false;
          op.spmm_variant = op.cols_p <= 256 ? 13 : 15;
          if (spmm_staged_fits(batch, op.cols_p, op.ld_out, elem, smem_cap_of(g), 16))
            // rows wider than 128 columns in FP32: the staged form, with 3 chunks per warp in flight
            // (R-MAT 21, the 15-vertex tree's p = 5 SpMM: 31.8 ms against 37.6 in registers)
            op.spmm_variant = 16;
        }
        const int shape = shapes && idx < (int)shapes->size() ? (*shapes)[idx] : 0;
        if (shape == kShapeSpmmBuckets && spmm_bucket_bytes(batch, k, op.cols_p, elem) <= kSpmmBucketTuneMaxBytes) {
          op.spmm_buckets = true;
          op.spmm_variant = 0;
        } else if (shape == kShapeSpmmBucketsB &&
                   spmm_bucket_bytes(batch, k, op.cols_p, elem) <= kSpmmBucketTuneMaxBytes) {
          op.spmm_buckets = true;
          op.spmm_variant = 7;
        } else if (shape == kShapeSpmmDirect) {  // the chunked loop with a runtime batch
          op.spmm_buckets = false;
          op.spmm_variant = 0;
        } else if (shape == kShapeSpmmPrefetch && spmm_cols_per_lane(batch, op.cols_p) <= 12) {
          op.spmm_buckets = false;
          op.spmm_variant = 1;
        } else if (shape == kShapeSpmmRegBuckets && reg_buckets_fit(batch, k, op.cols_p, elem, g)) {
          op.spmm_buckets = true;
          op.spmm_variant = 2;
        } else if (shape == kShapeSpmmDirectB) {
          op.spmm_buckets = false;
          op.spmm_variant = 5;
        } else if (shape == kShapeSpmmDirectBLane && op.ld_out < 65535) {
          op.spmm_buckets = false;
          op.spmm_variant = 6;
        } else if (shape == kShapeSpmmWide && op.ld_out < 65535) {
          op.spmm_buckets = false;
          op.spmm_variant = 12;
        } else if ((shape == kShapeSpmmGrouped || shape == kShapeSpmmGrouped8) &&
                   spmm_grouped_fits(batch, op.ld_out, elem, smem_cap_of(g))) {
          op.spmm_buckets = false;
          op.spmm_variant = shape == kShapeSpmmGrouped ? 13 : 15;
        } else if ((shape == kShapeSpmmStaged || shape == kShapeSpmmStaged8) &&
                   spmm_staged_fits(batch, op.cols_p, op.ld_out, elem, smem_cap_of(g),
                                    shape == kShapeSpmmStaged ? 16 : 17)) {
          op.spmm_buckets = false;
          op.spmm_variant = shape == kShapeSpmmStaged ? 16 : 17;
        } else if (shape == kShapeSpmmUnrolled && spmm_unrolled_fits(batch, op.cols_p, op.ld_out)) {
          op.spmm_buckets = false;
          op.spmm_variant = 11;
        } else if (shape == kShapeSpmmDirectBPriv && op.ld_out * 32 * elem <= kSpmmPrivMaxBytes) {
          op.spmm_buckets = false;
          op.spmm_variant = 10;
        } else if (shape == kShapeSpmmDirectB8 || shape == kShapeSpmmDirectB12) {
          op.spmm_buckets = false;
          op.spmm_variant = shape == kShapeSpmmDirectB8 ? 8 : 9;
        } else if ((shape == kShapeSpmmRing2 || shape == kShapeSpmmRing4) && batch >= 4) {
          op.spmm_buckets = false;
          op.spmm_variant = shape == kShapeSpmmRing2 ? 3 : 4;
        } else if (shape == kShapeSpmmPacked && spmm_packed_bytes(k, op.cols_p, op.ld_out) > 0) {
          op.spmm_buckets = false;
          op.spmm_variant = 0;
          op.spmm_pos_bytes = op.ld_out < 255 ? 1 : 2;
        }
        if (unpruned == 2) {  // the pruned sums one passive column at a time
          op.spmm_buckets = false;
          op.spmm_variant = 14;
          op.spmm_pos_bytes = 0;
        }
        op.shape = op.spmm_variant == 14   ? 0
                   : op.spmm_variant == 17 ? kShapeSpmmStaged8
                   : op.spmm_variant == 16 ? kShapeSpmmStaged
                   : op.spmm_variant == 15 ? kShapeSpmmGrouped8
                   : op.spmm_variant == 13 ? kShapeSpmmGrouped
                   : op.spmm_variant == 12 ? kShapeSpmmWide
                   : op.spmm_variant == 11 ? kShapeSpmmUnrolled
                   : op.spmm_variant == 10 ? kShapeSpmmDirectBPriv
                   : op.spmm_variant == 9  ? kShapeSpmmDirectB12
                   : op.spmm_variant == 8  ? kShapeSpmmDirectB8
                   : op.spmm_variant == 7  ? kShapeSpmmBucketsB
                   : op.spmm_variant == 6  ? kShapeSpmmDirectBLane
                   : op.spmm_variant == 5  ? kShapeSpmmDirectB
                   : op.spmm_variant == 3  ? kShapeSpmmRing2
                   : op.spmm_variant == 4  ? kShapeSpmmRing4
                   : op.spmm_variant == 2  ? kShapeSpmmRegBuckets
                   : op.spmm_buckets     ? kShapeSpmmBuckets
                   : op.spmm_pos_bytes   ? kShapeSpmmPacked
                   : op.spmm_variant     ? kShapeSpmmPrefetch
                                         : kShapeSpmmDirect;
        op.tab_off = !build_tabs             ? 0
                     : op.spmm_variant == 6  ? build_table(cr, k, (OpKind)(OP_SPMM + 400), Pc.size, 32 / batch,
                                                           &P->tabs, &tcache)
                     : op.spmm_variant == 11 ? build_table(cr, k, (OpKind)(OP_SPMM + 600), Pc.size, batch,
                                                           &P->tabs, &tcache)
                     : op.spmm_variant == 12 ? build_table(cr, k, (OpKind)(OP_SPMM + 700), Pc.size, batch,
                                                           &P->tabs, &tcache)
                     : op.spmm_variant == 13 || op.spmm_variant == 15
                                             ? build_table(cr, k, (OpKind)(OP_SPMM + 800), Pc.size, 0, &P->tabs,
                                                           &tcache)
                     : op.spmm_variant == 16 || op.spmm_variant == 17
                                             ? build_table(cr, k, (OpKind)(OP_SPMM + 900), Pc.size, 0, &P->tabs,
                                                           &tcache)
                     : op.spmm_variant == 14 ? build_table(cr, k, (OpKind)(OP_SPMM + 500), Pc.size, 0,
                                                           &P->tabs, &tcache)
                     : op.spmm_buckets       ? build_table(cr, k, (OpKind)(OP_SPMM + 100), Pc.size, 0, &P->tabs,
                                                           &tcache)
                     : op.spmm_pos_bytes   ? build_table(cr, k, (OpKind)(OP_SPMM + 300), Pc.size, op.spmm_pos_bytes,
                                                         &P->tabs, &tcache)
                                           : build_table(cr, k, OP_SPMM, Pc.size, 0, &P->tabs, &tcache);
        max_spmm_width = std::max<int64_t>(max_spmm_width, op.ld_out * batch);
        op.alg_bytes = 4 * (nv + 1 + nnz) + nv * batch + (double)elem * nv * batch * (double)(op.cols_p + op.cols_out);
        op.gather_bytes = nnz * (double)batch * (double)op.cols_p * elem;
        double by = nnz * 4 + (double)elem * nv * (double)(op.cols_p + op.cols_out);
        P->est_bytes += by;
        P->est_spmm_bytes += by;
        P->est_cost += (by + gather_factor * nnz * (double)op.cols_p * elem) / bw;
        P->n_spmm++;
      }
      use_buf(P, op.in_p, idx);
      P->ops.push_back(op);
    }
    // ---- the combine step
    const bool final = C.size == tk && tk == k;  // the single full color set
    if (A.a < 0 && !final) {
      // single-vertex active child: M_s(v, S + c(v)) = P(v, S), the same numbers
      table_buf[c] = pbuf[C.p];
      table_state[c] = p_state[C.p];
      table_w[c] = w_p(Pc.size);
      table_ld[c] = pad_ld(table_w[c], elem);
      continue;
    }
    PlanOp op{};
    op.t = C.size;
    op.a = A.size;
    op.p = Pc.size;
    op.in_p = pbuf[C.p];
    op.state_p = p_state[C.p];
    op.cols_p = w_p(Pc.size);
    op.ld_p = pad_ld(op.cols_p, elem);
    op.nsplit = (int64_t)cr.binom[C.size - 1][Pc.size];
    const int idx = (int)P->ops.size();
    if (A.a >= 0) {
      op.in_a = table_buf[C.a];
      op.state_a = table_state[C.a];
      op.cols_a = table_w[C.a];
      op.ld_a = table_ld[C.a];
    }
    if (final) {
      op.kind = A.a < 0 ? OP_FINAL_LEAF : OP_FINAL;
      op.final_reg = A.a >= 0 && final_reg_compiled(K, Pc.size) && final_reg_enabled();
      op.tab_off = (build_tabs && A.a >= 0) ? build_table(cr, k, OP_FINAL, k, A.size, &P->tabs, &tcache) : 0;
      op.out = P->buf_partials;
      if (A.a < 0) {
        op.alg_bytes = (double)elem * nv * batch;
        op.alg_flops = nv * batch;
      } else {
        op.alg_bytes = (double)elem * nv * batch * (double)(op.cols_a + op.cols_p);
        op.alg_flops = 2.0 * nv * batch * (double)op.cols_p;
      }
      double by = nv * ((A.a < 0 ? 0.0 : (double)op.cols_a) + (double)op.cols_p) * elem;
      P->est_bytes += by;
      P->est_fma += A.a < 0 ? 0.0 : nv * (double)op.cols_p;
      P->est_cost += by / bw;
    } else {
      op.kind = OP_EMA;
      op.cols_out = w_table(C.size);
      op.ld_out = pad_ld(op.cols_out, elem);
      const int smem_cap = g->smem_optin > 0 ? g->smem_optin : 227 * 1024;
      ema_shape(op.cols_a, op.cols_p, elem, smem_cap, &op.ema_rows, &op.ema_rpl);
      const int shape = shapes && idx < (int)shapes->size() ? (*shapes)[idx] : 0;
      const bool sym = A.size - 1 == Pc.size && table_buf[C.a] == pbuf[C.p];
      // default: vertex tiles when they fit (measured faster on R-MAT 20), else rows
      op.ema_vrpl = ema_vertex_fits(batch, 1, op.ld_a, op.ld_p, sym, elem, smem_cap) ? 1 : 0;
      if ((shape == 64 || shape == 32 || shape == 16 || shape == 8 || shape == 4 || shape == 2 || shape == 1) &&
          (op.cols_a + op.cols_p) * elem * (shape + 1) <= smem_cap) {
        op.ema_rows = shape;
        op.ema_rpl = shape == 64 ? 2 : 1;
        op.ema_vrpl = 0;
      } else if ((shape == kShapeEmaVertex1 || shape == kShapeEmaVertex2) &&
                 ema_vertex_fits(batch, shape - 100, op.ld_a, op.ld_p, sym, elem, smem_cap)) {
        op.ema_vrpl = shape - 100;
      }
      op.ema_sym = op.in_a == op.in_p && A.size - 1 == Pc.size;
      // the register form (FP32, compiled-in shapes): forced, or the default where it exists at 8 or
      // more colorings per pass (a thread holds one (vertex, coloring) row: its loads coalesce only
      // across interleaved colorings)
      if (elem == 4 && ema_reg_compiled(K, A.size - 1, Pc.size, op.ema_sym) &&
          ((shape == 0 && batch >= 8) || shape == kShapeEmaReg)) {
        op.ema_reg_k = K;
        op.ema_vrpl = 0;
      }
      // the scheduled form (one coloring per pass) when forced or tuned, and by default for rows of
      // 256 words or more (measured faster than every other form on every such combine of the 13-
      // and 15-vertex trees on R-MAT 21; slower on rows of about a hundred words)
      const bool sched_default = shape == 0 && op.ld_a + (op.ema_sym ? 0 : op.ld_p) >= 256;
      // two blocks per SM by default where each gets at least the rows one block would
      int upg0 = 1;
      const bool sched2 = shape == kShapeEmaSched2 ||
                          (sched_default && ema_sched_rows(op.cols_out, op.ld_a, op.ld_p, op.ema_sym, elem, smem_cap,
                                                           &upg0, 2) >=
                                                ema_sched_rows(op.cols_out, op.ld_a, op.ld_p, op.ema_sym, elem,
                                                               smem_cap, &upg0, 1));
      if (!op.ema_reg_k && batch == 1 && (shape == kShapeEmaSched || sched2 || sched_default)) {
        int upg = 1;
        const int r = ema_sched_rows(op.cols_out, op.ld_a, op.ld_p, op.ema_sym, elem, smem_cap, &upg, sched2 ? 2 : 1);
        if (r > 0) {
          op.ema_sched = r;
          op.ema_upg = upg;
          op.ema_vrpl = 0;
        }
      }
      op.shape = op.ema_reg_k    ? kShapeEmaReg
                 : op.ema_sched  ? (sched2 ? kShapeEmaSched2 : kShapeEmaSched)
                 : op.ema_vrpl   ? 100 + op.ema_vrpl
                                 : op.ema_rows;
      if (op.ema_sym) op.nsplit /= 2;  // C(2p, p) is even
      // the vertex-tile kernel takes the raw split indices (rows 0, no column offset)
      op.tab_off = !build_tabs ? 0
                   : op.ema_sched ? build_table(cr, k, op.ema_sym ? (OpKind)(OP_EMA + 400) : (OpKind)(OP_EMA + 300),
                                                C.size, A.size, &P->tabs, &tcache, op.ema_sym ? 0 : (int)op.ld_a, 0)
                   : build_tabs ? build_table(cr, k, op.ema_sym ? (OpKind)(OP_EMA + 200) : OP_EMA, C.size, A.size,
                                            &P->tabs, &tcache, op.ema_vrpl ? 0 : op.ema_rows,
                                            (op.ema_vrpl || op.ema_rows == 0) ? 0 : op.cols_a)
                              : 0;
      op.state_out = table_state[c] = n_states++;
      op.out = table_buf[c] = add_buf(P, "T" + std::to_string(c), rows * op.ld_out * elem, idx);
      table_w[c] = op.cols_out;
      table_ld[c] = op.ld_out;
      P->n_tables++;
      op.alg_bytes = (double)elem * nv * batch * (double)(op.cols_a + op.cols_p + op.cols_out);
      op.alg_flops = 2.0 * nv * batch * (double)op.cols_out * (double)op.nsplit;
      double by = (double)elem * nv * (double)(op.cols_a + op.cols_p + op.cols_out);
      double fm = nv * (double)op.cols_out * (double)op.nsplit;
      P->est_bytes += by;
      P->est_fma += fm;
      P->est_cost += std::max(by / bw, fm / fma_rate);
    }
    P->n_ema++;
    use_buf(P, op.in_a, idx);
    use_buf(P, op.in_p, idx);
    P->ops.push_back(op);
  }
  if (tk < k) {
    // more colors than template vertices: sum the root table over all its color sets
    int rc = -1;
    for (size_t c = 0; c < B.cls.size(); ++c)
      if (B.cls[c].size == tk) rc = (int)c;
    PlanOp op{};
    op.kind = OP_FINAL_SUM;
    op.t = tk;
    op.in_p = table_buf[rc];
    op.state_p = table_state[rc];
    op.cols_p = table_w[rc];
    op.ld_p = table_ld[rc];
    op.out = P->buf_partials;
    op.alg_bytes = (double)elem * nv * batch * (double)op.cols_p;
    op.alg_flops = nv * batch * (double)op.cols_p;
    P->est_bytes += nv * (double)op.cols_p * elem;
    P->est_cost += nv * (double)op.cols_p * elem / bw;
    use_buf(P, op.in_p, (int)P->ops.size());
    P->ops.push_back(op);
  }
  // A symmetric register-form eMA whose table only feeds the last step, which
  // multiplies it with the same passive table: one kernel does both per row
  // (the eMA's table never goes to HBM).  SGC_NO_FUSE=1 keeps them apart.
  const size_t nops = P->ops.size();
  if (nops >= 2 && !(std::getenv("SGC_NO_FUSE") && std::atoi(std::getenv("SGC_NO_FUSE")) == 1)) {
    PlanOp& e = P->ops[nops - 2];
    PlanOp& f = P->ops[nops - 1];
    if (e.kind == OP_EMA && e.ema_reg_k > 0 && e.ema_sym && f.kind == OP_FINAL && f.in_a == e.out &&
        f.in_p == e.in_p && f.p == e.p && ema_final_compiled(e.ema_reg_k, e.p)) {
      e.ema_final = true;
      f.final_fused = true;
      // the eMA's table is never stored: it takes no workspace, and the pair reads the passive
      // table once (the final op only sums the block partials)
      const double table_bytes = (double)elem * nv * (double)e.cols_out;
      P->est_bytes -= table_bytes + (double)elem * nv * (double)(f.cols_a + f.cols_p);
      P->bufs[e.out].bytes = 16;
      e.alg_bytes = (double)elem * nv * batch * (double)e.cols_p;
      f.alg_bytes = 8.0 * batch * (double)P->final_blocks;
    }
  }
  P->n_states = n_states;
  P->buf_states = add_buf(P, "states", 8LL * std::max(1, n_states), 0);
  bool grouped = false;
  for (const PlanOp& op : P->ops) grouped |= op.kind == OP_SPMM && spmm_variant_grouped(op.spmm_variant);
  if (grouped) {
    const int64_t nitems = (int64_t)g->n_seg + (g->n_act - g->n_heavy);
    P->buf_gids = add_buf(P, "group_ids", 4LL * batch * g->nnz, 0);
    P->buf_gcols = add_buf(P, "group_colors", (int64_t)batch * g->nnz, 0);
    P->buf_gkept = add_buf(P, "group_kept", 4LL * batch * nitems, 0);
  }
  P->scratch_width = max_spmm_width;
  P->buf_scratch = add_buf(P, "spmm_scratch", (int64_t)g->n_seg * max_spmm_width * elem, 0);
  P->buf_hist_heavy = add_buf(P, "hist_heavy", 4LL * g->n_heavy * batch * k, 0);
  const int last = (int)P->ops.size() - 1;
  for (int b : {P->buf_seeds, P->buf_colors, P->buf_out, P->buf_partials, P->buf_states, P->buf_scratch,
                P->buf_hist_heavy, P->buf_gids, P->buf_gcols, P->buf_gkept}) {
    if (b < 0) continue;
    P->bufs[b].first = 0;
    P->bufs[b].last = last;
  }
  place_buffers(P);
}

// Every index a table holds must stay inside the buffer the kernels use it on.
static bool tables_in_range(const Plan& P, int k) {
  for (const PlanOp& op : P.ops) {
    if (op.tab_off < 0 || P.tabs.empty()) continue;
    const uint32_t* t = P.tabs.data() + op.tab_off;
    const int64_t left = (int64_t)P.tabs.size() - op.tab_off;
    if (op.kind == OP_SPMM && op.spmm_variant == 6) {
      const int L = 32 / P.batch;
      const int64_t n = (int64_t)k * k * L * spmm_lane_nsp(op.cols_p, L);
      if ((n + 1) / 2 > left) return false;
      const uint16_t* h = reinterpret_cast<const uint16_t*>(t);
      for (int64_t i = 0; i < n; ++i)
        if (h[i] != 0xFFFFu && h[i] >= (uint32_t)op.cols_out) return false;
    } else if (op.kind == OP_SPMM && op.spmm_variant == 14) {
      const int64_t n = (int64_t)k * op.cols_out * k;
      if (n > left) return false;
      for (int64_t i = 0; i < n; ++i)
        if (t[i] != 0xFFFFFFFFu && t[i] >= (uint32_t)op.cols_p) return false;
    } else if (op.kind == OP_SPMM && (op.spmm_variant == 13 || op.spmm_variant == 15)) {
      const int64_t n = (int64_t)k * k * op.cols_p;
      if ((n + 1) / 2 > left) return false;
      const uint16_t* h = reinterpret_cast<const uint16_t*>(t);
      for (int64_t i = 0; i < n; ++i)
        if (h[i] != 0xFFFFu && h[i] >= (uint32_t)op.cols_out) return false;
    } else if (op.kind == OP_SPMM && (op.spmm_variant == 16 || op.spmm_variant == 17)) {
      // rows of whole 16-byte pieces, copied as such: the table must start on a 16-byte boundary
      const int64_t n = (int64_t)k * k * spmm_staged_pitch(op.cols_p);
      if (n / 2 > left || op.tab_off % 4 != 0) return false;
      const uint16_t* h = reinterpret_cast<const uint16_t*>(t);
      for (int64_t i = 0; i < n; ++i)
        if (h[i] != 0xFFFFu && h[i] >= (uint32_t)op.cols_out) return false;
    } else if (op.kind == OP_SPMM && op.spmm_variant == 12) {
      const int64_t n = (int64_t)k * k * (32 / P.batch) * spmm_wide_nch(P.batch, op.cols_p) * 4;
      if (n > left || op.tab_off % 4 != 0) return false;
      for (int64_t i = 0; i < n; ++i)
        for (int x = 0; x < 2; ++x) {
          const uint32_t v = t[i] >> (16 * x) & 0xffffu;
          if (v != 0xFFFFu && v >= (uint32_t)op.cols_out) return false;
        }
    } else if (op.kind == OP_SPMM && op.spmm_variant == 11) {
      const int64_t n = (int64_t)k * k * (32 / P.batch) * 4;
      if (n > left || op.tab_off % 4 != 0) return false;
      for (int64_t i = 0; i < n; ++i)
        for (int x = 0; x < 4; ++x) {
          const uint32_t v = t[i] >> (8 * x) & 0xffu;
          if (v != 0xFFu && v >= (uint32_t)op.cols_out) return false;
        }
    } else if (op.kind == OP_SPMM && op.spmm_pos_bytes > 0) {
      const int eb = op.spmm_pos_bytes;
      const int64_t ld = spmm_packed_ld(op.cols_p, eb);
      const int64_t nbytes = (int64_t)k * k * ld * eb;
      if ((nbytes + 3) / 4 > left) return false;
      const uint8_t* b = reinterpret_cast<const uint8_t*>(t);
      const uint32_t none = eb == 1 ? 0xFFu : 0xFFFFu;
      for (int64_t i = 0; i < nbytes; i += eb) {
        const uint32_t v = eb == 1 ? b[i] : (uint32_t)b[i] | (uint32_t)b[i + 1] << 8;
        if (v != none && v >= (uint32_t)op.cols_out) return false;
      }
    } else if (op.kind == OP_SPMM && !op.spmm_buckets) {
      const int64_t n = (int64_t)k * k * op.cols_p;
      if (n > left) return false;
      for (int64_t i = 0; i < n; ++i)
        if (t[i] != 0xFFFFFFFFu && t[i] >= (uint32_t)op.cols_out) return false;
    } else if (op.kind == OP_SPMM) {
      const int64_t n = (int64_t)k * op.cols_out * op.p;
      if (n > left) return false;
      for (int64_t i = 0; i < n; ++i)
        if ((int)(t[i] & 0xffu) >= k || (int64_t)(t[i] >> 8) >= op.cols_p) return false;
    } else if (op.kind == OP_UNPRUNED) {
      const int64_t n = 2 * op.cols_out * op.nsplit;
      if (n > left) return false;
      for (int64_t i = 0; i < n; i += 2)
        if (t[i] >= (uint32_t)op.cols_a || t[i + 1] >= (uint32_t)op.cols_p) return false;
      const int64_t n2 = (int64_t)k * op.cols_p * k;
      if (op.tab2_off < 0 || n2 > (int64_t)P.tabs.size() - op.tab2_off) return false;
      const uint32_t* t2 = P.tabs.data() + op.tab2_off;
      const int64_t wpt = op.in_p < 0 ? 1 : op.ld_p;  // entries of a passive row
      for (int64_t i = 0; i < n2; ++i)
        if (t2[i] != 0xFFFFFFFFu && (int64_t)t2[i] >= wpt) return false;
    } else if (op.kind == OP_EMA && op.ema_sched > 0) {
      const int64_t G = (op.cols_out + 31) / 32;
      if (2 * G > left) return false;
      const uint32_t lim_p = (uint32_t)(op.ema_sym ? op.cols_a : op.cols_p);
      int64_t terms = 0;
      for (int64_t gi = 0; gi < G; ++gi) {
        const int64_t first = t[2 * gi], n = t[2 * gi + 1];
        if ((first + n) * 32 > left) return false;
        for (int64_t i = first * 32; i < (first + n) * 32; ++i) {
          if (t[i] == 0xFFFFFFFFu) continue;
          if ((t[i] & 0xFFFFu) >= (uint32_t)op.cols_a || (t[i] >> 16) >= lim_p) return false;
          ++terms;
        }
      }
      if (terms != op.cols_out * op.nsplit) return false;  // every split term scheduled exactly once
    } else if (op.kind == OP_EMA && op.ema_reg_k == 0 && (op.ema_vrpl > 0 || op.ema_rows == 0)) {
      const int64_t n = 2 * op.cols_out * op.nsplit;
      if (n > left) return false;
      for (int64_t i = 0; i < n; i += 2)
        if (t[i] >= (uint32_t)op.cols_a || t[i + 1] >= (uint32_t)op.cols_p) return false;
    } else if (op.kind == OP_EMA) {
      const int64_t n = 2 * op.cols_out * op.nsplit;
      const uint32_t lim = (uint32_t)((op.cols_a + op.cols_p) * (op.ema_rows + 1));
      if (n > left) return false;
      for (int64_t i = 0; i < n; ++i)
        if (t[i] >= lim) return false;
    } else if (op.kind == OP_FINAL) {
      if (op.cols_p > left) return false;
      for (int64_t i = 0; i < op.cols_p; ++i)
        if (t[i] >= (uint32_t)op.cols_a) return false;
    }
  }
  return true;
}

std::vector<int> op_shape_candidates(const sgc_graph* g, const Plan& P, int i) {
  std::vector<int> c;
  const PlanOp& op = P.ops[i];
  const int smem_cap = g->smem_optin > 0 ? g->smem_optin : 227 * 1024;
  if (op.kind == OP_SPMM) {
    if (spmm_grouped_fits(P.batch, op.ld_out, P.elem, smem_cap)) {
      c.push_back(kShapeSpmmGrouped);
      if (op.cols_p > 256) c.push_back(kShapeSpmmGrouped8);  // chunks of 256 columns
    }
    if (spmm_staged_fits(P.batch, op.cols_p, op.ld_out, P.elem, smem_cap, 16)) c.push_back(kShapeSpmmStaged);
    if (spmm_staged_fits(P.batch, op.cols_p, op.ld_out, P.elem, smem_cap, 17)) c.push_back(kShapeSpmmStaged8);
    c.push_back(kShapeSpmmDirect);
    c.push_back(kShapeSpmmDirectB);
    if (op.ld_out < 65535) c.push_back(kShapeSpmmDirectBLane);
    if (spmm_unrolled_fits(P.batch, op.cols_p, op.ld_out)) c.push_back(kShapeSpmmUnrolled);
    else if (op.ld_out < 65535) c.push_back(kShapeSpmmWide);
    if (spmm_cols_per_lane(P.batch, op.cols_p) > 4) c.push_back(kShapeSpmmDirectB8);
    if (spmm_cols_per_lane(P.batch, op.cols_p) > 8) c.push_back(kShapeSpmmDirectB12);
    if (op.ld_out * 32 * P.elem <= kSpmmPrivMaxBytes) c.push_back(kShapeSpmmDirectBPriv);
    if (spmm_cols_per_lane(P.batch, op.cols_p) <= 12) c.push_back(kShapeSpmmPrefetch);
    if (spmm_bucket_bytes(P.batch, P.k, op.cols_p, P.elem) <= kSpmmBucketTuneMaxBytes) {
      c.push_back(kShapeSpmmBuckets);
      c.push_back(kShapeSpmmBucketsB);
    }
    if (reg_buckets_fit(P.batch, P.k, op.cols_p, P.elem, g)) c.push_back(kShapeSpmmRegBuckets);
    if (spmm_packed_bytes(P.k, op.cols_p, op.ld_out) > 0) c.push_back(kShapeSpmmPacked);
    if (P.batch >= 4 && op.cols_p <= 64) {  // the copy rings measured 3-5x slower on wide rows
      c.push_back(kShapeSpmmRing2);
      c.push_back(kShapeSpmmRing4);
    }
  } else if (op.kind == OP_EMA) {
    for (int r : {64, 32, 16, 8, 4, 2, 1})
      if ((op.cols_a + op.cols_p) * P.elem * (r + 1) <= smem_cap && c.size() < 5) c.push_back(r);
    for (int v : {1, 2})
      if (ema_vertex_fits(P.batch, v, op.ld_a, op.ld_p, op.ema_sym, P.elem, smem_cap)) c.push_back(100 + v);
    if (P.elem == 4 && ema_reg_compiled(P.k - 1, op.a - 1, op.p, op.ema_sym)) c.push_back(kShapeEmaReg);
    int upg = 1;
    if (P.batch == 1 && ema_sched_rows(op.cols_out, op.ld_a, op.ld_p, op.ema_sym, P.elem, smem_cap, &upg) > 0) {
      c.insert(c.begin(), kShapeEmaSched);
      const int r1 = ema_sched_rows(op.cols_out, op.ld_a, op.ld_p, op.ema_sym, P.elem, smem_cap, &upg);
      const int r2 = ema_sched_rows(op.cols_out, op.ld_a, op.ld_p, op.ema_sym, P.elem, smem_cap, &upg, 2);
      if (r2 > 0 && r2 != r1) c.insert(c.begin() + 1, kShapeEmaSched2);  // a different row count
    }
  }
  if (c.size() < 2) c.clear();
  return c;
}

sgc_status make_plan(const sgc_graph* g, const sgc_template* t, int precision, int root, int policy, int batch,
                     bool build_tabs, Plan* out, const std::vector<int>* shapes, int colors, int unpruned) {
  if (colors != 0 && (colors < t->k || colors > SGC_MAX_K))
    return fail(SGC_ERR_INVALID, "options.colors must be 0 or in [|T|, " + std::to_string(SGC_MAX_K) + "]");
  if (root >= t->k) return fail(SGC_ERR_INVALID, "options.root is not a template vertex");
  int best_root = -1, best_policy = 0;
  double best_cost = 0;
  int64_t best_ws = 0;
  for (int r = 0; r < t->k; ++r) {
    if (root >= 0 && r != root) continue;
    for (int pol = 0; pol < 2; ++pol) {
      if (policy >= 0 && pol != policy) continue;
      Plan P;
      plan_for(g, t, precision, r, pol, 1, false, &P, nullptr, colors, unpruned);
      if (best_root < 0 || P.est_cost < best_cost * 0.999 ||
          (P.est_cost <= best_cost * 1.001 && P.ws_bytes < best_ws)) {
        best_root = r;
        best_policy = pol;
        best_cost = P.est_cost;
        best_ws = P.ws_bytes;
      }
    }
  }
  plan_for(g, t, precision, best_root, best_policy, batch, build_tabs, out, shapes, colors, unpruned);
  if (build_tabs && !tables_in_range(*out, out->k)) return fail(SGC_ERR_INTERNAL, "index table out of range");
  return SGC_OK;
}

}  // namespace sgc
