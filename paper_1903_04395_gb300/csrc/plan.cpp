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

struct TabKey {
  int kind, t, a;
  bool operator<(const TabKey& o) const {
    return kind != o.kind ? kind < o.kind : (t != o.t ? t < o.t : a < o.a);
  }
};

}  // namespace

static int64_t build_table(const ColorIndex& ci, OpKind kind, int t, int a, std::vector<uint32_t>* tabs,
                           std::map<TabKey, int64_t>* cache) {
  TabKey key{(int)kind, t, a};
  auto it = cache->find(key);
  if (it != cache->end()) return it->second;
  const int k = ci.k;
  // align each table to 4 words
  while (tabs->size() % 4) tabs->push_back(0);
  int64_t off = (int64_t)tabs->size();
  if (kind == OP_GATHER) {
    // [c][S]: rank of S \ {c} among (t-1)-subsets, or ~0 if c is not in S
    const uint64_t ct = ci.nsets(t);
    for (int c = 0; c < k; ++c)
      for (uint64_t s = 0; s < ct; ++s) {
        uint32_t m = ci.unrank_mask(s, t);
        tabs->push_back((m >> c & 1u) ? ci.rank_mask(m & ~(1u << c)) : 0xFFFFFFFFu);
      }
  } else if (kind == OP_EMA) {
    // [j][S]: the j-th split (C_a, C_p) of color set S, packed I(C_a) | I(C_p) << 16
    const uint64_t ct = ci.nsets(t);
    const int p = t - a;
    const uint64_t ns = ci.binom[t][p];
    std::vector<uint32_t> tab(ns * ct);
    for (uint64_t s = 0; s < ct; ++s) {
      uint32_t m = ci.unrank_mask(s, t);
      uint64_t j = 0;
      // submasks of m with popcount a, in decreasing numeric order
      for (uint32_t sub = m;; sub = (sub - 1) & m) {
        if (__builtin_popcount(sub) == a) {
          tab[j * ct + s] = ci.rank_mask(sub) | (ci.rank_mask(m & ~sub) << 16);
          ++j;
        }
        if (sub == 0) break;
      }
    }
    tabs->insert(tabs->end(), tab.begin(), tab.end());
  } else if (kind == OP_FINAL) {
    // [I_p]: rank of the complement of C_p (an a-subset), t = k
    const int p = k - a;
    const uint32_t full = (k == 32) ? 0xFFFFFFFFu : ((1u << k) - 1);
    for (uint64_t s = 0; s < ci.nsets(p); ++s) tabs->push_back(ci.rank_mask(full & ~ci.unrank_mask(s, p)));
  } else if (kind == OP_FINAL_LEAF) {
    // [c]: rank of all colors but c among (k-1)-subsets
    const uint32_t full = (1u << k) - 1;
    for (int c = 0; c < k; ++c) tabs->push_back(ci.rank_mask(full & ~(1u << c)));
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

static void plan_for(const sgc_graph* g, const sgc_template* t, int precision, int root, int policy,
                     int batch, bool build_tabs, Plan* P) {
  Rooted R;
  root_tree(t, root, &R);
  Builder B(R, policy);
  const int top = B.build(root, 0);
  const int k = t->k;
  ColorIndex ci(k);

  P->k = k;
  P->root = root;
  P->policy = policy;
  P->batch = batch;
  P->precision = precision;
  P->elem = precision == SGC_FP64 ? 8 : 4;
  P->rows = (int64_t)g->n_act * batch;
  P->bufs.clear();
  P->ops.clear();
  P->tabs.clear();
  const int64_t rows = P->rows;
  const int elem = P->elem;
  const double nv = (double)g->n_act, nnz = (double)g->nnz;

  // fixed buffers; lifetimes are stretched to the whole pass below
  P->buf_seeds = add_buf(P, "seeds", 8LL * batch, 0);
  P->buf_colors = add_buf(P, "colors", rows, 0);
  P->buf_out = add_buf(P, "out", 8LL * batch, 0);
  P->final_blocks = (4 * std::max(1, g->num_sms) + 31) / 32 * 32;  // multiple of 32: see k_final
  P->buf_partials = add_buf(P, "partials", 8LL * batch * P->final_blocks, 0);

  std::vector<int> table_buf(B.cls.size(), -1), pbuf(B.cls.size(), -1);
  std::vector<int> table_state(B.cls.size(), -1), p_state(B.cls.size(), -1);
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
      op.cols_out = (int64_t)ci.nsets(Pc.size);
      op.ld_out = pad_ld(op.cols_out, elem);
      op.state_out = p_state[C.p] = n_states++;
      const int idx = (int)P->ops.size();
      op.out = pbuf[C.p] = add_buf(P, "P" + std::to_string(c), rows * op.ld_out * elem, idx);
      if (Pc.a < 0) {
        op.kind = OP_HIST;
        op.in_p = P->buf_colors;
        op.alg_bytes = 4 * (nv + 1) + 4 * nnz + nv * batch + (double)elem * nv * batch * (double)op.cols_out;
        double by = nnz * 4 + nnz * 1 + nv * (double)op.cols_out * elem;
        P->est_bytes += by;
        P->est_spmm_bytes += by;
        P->est_cost += by / bw;
      } else {
        op.kind = OP_SPMM;
        op.in_p = table_buf[C.p];
        op.cols_p = op.cols_out;
        op.ld_p = op.ld_out;
        op.state_p = table_state[C.p];
        max_spmm_width = std::max<int64_t>(max_spmm_width, op.ld_out * batch);
        const SpmmShape sh = spmm_shape(op.ld_out * batch, elem);
        op.alg_bytes = 4 * (nv + 1 + nnz) * (double)sh.tiles + 2.0 * elem * nv * batch * (double)op.cols_out;
        double by = nnz * 4 + 2.0 * nv * (double)op.cols_out * elem;
        P->est_bytes += by;
        P->est_spmm_bytes += by;
        P->est_cost += (by + gather_factor * nnz * (double)op.cols_out * elem) / bw;
        P->n_spmm++;
      }
      use_buf(P, op.in_p, idx);
      P->ops.push_back(op);
    }
    // ---- the combine step
    PlanOp op{};
    op.t = C.size;
    op.a = A.size;
    op.p = Pc.size;
    op.in_p = pbuf[C.p];
    op.state_p = p_state[C.p];
    op.cols_p = (int64_t)ci.nsets(Pc.size);
    op.ld_p = pad_ld(op.cols_p, elem);
    op.nsplit = (int64_t)ci.binom[C.size][Pc.size];
    const int idx = (int)P->ops.size();
    if (A.a >= 0) {
      op.in_a = table_buf[C.a];
      op.state_a = table_state[C.a];
      op.cols_a = (int64_t)ci.nsets(A.size);
      op.ld_a = pad_ld(op.cols_a, elem);
    } else {
      op.in_a = P->buf_colors;
    }
    const bool final = C.size == k;
    if (final) {
      op.kind = A.a < 0 ? OP_FINAL_LEAF : OP_FINAL;
      op.tab_off = build_tabs ? build_table(ci, op.kind, k, A.size, &P->tabs, &tcache) : 0;
      op.out = P->buf_partials;
      if (A.a < 0) {
        op.alg_bytes = nv * batch + (double)elem * nv * batch;
        op.alg_flops = nv * batch;
      } else {
        op.alg_bytes = (double)elem * nv * batch * (double)(op.cols_a + op.cols_p);
        op.alg_flops = 2.0 * nv * batch * (double)op.cols_p;
      }
      double by = nv * ((A.a < 0 ? 1.0 : (double)op.cols_a) + (A.a < 0 ? 1.0 : (double)op.cols_p)) * elem;
      P->est_bytes += by;
      P->est_fma += A.a < 0 ? 0.0 : nv * (double)op.cols_p;
      P->est_cost += by / bw;
    } else {
      op.kind = A.a < 0 ? OP_GATHER : OP_EMA;
      op.cols_out = (int64_t)ci.nsets(C.size);
      op.ld_out = pad_ld(op.cols_out, elem);
      op.tab_off = build_tabs ? build_table(ci, op.kind, C.size, A.size, &P->tabs, &tcache) : 0;
      op.state_out = table_state[c] = n_states++;
      op.out = table_buf[c] = add_buf(P, "T" + std::to_string(c), rows * op.ld_out * elem, idx);
      P->n_tables++;
      if (A.a < 0) {
        op.alg_bytes = nv * batch + (double)elem * nv * batch * (double)(op.cols_p + op.cols_out);
      } else {
        op.alg_bytes = (double)elem * nv * batch * (double)(op.cols_a + op.cols_p + op.cols_out);
        op.alg_flops = 2.0 * nv * batch * (double)op.cols_out * (double)op.nsplit;
      }
      double by = nv * ((A.a < 0 ? 0.0 : (double)op.cols_a) + (double)op.cols_p + (double)op.cols_out) * elem;
      double fm = A.a < 0 ? 0.0 : nv * (double)op.cols_out * (double)op.nsplit;
      P->est_bytes += by;
      P->est_fma += fm;
      P->est_cost += std::max(by / bw, fm / fma_rate);
    }
    P->n_ema++;
    use_buf(P, op.in_a, idx);
    use_buf(P, op.in_p, idx);
    P->ops.push_back(op);
  }
  P->n_states = n_states;
  P->buf_states = add_buf(P, "states", 8LL * std::max(1, n_states), 0);
  P->scratch_width = max_spmm_width;
  P->buf_scratch = add_buf(P, "spmm_scratch", (int64_t)g->n_seg * max_spmm_width * elem, 0);
  P->buf_hist_heavy = add_buf(P, "hist_heavy", 4LL * g->n_heavy * batch * k, 0);
  const int last = (int)P->ops.size() - 1;
  for (int b : {P->buf_seeds, P->buf_colors, P->buf_out, P->buf_partials, P->buf_states, P->buf_scratch,
                P->buf_hist_heavy}) {
    P->bufs[b].first = 0;
    P->bufs[b].last = last;
  }
  place_buffers(P);
}

sgc_status make_plan(const sgc_graph* g, const sgc_template* t, int precision, int root, int policy, int batch,
                     bool build_tabs, Plan* out) {
  if (root >= t->k) return fail(SGC_ERR_INVALID, "options.root is not a template vertex");
  int best_root = -1, best_policy = 0;
  double best_cost = 0;
  int64_t best_ws = 0;
  for (int r = 0; r < t->k; ++r) {
    if (root >= 0 && r != root) continue;
    for (int pol = 0; pol < 2; ++pol) {
      if (policy >= 0 && pol != policy) continue;
      Plan P;
      plan_for(g, t, precision, r, pol, 1, false, &P);
      if (best_root < 0 || P.est_cost < best_cost * 0.999 ||
          (P.est_cost <= best_cost * 1.001 && P.ws_bytes < best_ws)) {
        best_root = r;
        best_policy = pol;
        best_cost = P.est_cost;
        best_ws = P.ws_bytes;
      }
    }
  }
  plan_for(g, t, precision, best_root, best_policy, batch, build_tabs, out);
  return SGC_OK;
}

}  // namespace sgc
