"""Independent checks that pin the oracle: brute force, closed forms, textbook
definitions.  Nothing here calls the oracle or the CUDA library, and nothing
here shares code with either.

* ``brute_force_maps``: enumerate every injective map of the template's
  vertices into the graph's and keep those that preserve edges and use k
  distinct colors (the problem statement of Section 2.1, by definition).
* ``star_copies``: colorful copies of the star K_{1,k-1} centred at v are the
  ways to pick one neighbour of each color other than c(v):
  prod_{c != c(v)} h_c(v).
* ``complete_graph_maps``: in K_n every injective map is edge-preserving, so
  the colorful maps of any k-vertex tree are k! * prod_c n_c (assign the k
  template vertices a bijection onto the colors, then a vertex of that
  color).
* ``aut_brute``: automorphisms of a tree by checking all vertex permutations.
* ``splitmix64``: the published SplitMix64 output function in Python ints.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed: int, j: int) -> int:
    z = (seed + (j + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def color_of(seed: int, v: int, k: int) -> int:
    return ((splitmix64(seed, v) >> 32) * k) >> 32


def edges_of(parent):
    return [(i, int(p)) for i, p in enumerate(parent) if p >= 0]


def adjacency_sets(row_ptr, col_idx):
    n = len(row_ptr) - 1
    return [set(int(x) for x in col_idx[row_ptr[v]:row_ptr[v + 1]]) for v in range(n)]


def brute_force_maps(row_ptr, col_idx, parent, cols) -> int:
    """Colorful injective edge-preserving maps T -> G, by enumeration."""
    adj = adjacency_sets(row_ptr, col_idx)
    n = len(adj)
    k = len(parent)
    tedges = edges_of(parent)
    total = 0
    for phi in itertools.permutations(range(n), k):
        if len({int(cols[x]) for x in phi}) != k:
            continue
        if all(phi[b] in adj[phi[a]] for a, b in tedges):
            total += 1
    return total


def star_copies(row_ptr, col_idx, cols, k) -> int:
    """Colorful copies of K_{1,k-1} (k >= 3): sum_v prod_{c != c(v)} h_c(v)."""
    n = len(row_ptr) - 1
    total = 0
    for v in range(n):
        h = [0] * k
        for u in col_idx[row_ptr[v]:row_ptr[v + 1]]:
            h[int(cols[u])] += 1
        prod = 1
        for c in range(k):
            if c != int(cols[v]):
                prod *= h[c]
        total += prod
    return total


def complete_graph_maps(cols, k) -> int:
    counts = np.bincount(np.asarray(cols, dtype=np.int64), minlength=k)
    prod = 1
    for c in range(k):
        prod *= int(counts[c])
    return math.factorial(k) * prod


def aut_brute(parent) -> int:
    k = len(parent)
    es = [tuple(e) for e in edges_of(parent)]
    eset = {frozenset(e) for e in es}
    count = 0
    for perm in itertools.permutations(range(k)):
        if all(frozenset((perm[a], perm[b])) in eset for a, b in es):
            count += 1
    return count


def bichromatic_edge_maps(row_ptr, col_idx, cols) -> int:
    """Colorful maps of the 2-vertex template: ordered edges with distinct end colors."""
    n = len(row_ptr) - 1
    return sum(1 for v in range(n) for u in col_idx[row_ptr[v]:row_ptr[v + 1]] if cols[v] != cols[u])


def rooted_children(parent, root=None):
    """Children lists of the tree rooted at `root` (default: the entry -1), each ascending: the
    partition order of Section 2.1, item 2, with children cut in index order."""
    k = len(parent)
    adj = [[] for _ in range(k)]
    for i, p in enumerate(parent):
        if p >= 0:
            adj[i].append(int(p))
            adj[int(p)].append(i)
    if root is None:
        root = [i for i, p in enumerate(parent) if p < 0][0]
    kids = [[] for _ in range(k)]
    seen = {root}
    order = [root]
    for x in order:
        for y in sorted(adj[x]):
            if y not in seen:
                seen.add(y)
                kids[x].append(y)
                order.append(y)
    return root, kids


def _subtree(kids, x):
    out = [x]
    for c in kids[x]:
        out += _subtree(kids, c)
    return out


def rooted_embedding_counts(adj, cols, vertices, edges, root):
    """N(v, S, C) by enumeration: injective edge-preserving maps of the rooted sub-template S
    (vertex list, edge list, root) into the graph, grouped by the image of the root and the set of
    image colors, kept only when the image colors are distinct."""
    n = len(adj)
    pos = {x: i for i, x in enumerate(vertices)}
    counts = {}
    for phi in itertools.permutations(range(n), len(vertices)):
        cset = frozenset(int(cols[y]) for y in phi)
        if len(cset) != len(vertices):
            continue
        if all(phi[pos[b]] in adj[phi[pos[a]]] for a, b in edges):
            key = (phi[pos[root]], cset)
            counts[key] = counts.get(key, 0) + 1
    return counts


def brute_max_intermediate(row_ptr, col_idx, parent, cols, root=None):
    """Largest value the DP of Section 2.1 holds, found without the DP: every sub-template table
    (x with the subtrees of its children j, j+1, ...), every neighbour-sum buffer
    P(v, C) = sum_{u in N(v)} N(u, T_p, C) over all |T_p|-sets C, every vertex's root-table sum and
    the total, with each table entry counted by enumerating embeddings.  Entries that are zero
    are included (so the result is at least 0, and 1 once a leaf table exists)."""
    adj = adjacency_sets(row_ptr, col_idx)
    n = len(adj)
    r, kids = rooted_children(parent, root)
    tree_edges = edges_of(parent)
    best = 0

    def sub_vertices(x, j):
        out = [x]
        for c in kids[x][j:]:
            out += _subtree(kids, c)
        return out

    def table(x, j):
        vs = sub_vertices(x, j)
        vset = set(vs)
        es = [(a, b) for a, b in tree_edges if a in vset and b in vset]
        return rooted_embedding_counts(adj, cols, vs, es, x)

    for x in range(len(parent)):
        for j in range(len(kids[x]) + 1):
            t = table(x, j)
            if n > 0:
                best = max(best, max(t.values(), default=0), 1 if j == len(kids[x]) else 0)
            if j < len(kids[x]):
                tp = table(kids[x][j], 0)
                psum = {}
                for (u, cset), c in tp.items():
                    for v in adj[u]:
                        psum[(v, cset)] = psum.get((v, cset), 0) + c
                best = max(best, max(psum.values(), default=0))
    full = table(r, 0)
    rows = [0] * n
    for (v, _), c in full.items():
        rows[v] += c
    best = max([best, sum(rows)] + rows)
    return best
