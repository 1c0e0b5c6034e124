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
