"""Pins for the CPU oracle (no GPU): every check compares the oracle with
something other than itself - enumeration, closed forms, textbook
definitions - chosen so that a dropped term, a wrong index or a transposed
operand in the dynamic program fails at least one of them."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import sgcgen
from tests import pins

SMALL_TREES = [
    sgcgen.path_tree(1), sgcgen.path_tree(2), sgcgen.path_tree(3), sgcgen.path_tree(4), sgcgen.path_tree(5),
    sgcgen.star_tree(4), sgcgen.star_tree(5), sgcgen.spider_tree([1, 1, 2]), sgcgen.spider_tree([2, 1]),
    sgcgen.pruefer_tree(5, 3), sgcgen.pruefer_tree(6, 11), sgcgen.pruefer_tree(6, 4),
    np.array([2, 2, -1, 1, 1], dtype=np.int32),   # root not at vertex 0, children out of index order
]


def _small_graphs():
    yield "er8", sgcgen.er(8, 14, 1)
    yield "er9", sgcgen.er(9, 18, 2)
    # a hub joined to a path: mixes high and low degrees
    yield "hub", sgcgen.from_edges(9, [(0, i) for i in range(1, 7)] + [(1, 2), (2, 3), (3, 7), (7, 8), (8, 5)])


@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("name,graph", list(_small_graphs()))
def test_brute_force_matches_dp(name, graph, wide):
    # both builds of the oracle: 128-bit counts and 192-bit limbs
    rp, ci = graph
    n = len(rp) - 1
    for parent in SMALL_TREES:
        k = len(parent)
        if k > 6:
            continue
        for seed in (1, 2, 3):
            cols = oracle.colors(seed, n, k)
            want = pins.brute_force_maps(rp, ci, parent, cols)
            got = oracle.count(rp, ci, parent, cols, wide=wide)
            assert got.maps == want, (name, list(parent), seed)
            assert oracle.count(rp, ci, parent, cols, mode="literal", wide=wide).maps == want


def test_brute_force_with_spread_colors():
    # colorings that are all-colorful make every embedding count
    rp, ci = sgcgen.er(7, 12, 5)
    for parent in SMALL_TREES:
        k = len(parent)
        if k > 6:
            continue
        cols = np.arange(7) % k
        assert oracle.count(rp, ci, parent, cols).maps == pins.brute_force_maps(rp, ci, parent, cols)


def test_star_closed_form_per_coloring():
    rp, ci = sgcgen.er(300, 1500, 3)
    for k in (3, 4, 5):
        star = sgcgen.star_tree(k)
        aut = math.factorial(k - 1)
        for seed in (1, 7, 19):
            cols = oracle.colors(seed, 300, k)
            r = oracle.count(rp, ci, star, cols)
            assert r.maps % aut == 0
            assert r.maps // aut == pins.star_copies(rp, ci, cols, k)


def test_star_closed_form_skewed_graph():
    rp, ci = sgcgen.rmat(9, edge_factor=8, seed=3)
    k = 4
    cols = oracle.colors(5, len(rp) - 1, k)
    r = oracle.count(rp, ci, sgcgen.star_tree(k), cols)
    assert r.maps == math.factorial(k - 1) * pins.star_copies(rp, ci, cols, k)


def test_complete_graph_any_tree():
    for nn in (6, 9, 12):
        rp, ci = sgcgen.complete_graph(nn)
        for parent in [sgcgen.path_tree(4), sgcgen.path_tree(5), sgcgen.star_tree(5), sgcgen.pruefer_tree(6, 2),
                       sgcgen.spider_tree([2, 2, 1])]:
            k = len(parent)
            for seed in (1, 2):
                cols = oracle.colors(seed, nn, k)
                assert oracle.count(rp, ci, parent, cols).maps == pins.complete_graph_maps(cols, k)


def test_complete_graph_path_expectation():
    # E[colorful paths] * k^k/k! = n!/((n-k)! * 2) copies of P_k in K_n: exact over all colorings of K_n
    # is too many; average the exact closed form per coloring instead over many seeds and compare with
    # the oracle on a subset.
    nn, k = 7, 4
    rp, ci = sgcgen.complete_graph(nn)
    total = Fraction(0)
    for cols in itertools.product(range(k), repeat=nn):
        total += pins.complete_graph_maps(cols, k)
    mean_maps = total / k ** nn
    copies = mean_maps / 2 * Fraction(k ** k, math.factorial(k))
    assert copies == Fraction(math.factorial(nn), math.factorial(nn - k) * 2)


@pytest.mark.parametrize("parent", SMALL_TREES + [sgcgen.pruefer_tree(7, s) for s in range(1, 6)]
                         + [sgcgen.spider_tree([2, 2, 2]), sgcgen.star_tree(7)])
def test_automorphisms_brute(parent):
    assert oracle.automorphisms(parent) == pins.aut_brute(parent)


def test_automorphisms_closed_forms():
    assert oracle.automorphisms(sgcgen.path_tree(1)) == 1
    for k in range(2, 16):
        assert oracle.automorphisms(sgcgen.path_tree(k)) == 2
    for k in range(3, 12):
        assert oracle.automorphisms(sgcgen.star_tree(k)) == math.factorial(k - 1)
    assert oracle.automorphisms(sgcgen.spider_tree([3, 3, 3])) == 6
    assert oracle.automorphisms(sgcgen.spider_tree([3, 3, 2])) == 2
    assert oracle.automorphisms(sgcgen.spider_tree([1, 2, 3])) == 1


def test_root_choice_invariance():
    rp, ci = sgcgen.er(60, 200, 4)
    for parent in [sgcgen.pruefer_tree(6, 5), sgcgen.spider_tree([1, 2, 2]), sgcgen.path_tree(6)]:
        k = len(parent)
        cols = oracle.colors(9, 60, k)
        ref = oracle.count(rp, ci, parent, cols).maps
        for r in range(k):
            assert oracle.count(rp, ci, parent, cols, root=r).maps == ref


def test_literal_equals_pruned():
    # Eq. 2: hoisting the neighbour sum is an exact identity in integers
    rp, ci = sgcgen.er(120, 500, 8)
    for parent in [sgcgen.pruefer_tree(6, 1), sgcgen.spider_tree([2, 2, 1])]:
        k = len(parent)
        cols = oracle.colors(3, 120, k)
        a = oracle.count(rp, ci, parent, cols)
        b = oracle.count(rp, ci, parent, cols, mode="literal")
        assert a.maps == b.maps


def test_special_templates():
    rp, ci = sgcgen.er(100, 300, 6)
    n = 100
    # k = 1: every vertex is one colorful map
    assert oracle.count(rp, ci, sgcgen.path_tree(1), np.zeros(n, np.uint8)).maps == n
    # k = 2: ordered edges whose ends differ in color
    cols = oracle.colors(2, n, 2)
    assert oracle.count(rp, ci, sgcgen.path_tree(2), cols).maps == pins.bichromatic_edge_maps(rp, ci, cols)


def test_maps_divisible_by_aut():
    rp, ci = sgcgen.er(200, 900, 12)
    for parent in [sgcgen.spider_tree([2, 2, 2]), sgcgen.star_tree(5), sgcgen.path_tree(6)]:
        k = len(parent)
        aut = oracle.automorphisms(parent)
        for seed in (1, 2, 3):
            assert oracle.count(rp, ci, parent, oracle.colors(seed, 200, k)).maps % aut == 0


def test_tree_in_itself_is_aut():
    for parent in [sgcgen.pruefer_tree(8, 3), sgcgen.spider_tree([2, 3, 1])]:
        rp, ci = sgcgen.tree_graph(parent)
        k = len(parent)
        assert oracle.count(rp, ci, parent, np.arange(k)).maps == pins.aut_brute(parent)


def test_star_expectation_unbiased():
    # E[estimate] = number of copies of K_{1,k-1} = sum_v C(deg v, k-1); the color-coding estimator is
    # unbiased (Section 2.1: a copy is colorful with probability k!/k^k).
    rp, ci = sgcgen.er(40, 90, 21)
    k = 3
    deg = np.diff(rp)
    truth = sum(math.comb(int(d), k - 1) for d in deg)
    e = oracle.estimate(rp, ci, sgcgen.star_tree(k), list(range(1, 3001)))
    ests = np.array(e.estimates)
    se = ests.std(ddof=1) / math.sqrt(len(ests))
    assert abs(e.mean - truth) < 5 * se, (e.mean, truth, se)


def test_colorset_index_bijection_and_colex():
    for k in range(1, 13):
        for h in range(0, k + 1):
            subsets = list(itertools.combinations(range(k), h))
            idx = [oracle.colorset_index(list(s)) for s in subsets]
            assert sorted(idx) == list(range(math.comb(k, h)))
            # colex order: compare by largest element first
            order = sorted(subsets, key=lambda s: tuple(reversed(s)))
            assert [oracle.colorset_index(list(s)) for s in order] == list(range(math.comb(k, h)))
            for s, i in zip(subsets, idx):
                assert oracle.colorset_unindex(i, h, k) == list(s)


def test_coloring_matches_published_splitmix64():
    for seed in (0, 1, 2, 12345, 2 ** 63 + 5):
        for k in (2, 5, 10, 15):
            cols = oracle.colors(seed, 300, k)
            assert [int(c) for c in cols] == [pins.color_of(seed, v, k) for v in range(300)]
    # the input generator's copy of the same stream agrees with the published definition
    assert all(sgcgen.splitmix64_draw(77, j) == pins.splitmix64(77, j) for j in range(50))


def test_coloring_roughly_uniform():
    cols = oracle.colors(1, 100000, 10)
    counts = np.bincount(cols, minlength=10)
    assert counts.min() > 9500 and counts.max() < 10500


def test_invalid_templates_rejected():
    rp, ci = sgcgen.er(10, 20, 1)
    cols = np.zeros(10, np.uint8)
    with pytest.raises(ValueError):
        oracle.count(rp, ci, np.array([-1, -1, 0], np.int32), cols)   # two roots
    with pytest.raises(ValueError):
        oracle.count(rp, ci, np.array([1, 2, 0], np.int32), cols)     # cycle, no root
    with pytest.raises(ValueError):
        oracle.count(rp, ci, np.array([-1, 0], np.int32), np.full(10, 3, np.uint8))  # color >= k


# ---------------------------------------------------------------- k > |T| colors
# Section 2.1 draws colors from k >= |T|; a map is colorful when its |T| images
# get |T| distinct colors, and the estimate divides by k! / ((k - |T|)! k^|T|).

@pytest.mark.parametrize("name,graph", list(_small_graphs()))
def test_more_colors_brute_force(name, graph):
    rp, ci = graph
    n = len(rp) - 1
    for parent in SMALL_TREES:
        t = len(parent)
        if t > 5:
            continue
        for extra in (1, 2):
            k = t + extra
            for seed in (1, 2):
                cols = oracle.colors(seed, n, k)
                want = pins.brute_force_maps(rp, ci, parent, cols)
                assert oracle.count(rp, ci, parent, cols, ncolors=k).maps == want, (name, list(parent), k, seed)
                assert oracle.count(rp, ci, parent, cols, ncolors=k, mode="literal").maps == want


def test_more_colors_complete_graph():
    # K_n: every injective map is edge-preserving, so the colorful maps of a t-tree are the ordered
    # t-tuples of vertices with distinct colors: t! * e_t(n_0, ..., n_{k-1}) (elementary symmetric)
    n = 30
    rp, ci = sgcgen.complete_graph(n)
    for parent, k in ((sgcgen.path_tree(4), 6), (sgcgen.pruefer_tree(5, 2), 7), (sgcgen.star_tree(3), 9)):
        t = len(parent)
        for seed in (3, 4):
            counts = np.bincount(oracle.colors(seed, n, k), minlength=k)
            e_t = sum(math.prod(int(counts[c]) for c in S) for S in itertools.combinations(range(k), t))
            assert oracle.count(rp, ci, parent, oracle.colors(seed, n, k), ncolors=k).maps == \
                math.factorial(t) * e_t


def test_more_colors_estimate_unbiased():
    # E[estimate] with k = |T| + 2 colors is still the number of copies (the star closed form)
    rp, ci = sgcgen.er(40, 90, 21)
    t = 3
    truth = sum(math.comb(int(d), t - 1) for d in np.diff(rp))
    e = oracle.estimate(rp, ci, sgcgen.star_tree(t), list(range(1, 3001)), ncolors=t + 2)
    ests = np.array(e.estimates)
    se = ests.std(ddof=1) / math.sqrt(len(ests))
    assert abs(e.mean - truth) < 5 * se, (e.mean, truth, se)
    assert oracle.colorful_probability(3, 5) == Fraction(5 * 4 * 3, 5 ** 3)


def test_more_colors_rejects_too_few():
    rp, ci = sgcgen.er(8, 14, 1)
    with pytest.raises(Exception):
        oracle.count(rp, ci, sgcgen.path_tree(4), oracle.colors(1, 8, 3), ncolors=3)


# ------------------------------------------------ the largest intermediate
# max_intermediate decides whether an FP64 computation of the same DP is exact
# (every value below 2^53), so it is pinned against enumeration and closed forms.

@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("name,graph", list(_small_graphs()))
def test_max_intermediate_brute_force(name, graph, wide):
    rp, ci = graph
    n = len(rp) - 1
    for parent in SMALL_TREES:
        k = len(parent)
        if k > 5 or k < 2:
            continue
        for cols in [oracle.colors(1, n, k), oracle.colors(2, n, k), np.arange(n) % k]:
            want = pins.brute_max_intermediate(rp, ci, parent, cols)
            assert oracle.count(rp, ci, parent, cols, wide=wide).max_intermediate == want, (name, list(parent))


def test_max_intermediate_monochrome_is_max_degree():
    # one color everywhere: no sub-template of two or more vertices is colorful, so every combined
    # table and the final sum are 0; a leaf's neighbour-sum buffer holds deg(v) at the set {0}
    rp, ci = sgcgen.rmat(10, edge_factor=8, seed=2)
    n = len(rp) - 1
    maxdeg = int(np.diff(rp).max())
    for parent in [sgcgen.path_tree(3), sgcgen.star_tree(5), sgcgen.pruefer_tree(7, 4)]:
        r = oracle.count(rp, ci, parent, np.zeros(n, np.uint8))
        assert r.maps == 0
        assert r.max_intermediate == max(1, maxdeg)


def test_max_intermediate_star_graph_edge_template():
    # K_{1,m}, hub color 0, leaves color 1, the 2-vertex template: the hub's neighbour sum for {1} is m,
    # its root-table entry m, each leaf's 1, and the total 2m, the largest value
    for m in (1, 5, 40):
        rp, ci = sgcgen.from_edges(m + 1, [(0, i) for i in range(1, m + 1)])
        cols = np.array([0] + [1] * m, np.uint8)
        r = oracle.count(rp, ci, sgcgen.path_tree(2), cols)
        assert r.maps == 2 * m
        assert r.max_intermediate == 2 * m


# ---------------------------------------------- counts beyond 128 bits
# Exact counts of 15-vertex trees on R-MAT graphs of 2^16 vertices exceed 2^128; the oracle then
# recomputes them with 192-bit limbs.  Pinned by the star closed form past 2^128.

def test_wide_counts_star_closed_form_beyond_128_bits():
    # K_{1,14} in a star graph whose hub (color 0) has h leaves of each color 1..14: the hub is the
    # only centre, copies = h^14, maps = 14! * h^14 (|Aut| = 14!), about 2^134 for h = 128
    h, k = 128, 15
    leaves = [(0, 1 + c * h + i) for c in range(k - 1) for i in range(h)]
    rp, ci = sgcgen.from_edges(1 + (k - 1) * h, leaves)
    cols = np.array([0] + [1 + c for c in range(k - 1) for _ in range(h)], np.uint8)
    want = math.factorial(k - 1) * h ** (k - 1)
    assert want > 2 ** 128
    with pytest.raises(oracle.OracleOverflow):
        oracle.count(rp, ci, sgcgen.star_tree(k), cols, wide=False)
    r = oracle.count(rp, ci, sgcgen.star_tree(k), cols)
    assert r.maps == want
    assert r.max_intermediate == want
    assert oracle.count(rp, ci, sgcgen.star_tree(k), cols, wide=True).maps == want


def test_wide_equals_narrow_below_128_bits():
    rp, ci = sgcgen.rmat(10, edge_factor=8, seed=5)
    n = len(rp) - 1
    for parent in [sgcgen.pruefer_tree(9, 3), sgcgen.spider_tree([3, 3, 2])]:
        cols = oracle.colors(4, n, len(parent))
        a = oracle.count(rp, ci, parent, cols, wide=False, per_vertex=True)
        b = oracle.count(rp, ci, parent, cols, wide=True, per_vertex=True)
        assert (a.maps, a.max_intermediate, a.per_vertex) == (b.maps, b.max_intermediate, b.per_vertex)
