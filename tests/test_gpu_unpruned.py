"""The ablations (sgc_options.unpruned): Algorithm 1's loop order on the GPU (1), and the pruned
neighbour sums taken one passive column at a time instead of by the row-wise SpMM (2).

Without the hoisted neighbour sums of Eq. 2 every combine takes the neighbour
sum again for each color set and split; the counts must not change: exact
oracle maps in FP64 (the oracle's literal mode is the same loop order), FP32
within 1e-5, also with more colors than template vertices.
"""
import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_unpruned_matches_oracle(precision):
    sgc.build()
    rp, ci = sgcgen.rmat(10, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=12)
    g = sgc.Graph(rp, ci)
    n = len(rp) - 1
    for parent, extra in ((sgcgen.path_tree(4), 0), (sgcgen.spider_tree([2, 2, 1]), 0),
                          (sgcgen.pruefer_tree(6, 1006), 0), (sgcgen.star_tree(5), 0),
                          (sgcgen.pruefer_tree(5, 1005), 2)):
        t = len(parent)
        k = t + extra
        tp = sgc.Template(parent)
        seeds = list(range(40, 51))  # 8 + 2 + 1
        r = sgc.count(g, tp, seeds, precision=precision, unpruned=True, colors=k if extra else 0)
        res = [oracle.count(rp, ci, parent, oracle.colors(s, n, k), ncolors=k, mode="literal") for s in seeds]
        want = np.array([x.maps for x in res], dtype=np.float64)
        if precision == "fp64" and max(x.max_intermediate for x in res) < 2 ** 53:
            assert np.array_equal(r.maps, want), (list(parent), k, r.maps, want)
        else:
            tol = 1e-12 if precision == "fp64" else 1e-5
            assert np.allclose(r.maps, want, rtol=tol, atol=0), (list(parent), k, r.maps, want)
        pruned = sgc.count(g, tp, seeds, precision=precision, colors=k if extra else 0)
        assert np.allclose(pruned.maps, r.maps, rtol=1e-5 if precision == "fp32" else 0, atol=0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pruned_by_column_matches_oracle(precision):
    # the pruned sums of Section 4.2 one column at a time (thread per vertex and column): the oracle's
    # counts (FP64 exactly while below 2^53), heavy rows included
    sgc.build()
    rp, ci = sgcgen.rmat(12, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=12)
    g = sgc.Graph(rp, ci)
    assert g.stats()["n_heavy"] > 0
    n = len(rp) - 1
    for parent, extra in ((sgcgen.spider_tree([3, 3, 3]), 0), (sgcgen.pruefer_tree(8, 1008), 0),
                          (sgcgen.pruefer_tree(6, 1006), 2)):
        k = len(parent) + extra
        tp = sgc.Template(parent)
        seeds = list(range(60, 71))  # 8 + 2 + 1
        r = sgc.count(g, tp, seeds, precision=precision, unpruned=2, colors=k if extra else 0)
        res = [oracle.count(rp, ci, parent, oracle.colors(s, n, k), ncolors=k) for s in seeds]
        want = np.array([x.maps for x in res], dtype=np.float64)
        if precision == "fp64" and max(x.max_intermediate for x in res) < 2 ** 53:
            assert np.array_equal(r.maps, want), (list(parent), k, r.maps, want)
        else:
            tol = 1e-12 if precision == "fp64" else 1e-5
            assert np.allclose(r.maps, want, rtol=tol, atol=0), (list(parent), k, r.maps, want)
