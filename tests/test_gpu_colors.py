"""More colors than template vertices (Section 2.1: colors drawn from k >= |T|).

The GPU path with sgc_options.colors = k > |T| must give the exact oracle's
colorful maps (sum of the root table over every |T|-subset of colors) per
coloring - FP64 exactly, FP32 within 1e-5 - and the estimate that divides by
the colorful probability k! / ((k - |T|)! k^|T|).
"""
import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("extra", [1, 3])
def test_more_colors_match_oracle(precision, extra):
    sgc.build()
    rp, ci = sgcgen.rmat(11, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=9)
    n = len(rp) - 1
    g = sgc.Graph(rp, ci)
    # root active child a single vertex (the root table is the passive P) and a general root eMA
    for parent in (sgcgen.path_tree(4), sgcgen.spider_tree([2, 2, 1]), sgcgen.pruefer_tree(6, 1006),
                   sgcgen.star_tree(5)):
        t = len(parent)
        k = t + extra
        tp = sgc.Template(parent)
        seeds = list(range(300, 311))  # passes of 8 + 2 + 1 colorings
        r = sgc.count(g, tp, seeds, precision=precision, colors=k)
        ref = oracle.estimate(rp, ci, parent, seeds, ncolors=k)
        want = np.array(ref.maps, dtype=np.float64)
        if precision == "fp64" and ref.max_intermediate < 2 ** 53:
            assert np.array_equal(r.maps, want), (list(parent), k, r.maps, want)
        else:
            tol = 1e-12 if precision == "fp64" else 1e-5
            assert np.allclose(r.maps, want, rtol=tol, atol=0), (list(parent), k, r.maps, want)
        assert r.estimate == pytest.approx(ref.mean, rel=1e-12 if precision == "fp64" else 1e-5)


def test_colors_out_of_range_rejected():
    sgc.build()
    rp, ci = sgcgen.er(200, 600, 3)
    g = sgc.Graph(rp, ci)
    t = sgc.Template(sgcgen.path_tree(5))
    for bad in (4, sgc.SGC_MAX_K + 1):
        with pytest.raises(sgc.SgcError) as ei:
            sgc.count(g, t, [1, 2], colors=bad)
        assert ei.value.status == sgc.SGC_ERR_INVALID
