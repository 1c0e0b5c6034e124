"""Templates of 17 and 18 vertices (the largest supported, k = |T| colors: relative color sets of
up to C(17, 8) = 24310 per row) against the exact oracle on a small graph: FP64 exactly while every
count is below 2^53, FP32 within 1e-5."""
import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu


SEEDS = [1, 2]
PARENTS = (sgcgen.path_tree(18), sgcgen.pruefer_tree(17, 3), sgcgen.spider_tree([6, 6, 5]))


@pytest.fixture(scope="module")
def case():
    sgc.build()
    rp, ci = sgcgen.er(160, 1100, 4)
    n = len(rp) - 1
    want = [[oracle.count(rp, ci, p, oracle.colors(s, n, len(p))) for s in SEEDS] for p in PARENTS]
    return sgc.Graph(rp, ci), want


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_largest_templates_match_oracle(case, precision):
    g, oracle_res = case
    for parent, res in zip(PARENTS, oracle_res):
        t = sgc.Template(parent)
        seeds = SEEDS
        want = np.array([float(r.maps) for r in res])
        got = sgc.count(g, t, seeds, precision=precision).maps
        if precision == "fp64" and all(r.max_intermediate < 2 ** 53 for r in res):
            assert np.array_equal(got, want), (len(parent), got, want)
        else:
            assert np.allclose(got, want, rtol=1e-5 if precision == "fp32" else 1e-12, atol=0), (got, want)
        assert want.max() > 0
