"""The (eps, delta) driver: sgc_estimate stops by its rule, on the oracle's numbers.

The estimate it returns must be the mean of the oracle's per-coloring estimates
(maps / |Aut(T)| * k^k / k!, Section 2.1) over exactly the seeds it used, and the
normal-approximation stopping rule must hold at the count it stopped at and fail
one chunk earlier.
"""
import math
import statistics

import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu


def rule(estimates, eps, delta):
    n = len(estimates)
    m = statistics.fmean(estimates)
    s = statistics.stdev(estimates) if n > 1 else 0.0
    z = statistics.NormalDist().inv_cdf(1 - delta / 2)
    return z * s / math.sqrt(n), m


@pytest.mark.parametrize("eps,delta,chunk", [(0.05, 0.05, 8), (0.02, 0.1, 16)])
def test_estimate_stops_by_its_rule(eps, delta, chunk):
    sgc.build()
    rp, ci = sgcgen.er(1500, 9000, 17)
    parent = sgcgen.pruefer_tree(5, 1005)
    g = sgc.Graph(rp, ci)
    t = sgc.Template(parent)
    opt = sgc.sgc_options_init(precision=sgc.SGC_FP64, batch=chunk)
    est, n, rel = sgc.sgc_estimate(g.handle, t.handle, eps, delta, first_seed=500, min_iter=2 * chunk,
                                   max_iter=4096, opt=opt)
    assert 2 * chunk <= n <= 4096 and n % chunk == 0
    ref = oracle.estimate(rp, ci, parent, [500 + i for i in range(n)])
    assert est == pytest.approx(ref.mean, rel=1e-12)
    half, m = rule(ref.estimates, eps, delta)
    assert rel == pytest.approx(half / m, rel=1e-9)
    if n < 4096:
        assert half <= eps * m * (1 + 1e-12)
    if n > 2 * chunk:  # one chunk earlier the rule did not hold yet
        half0, m0 = rule(ref.estimates[:n - chunk], eps, delta)
        assert half0 > eps * m0


def test_estimate_caps_at_max_iter():
    sgc.build()
    rp, ci = sgcgen.er(800, 3000, 5)
    g = sgc.Graph(rp, ci)
    t = sgc.Template(sgcgen.path_tree(6))
    est, n, rel = sgc.sgc_estimate(g.handle, t.handle, 1e-6, 0.01, first_seed=1, max_iter=24,
                                   opt=sgc.sgc_options_init(precision=sgc.SGC_FP64, batch=8))
    assert n == 24 and rel > 1e-6
    ref = oracle.estimate(rp, ci, sgcgen.path_tree(6), list(range(1, 25)))
    assert est == pytest.approx(ref.mean, rel=1e-12)
