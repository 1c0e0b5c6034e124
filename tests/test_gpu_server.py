"""The continuous-batching counting server (sgc_server_*): each request's result is
the same alone and in a mix of overlapping requests (FP64 exactly, FP32 within the
FP32 tolerance), and equals the oracle; the memory budget, timeouts and teardown
behave as documented."""
import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5

QUERIES = [  # (template, seeds, precision)
    (sgcgen.path_tree(5), [1, 2, 3], "fp64"),
    (sgcgen.pruefer_tree(7, 5), list(range(10, 21)), "fp32"),
    (sgcgen.spider_tree([2, 2, 1]), [4], "fp32"),
    (sgcgen.star_tree(5), [5, 6], "fp64"),
    (sgcgen.pruefer_tree(8, 2), list(range(30, 35)), "fp32"),
    (sgcgen.path_tree(1), [1, 2], "fp32"),
    (sgcgen.pruefer_tree(6, 9), list(range(40, 48)), "fp64"),
]


@pytest.fixture(scope="module")
def graph():
    sgc.build()
    rp, ci = sgcgen.er(4000, 20000, 21)
    return rp, ci, sgc.Graph(rp, ci)


def _run(graph_obj, queries, mixed, budget=2 << 30, inflight=4):
    srv = sgc.Server(graph_obj, budget, inflight)
    tpls = [sgc.Template(p) for p, _, _ in queries]
    out = []
    try:
        if mixed:
            tickets = [srv.submit(t, s, prec) for t, (_, s, prec) in zip(tpls, queries)]
            for tk, (_, s, _) in zip(tickets, queries):
                out.append(srv.wait(tk, len(s)))
        else:
            for t, (_, s, prec) in zip(tpls, queries):
                out.append(srv.wait(srv.submit(t, s, prec), len(s)))
        stats = srv.stats()
    finally:
        srv.close()
    return out, stats


def test_alone_equals_mixed_equals_oracle(graph):
    rp, ci, g = graph
    alone, _ = _run(g, QUERIES, mixed=False)
    mixed, stats = _run(g, QUERIES * 3, mixed=True)
    assert stats["completed"] == 3 * len(QUERIES) and stats["failed"] == 0
    assert stats["peak_inflight"] >= 2  # requests ran at the same time
    assert 0 < stats["latency_p50_ms"] <= stats["latency_p99_ms"]
    n = len(rp) - 1
    for i, (parent, seeds, prec) in enumerate(QUERIES):
        a = alone[i][1]
        want = np.array([float(oracle.count(rp, ci, parent, oracle.colors(s, n, len(parent))).maps)
                         for s in seeds])
        for rep in range(3):
            m = mixed[rep * len(QUERIES) + i][1]
            if prec == "fp64":
                assert np.array_equal(a, m)
            else:
                assert np.allclose(a, m, rtol=FP32_RTOL, atol=0)
        tol = 0.0 if prec == "fp64" else FP32_RTOL
        assert np.all(np.abs(a - want) <= tol * want), (i, a, want)
        # the estimate is the mean of maps / |Aut| * k^k / k!
        k = len(parent)
        import math
        est = np.mean(a) / oracle.automorphisms(parent) * k ** k / math.factorial(k)
        assert abs(alone[i][0] - est) <= 1e-9 * max(est, 1)


def test_request_above_budget_fails_cleanly(graph):
    rp, ci, g = graph
    srv = sgc.Server(g, 1 << 16, 2)  # 64 KB: too small for any table
    try:
        t = sgc.Template(sgcgen.path_tree(6))
        tk = srv.submit(t, [1])
        with pytest.raises(sgc.SgcError) as ei:
            srv.wait(tk, 1)
        assert ei.value.status == sgc.SGC_ERR_OOM
        assert srv.stats()["failed"] == 1
    finally:
        srv.close()


def test_wait_timeout_then_result(graph):
    rp, ci = sgcgen.rmat(16, seed=3)
    g = sgc.Graph(rp, ci)
    srv = sgc.Server(g, 8 << 30, 2)
    try:
        t = sgc.Template(sgcgen.path_tree(12))
        tickets = [srv.submit(t, [i]) for i in range(4)]
        with pytest.raises(sgc.SgcError) as ei:
            srv.wait(tickets[-1], 1, timeout_ms=0)
        assert ei.value.status == sgc.SGC_ERR_TIMEOUT
        for tk in tickets:
            est, maps, lat = srv.wait(tk, 1)
            assert maps[0] > 0 and lat > 0
    finally:
        srv.close()


def test_destroy_with_queued_requests(graph):
    rp, ci, g = graph
    srv = sgc.Server(g, 1 << 30, 1)
    t = sgc.Template(sgcgen.pruefer_tree(8, 4))
    for i in range(20):
        srv.submit(t, list(range(i * 8, i * 8 + 8)))
    srv.close()  # cancels what has not started, waits for what runs; must not hang


def test_passes_of_fewer_colorings_fit_the_request_range():
    # a request's last passes take fewer colorings; a pass of one coloring uses the grouped SpMM and
    # its neighbour-group buffers, which on a graph with many stored entries make its workspace larger
    # than the top pass's: every pass must still fit the range the server gave the request, and the
    # results equal sgc_count's, alone and side by side
    sgc.build()
    rp, ci = sgcgen.rmat(16, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1)
    g = sgc.Graph(rp, ci)
    parent = sgcgen.path_tree(4)
    t = sgc.Template(parent)
    assert sgc.plan(g, t, batch=1)["workspace_bytes"] > sgc.plan(g, t, batch=2)["workspace_bytes"]
    queries = [(parent, [1, 2, 3], "fp64"), (parent, [4, 5, 6, 7, 8], "fp64"),
               (sgcgen.pruefer_tree(6, 3), [9, 10, 11], "fp32")]
    want = [sgc.count(g, sgc.Template(p), s, precision=prec).maps for p, s, prec in queries]
    for mixed in (False, True):
        out, stats = _run(g, queries * (2 if mixed else 1), mixed=mixed, budget=8 << 30)
        assert stats["failed"] == 0
        for i, (_, seeds, prec) in enumerate(queries * (2 if mixed else 1)):
            got = out[i][1]
            ref = want[i % len(queries)]
            if prec == "fp64":
                assert np.array_equal(got, ref), (i, got, ref)
            else:
                assert np.allclose(got, ref, rtol=FP32_RTOL, atol=0), (i, got, ref)
