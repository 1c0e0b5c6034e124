"""GPU parity: the CUDA path through the C ABI against the exact CPU oracle.

Tolerances:
* FP64 tables: bit-exact while the oracle's largest intermediate value is
  below 2^53 (every partial sum is then an exactly representable integer, so
  summation order cannot matter); otherwise relative 1e-12.
* FP32 tables: relative error per coloring at most 1e-5 (FP32 accumulation
  inside SpMM and eMA, FP64 final reduction).
"""
import os

import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5
FP64_RTOL_BEYOND_2_53 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    sgc.build()


def _oracle_maps(rp, ci, parent, seeds):
    n = len(rp) - 1
    k = len(parent)
    res = [oracle.count(rp, ci, parent, oracle.colors(int(s), n, k)) for s in seeds]
    return [r.maps for r in res], max(r.max_intermediate for r in res)


def _check(got, want, mx, precision):
    got = np.asarray(got)
    for g, w in zip(got, want):
        if precision == "fp64":
            if mx < 2 ** 53:
                assert g == float(w), (g, w)
            else:
                assert abs(g - w) <= FP64_RTOL_BEYOND_2_53 * w
        else:
            if w == 0:
                assert g == 0.0
            else:
                assert abs(g - w) <= FP32_RTOL * w, (g, w, abs(g - w) / w)


TREES = {
    "p1": sgcgen.path_tree(1), "p2": sgcgen.path_tree(2), "p3": sgcgen.path_tree(3), "p5": sgcgen.path_tree(5),
    "p7": sgcgen.path_tree(7), "star5": sgcgen.star_tree(5), "star7": sgcgen.star_tree(7),
    "spider222": sgcgen.spider_tree([2, 2, 2]), "spider123": sgcgen.spider_tree([1, 2, 3]),
    "pr6": sgcgen.pruefer_tree(6, 3), "pr8": sgcgen.pruefer_tree(8, 5), "pr9": sgcgen.pruefer_tree(9, 2),
    "rootless0": np.array([2, 2, -1, 1, 1, 3], dtype=np.int32),
}


@pytest.fixture(scope="module")
def er_small():
    rp, ci = sgcgen.er(3000, 15000, 4)
    return rp, ci, sgc.Graph(rp, ci)


@pytest.mark.parametrize("name", list(TREES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_small_trees_er(er_small, name, precision):
    rp, ci, g = er_small
    parent = TREES[name]
    seeds = [1, 2, 3]
    want, mx = _oracle_maps(rp, ci, parent, seeds)
    r = sgc.count(g, sgc.Template(parent), seeds, precision=precision)
    _check(r.maps, want, mx, precision)


def test_c1_er2000_path5_exact():
    # Erdos-Renyi G(n=2000, avg degree 10), seed 1; 5-vertex path; k = 5; one coloring; FP64 tables
    rp, ci = sgcgen.er(2000, 10000, 1)
    parent = sgcgen.path_tree(5)
    want = oracle.estimate(rp, ci, parent, [1])
    g = sgc.Graph(rp, ci)
    r = sgc.count(g, sgc.Template(parent), [1], precision="fp64")
    assert want.max_intermediate < 2 ** 53
    assert r.maps[0] == float(want.maps[0])
    assert abs(r.estimate - want.mean) <= 1e-12 * want.mean
    r32 = sgc.count(g, sgc.Template(parent), [1], precision="fp32")
    assert abs(r32.maps[0] - want.maps[0]) <= FP32_RTOL * want.maps[0]


def test_heavy_rows_and_isolated_vertices():
    # hubs far above the segment length plus isolated vertices and a ragged tail
    hub_edges = [(0, i) for i in range(1, 1500)] + [(1, i) for i in range(2, 900)] + [(2, i) for i in range(1000, 1400)]
    rp0, ci0 = sgcgen.er(1600, 4000, 9)
    edges = set(hub_edges)
    for v in range(1600):
        for u in ci0[rp0[v]:rp0[v + 1]]:
            if v < u:
                edges.add((v, int(u)))
    n = 1700  # vertices 1600..1699 are isolated
    rp, ci = sgcgen.from_edges(n, sorted(edges))
    g = sgc.Graph(rp, ci)
    st = g.stats()
    assert st["n_heavy"] >= 3 and st["n_active"] < n
    for parent in (sgcgen.path_tree(4), sgcgen.spider_tree([2, 1, 1]), sgcgen.pruefer_tree(6, 8)):
        want, mx = _oracle_maps(rp, ci, parent, [5, 6])
        for precision in ("fp64", "fp32"):
            _check(sgc.count(g, sgc.Template(parent), [5, 6], precision=precision).maps, want, mx, precision)


def test_small_segment_length_spans_many_segments():
    os.environ["SGC_SEG_LEN"] = "32"
    try:
        rp, ci = sgcgen.rmat(11, edge_factor=8, seed=2)
        g = sgc.Graph(rp, ci)
    finally:
        del os.environ["SGC_SEG_LEN"]
    assert g.stats()["n_segments"] > g.stats()["n_heavy"] > 10
    parent = sgcgen.pruefer_tree(7, 4)
    want, mx = _oracle_maps(rp, ci, parent, [1, 2])
    for precision in ("fp64", "fp32"):
        _check(sgc.count(g, sgc.Template(parent), [1, 2], precision=precision).maps, want, mx, precision)


def test_batching_is_invisible():
    # 13 colorings run as passes of 8 + 4 + 1; each must equal its own single run and the oracle
    rp, ci = sgcgen.er(5000, 30000, 2)
    g = sgc.Graph(rp, ci)
    t = sgc.Template(sgcgen.spider_tree([2, 2, 1]))
    seeds = list(range(100, 113))
    want, mx = _oracle_maps(rp, ci, sgcgen.spider_tree([2, 2, 1]), seeds)
    for precision in ("fp64", "fp32"):
        batched = sgc.count(g, t, seeds, precision=precision).maps
        _check(batched, want, mx, precision)
        single = np.array([sgc.count(g, t, [s], precision=precision, batch=1).maps[0] for s in seeds[:4]])
        assert np.array_equal(single, batched[:4]) if precision == "fp64" else np.allclose(single, batched[:4],
                                                                                              rtol=FP32_RTOL)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_passes_with_different_spmm_forms(precision):
    # 11 colorings run as passes of 8 + 2 + 1; the SpMM form of a step can differ between
    # batch sizes (bucketed for narrow rows), so each pass must use its own index tables
    rp, ci = sgcgen.er(3000, 12000, 11)
    parent = sgcgen.pruefer_tree(7, 5)
    seeds = list(range(100, 111))
    want, mx = _oracle_maps(rp, ci, parent, seeds)
    _check(sgc.count(sgc.Graph(rp, ci), sgc.Template(parent), seeds, precision=precision).maps, want, mx, precision)


def test_every_root_gives_the_same_count():
    rp, ci = sgcgen.er(2000, 9000, 3)
    g = sgc.Graph(rp, ci)
    parent = sgcgen.pruefer_tree(7, 9)
    t = sgc.Template(parent)
    ref = sgc.count(g, t, [4, 5], precision="fp64").maps
    want, _ = _oracle_maps(rp, ci, parent, [4, 5])
    assert list(ref) == [float(w) for w in want]
    for root in range(7):
        assert np.array_equal(sgc.count(g, t, [4, 5], precision="fp64", root=root).maps, ref)


def test_special_cases():
    rp, ci = sgcgen.er(500, 1000, 5)
    g = sgc.Graph(rp, ci)
    # k = 1: every vertex, including isolated ones
    assert sgc.count(g, sgc.Template([-1]), [1, 2]).maps.tolist() == [500.0, 500.0]
    # no edges at all
    rp0 = np.zeros(11, dtype=np.int32)
    g0 = sgc.Graph(rp0, np.zeros(0, dtype=np.int32))
    assert sgc.count(g0, sgc.Template(sgcgen.path_tree(3)), [1]).maps.tolist() == [0.0]
    # n_iter = 0 (keep the template object alive while its handle is in use)
    t3 = sgc.Template(sgcgen.path_tree(3))
    est, maps = sgc.sgc_count(g.handle, t3.handle, [])
    assert est == 0.0 and len(maps) == 0


def test_complete_graph_closed_form_on_gpu():
    # colorful maps of any k-tree in K_n = k! * prod_c n_c
    import math
    nn = 40
    rp, ci = sgcgen.complete_graph(nn)
    g = sgc.Graph(rp, ci)
    for parent in (sgcgen.path_tree(6), sgcgen.pruefer_tree(7, 1)):
        k = len(parent)
        r = sgc.count(g, sgc.Template(parent), [11, 12], precision="fp64")
        for s, m in zip([11, 12], r.maps):
            counts = np.bincount(oracle.colors(s, nn, k), minlength=k)
            assert m == float(math.factorial(k) * int(np.prod(counts.astype(object))))


# path 0-1-2-3 as CSR, then one defect each
_GOOD_RP = [0, 1, 3, 5, 6]
_GOOD_CI = [1, 0, 2, 1, 3, 2]
_BAD_CSR = {
    "asymmetric": (_GOOD_RP, [2, 0, 2, 1, 3, 2]),
    "self_loop": (_GOOD_RP, [0, 0, 2, 1, 3, 2]),
    "unsorted": (_GOOD_RP, [1, 2, 0, 1, 3, 2]),
    "duplicate": ([0, 1, 3, 5, 6], [1, 0, 0, 1, 3, 2]),
    "col_range": (_GOOD_RP, [1, 0, 2, 1, 3, 4]),
    "row_ptr": ([0, 3, 1, 5, 6], _GOOD_CI),
    "nnz_mismatch": ([0, 1, 3, 5, 7], _GOOD_CI + [0]),
    # star 0-{1,2,3} plus directed entries 4->0 and 5->0: every mirror search succeeds, the
    # one-sided entries are only caught by the searched / skipped entry counts
    "asymmetric_one_sided": ([0, 3, 4, 5, 6, 7, 8], [1, 2, 3, 0, 0, 0, 0, 0]),
}


def test_good_csr_accepted():
    g = sgc.Graph(np.array(_GOOD_RP), np.array(_GOOD_CI))
    assert g.stats()["n_active"] == 4


@pytest.mark.parametrize("bad", list(_BAD_CSR))
def test_invalid_csr_rejected(bad):
    rp, ci = _BAD_CSR[bad]
    with pytest.raises(sgc.SgcError) as ei:
        sgc.Graph(np.array(rp, dtype=np.int32), np.array(ci, dtype=np.int32))
    assert ei.value.status == sgc.SGC_ERR_INVALID


def test_device_buffers_api():
    torch = pytest.importorskip("torch")
    rp, ci = sgcgen.er(4000, 20000, 6)
    d_rp = torch.from_numpy(rp).cuda()
    d_ci = torch.from_numpy(ci).cuda()
    g = sgc.Graph.from_device(len(rp) - 1, len(ci), d_rp.data_ptr(), d_ci.data_ptr())
    parent = sgcgen.spider_tree([2, 2, 1])
    t = sgc.Template(parent)
    seeds = torch.tensor([3, 4, 5], dtype=torch.int64).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    opt = sgc.sgc_options_init(precision=sgc.SGC_FP64, stream=stream.cuda_stream)
    sgc.sgc_count_device(g.handle, t.handle, seeds.data_ptr(), 3, opt, out.data_ptr())
    torch.cuda.synchronize()
    want, mx = _oracle_maps(rp, ci, parent, [3, 4, 5])
    _check(out.cpu().numpy(), want, mx, "fp64")


@pytest.mark.slow
def test_reduced_c3_rmat16_trees():
    # same templates and seeds as the scale-21 workload, on R-MAT scale 16 (a=.57, b=.19, c=.19)
    rp, ci = sgcgen.rmat(16, seed=1)
    g = sgc.Graph(rp, ci)
    cases = [sgcgen.path_tree(12), sgcgen.pruefer_tree(13, 7)]
    for parent in cases:
        seeds = [1, 2]
        want, mx = _oracle_maps(rp, ci, parent, seeds)
        _check(sgc.count(g, sgc.Template(parent), seeds, precision="fp32").maps, want, mx, "fp32")
        _check(sgc.count(g, sgc.Template(parent), seeds, precision="fp64").maps, want, mx, "fp64")
