"""Several templates in one call, the recorded launch sequence and the launch shapes.

* sgc_count_many (templates counted side by side on several streams, one CUDA
  graph launch) returns, per template, what sgc_count returns alone - and the
  exact oracle's colorful maps (FP64 exactly, FP32 within 1e-5).
* A recorded launch sequence replays with new seeds (the seeds are staged, not
  baked into the recording).
* Every forced SpMM and eMA launch shape gives the oracle's counts; the
  autotuner's report is well formed and its tuned plan counts the same.
The shapes only reschedule the sums of Eq. 2 and of the eMA (Section 4.5).
"""
import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5


@pytest.fixture(scope="module")
def er_graph():
    sgc.build()
    rp, ci = sgcgen.er(3000, 15000, 21)
    return rp, ci, sgc.Graph(rp, ci)


def parents():
    return [sgcgen.path_tree(3), sgcgen.pruefer_tree(5, 1005), sgcgen.pruefer_tree(7, 1007),
            sgcgen.spider_tree([2, 2, 1]), sgcgen.star_tree(6), np.array([-1], dtype=np.int32)]


class Exact(np.ndarray):
    """Oracle maps, remembering whether every intermediate count stayed below 2^53."""


def oracle_maps(rp, ci, parent, seeds):
    n = len(rp) - 1
    res = [oracle.count(rp, ci, parent, oracle.colors(int(s), n, len(parent))) for s in seeds]
    out = np.array([r.maps for r in res], dtype=np.float64).view(Exact)
    out.exact = all(r.max_intermediate < 2 ** 53 for r in res)
    return out


def check(got, want, precision):
    if precision == "fp64":
        if getattr(want, "exact", True):
            assert np.array_equal(got, np.asarray(want)), (got, want)
        else:  # FP64 rounding once counts pass 2^53
            assert np.allclose(got, np.asarray(want), rtol=1e-12, atol=0), (got, want)
    else:
        assert np.allclose(got, np.asarray(want), rtol=FP32_RTOL, atol=0), (got, want)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_many_matches_single_and_oracle(er_graph, precision, use_graph):
    rp, ci, g = er_graph
    ps = parents()
    ts = [sgc.Template(p) for p in ps]
    n_iter = 11  # passes of 8 + 2 + 1 colorings
    seeds = np.arange(len(ts) * n_iter, dtype=np.uint64).reshape(len(ts), n_iter) * 7 + 3
    est, maps = sgc.count_many(g, ts, seeds, precision=precision, use_graph=use_graph)
    assert maps.shape == (len(ts), n_iter)
    for j, (p, t) in enumerate(zip(ps, ts)):
        single = sgc.count(g, t, seeds[j], precision=precision, use_graph=False)
        if precision == "fp64":
            assert np.array_equal(maps[j], single.maps), (j, maps[j], single.maps)
            assert est[j] == pytest.approx(single.estimate, rel=1e-15)
        else:
            assert np.allclose(maps[j], single.maps, rtol=1e-6, atol=0)
        check(maps[j], oracle_maps(rp, ci, p, seeds[j]), precision)


def test_recorded_sequence_replays_with_new_seeds(er_graph):
    rp, ci, g = er_graph
    ps = parents()[1:4]
    ts = [sgc.Template(p) for p in ps]
    n_iter = 5
    launches = []
    for call in range(3):
        seeds = np.arange(len(ts) * n_iter, dtype=np.uint64).reshape(len(ts), n_iter) + 1000 * (call + 1)
        k0 = g.stats()["kernel_launches"]
        _, maps = sgc.count_many(g, ts, seeds, precision="fp64", use_graph=True)
        launches.append(g.stats()["kernel_launches"] - k0)
        for j, p in enumerate(ps):
            check(maps[j], oracle_maps(rp, ci, p, seeds[j]), "fp64")
    # the replays launch the same recorded kernels
    assert launches[0] > 0 and launches[0] == launches[1] == launches[2]


@pytest.mark.parametrize("spmm_shape", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_spmm_shape(precision, spmm_shape):
    sgc.build()
    rp, ci = sgcgen.rmat(13, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=3)
    g = sgc.Graph(rp, ci)
    assert g.stats()["n_heavy"] > 0  # rows split into segments are covered
    # register buckets take one coloring per pass, the grouped form at most 4 (passes of 4, 4, 2, 1)
    batch = 1 if spmm_shape == 4 else 4 if spmm_shape in (16, 17) else 0
    for parent in (sgcgen.pruefer_tree(8, 1008), sgcgen.spider_tree([3, 3, 3]), sgcgen.pruefer_tree(13, 7)):
        t = sgc.Template(parent)
        seeds = np.arange(1, 12 if len(parent) < 13 else 3, dtype=np.uint64)  # 8 + 2 + 1
        r = sgc.count(g, t, seeds, precision=precision, spmm_shape=spmm_shape, batch=batch)
        check(r.maps, oracle_maps(rp, ci, parent, seeds), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("batch", [1, 2, 4])
def test_grouped_spmm(batch, precision):
    # neighbours grouped by color, each color's rows summed in registers and scattered once: the
    # oracle's counts (FP64 exactly while below 2^53), equal FP64 maps to the direct form, narrow
    # and wide rows (the 13-vertex tree) and heavy-row segments
    sgc.build()
    rp, ci = sgcgen.rmat(13, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=6)
    g = sgc.Graph(rp, ci)
    assert g.stats()["n_heavy"] > 0
    for parent in (sgcgen.spider_tree([3, 3, 3]), sgcgen.pruefer_tree(13, 7), sgcgen.path_tree(6)):
        t = sgc.Template(parent)
        seeds = np.arange(90, 90 + 2 * batch + 1, dtype=np.uint64)  # passes of batch, batch, 1
        a = sgc.count(g, t, seeds, precision=precision, spmm_shape=16, batch=batch)
        a8 = sgc.count(g, t, seeds, precision=precision, spmm_shape=17, batch=batch)
        # the same terms; a position's color groups may come in another order across chunk borders
        assert np.allclose(a.maps, a8.maps, rtol=1e-12 if precision == "fp64" else 1e-6, atol=0)
        if precision == "fp64":
            b = sgc.count(g, t, seeds, precision=precision, spmm_shape=8, batch=batch)
            assert np.array_equal(a.maps, b.maps) or np.allclose(a.maps, b.maps, rtol=1e-12, atol=0)
        few = seeds[: (len(seeds) if len(parent) < 13 else 1)]
        check(a.maps[: len(few)], oracle_maps(rp, ci, parent, few), precision)


def test_staged_spmm_sums_in_the_same_order():
    # neighbour rows and output positions copied into shared-memory rings by asynchronous copies:
    # the ring's depth (shape 18: 3 chunks, 19: 2) does not change the sums, so their FP32 maps are
    # equal bit for bit; against the register form (512-column chunks) rows of up to 512 columns sum
    # in the same order and 1,024-column chunks group a position's terms differently.  Rows of 165
    # to 2,002 columns (one or two chunks), heavy-row segments, rows whose neighbours all share
    # their color, the oracle.
    sgc.build()
    rp, ci = sgcgen.rmat(13, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=6)
    g = sgc.Graph(rp, ci)
    assert g.stats()["n_heavy"] > 0
    for parent in (sgcgen.path_tree(12), sgcgen.pruefer_tree(13, 7), sgcgen.pruefer_tree(15, 9)):
        t = sgc.Template(parent)
        seeds = np.arange(40, 43, dtype=np.uint64)
        a = sgc.count(g, t, seeds, precision="fp32", spmm_shape=16, batch=1)
        b = sgc.count(g, t, seeds, precision="fp32", spmm_shape=19, batch=1)
        c = sgc.count(g, t, seeds, precision="fp32", spmm_shape=18, batch=1)
        assert np.array_equal(b.maps, c.maps)
        assert np.allclose(a.maps, c.maps, rtol=1e-6, atol=0)
        if len(parent) <= 13:
            check(c.maps[:1], oracle_maps(rp, ci, parent, seeds[:1]), "fp32")


@pytest.mark.parametrize("batch", [1, 4, 8, 32])
def test_wide_spmm_sums_in_the_same_order(batch):
    # 16-bit positions in chunks of eight: FP32 maps equal the batch-specialised direct form's bit
    # for bit, for narrow and wide rows (the 13-vertex tree's passive tables), heavy segments too
    sgc.build()
    rp, ci = sgcgen.rmat(13, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=6)
    g = sgc.Graph(rp, ci)
    assert g.stats()["n_heavy"] > 0
    for parent in (sgcgen.spider_tree([3, 3, 3]), sgcgen.pruefer_tree(13, 7)):
        t = sgc.Template(parent)
        seeds = np.arange(70, 70 + batch, dtype=np.uint64)
        a = sgc.count(g, t, seeds, precision="fp32", spmm_shape=8, batch=batch)
        b = sgc.count(g, t, seeds, precision="fp32", spmm_shape=15, batch=batch)
        assert np.array_equal(a.maps, b.maps)
        # the oracle on a few colorings (the 13-vertex tree is slow on the host)
        few = seeds[: (8 if len(parent) < 13 else 1)]
        check(b.maps[: len(few)], oracle_maps(rp, ci, parent, few), "fp32")


@pytest.mark.parametrize("batch", [4, 8, 16])
def test_unrolled_spmm_sums_in_the_same_order(batch):
    # the unrolled direct form reads its positions differently but adds the same terms in the
    # same order: FP32 maps equal the batch-specialised direct form's bit for bit (heavy-row
    # segments included)
    sgc.build()
    rp, ci = sgcgen.rmat(14, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=6)
    g = sgc.Graph(rp, ci)
    assert g.stats()["n_heavy"] > 0
    for parent in (sgcgen.spider_tree([3, 3, 3]), sgcgen.pruefer_tree(9, 1009), sgcgen.path_tree(6)):
        t = sgc.Template(parent)
        seeds = np.arange(40, 40 + 2 * batch, dtype=np.uint64)
        a = sgc.count(g, t, seeds, precision="fp32", spmm_shape=8, batch=batch)
        b = sgc.count(g, t, seeds, precision="fp32", spmm_shape=14, batch=batch)
        assert np.array_equal(a.maps, b.maps)
        check(b.maps, oracle_maps(rp, ci, parent, seeds), "fp32")


@pytest.mark.parametrize("ema_rows", [64, 32, 16, 8, 4, 2, 1, 101, 102, 103, 104, 105])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_ema_shape(ema_rows, precision):
    sgc.build()
    rp, ci = sgcgen.rmat(12, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=4)
    g = sgc.Graph(rp, ci)
    # the spider's eMA is symmetric (a table with itself), the others are not;
    # vertex tiles need 4..32 colorings per pass: 16 + 8 + 1 exercises both kernels;
    # the scheduled forms (104, 105: half the rows, two blocks per SM) take one coloring per pass,
    # tiles of up to 8 rows with a ragged last one
    batch = 1 if ema_rows in (104, 105) else 16
    for parent in (sgcgen.pruefer_tree(9, 1009), sgcgen.path_tree(8), sgcgen.spider_tree([3, 3, 3]),
                   sgcgen.pruefer_tree(13, 7)):
        t = sgc.Template(parent)
        seeds = np.arange(20, 45 if len(parent) < 13 else 22, dtype=np.uint64)
        r = sgc.count(g, t, seeds, precision=precision, ema_rows=ema_rows, batch=batch)
        check(r.maps, oracle_maps(rp, ci, parent, seeds), precision)


def _two_branch_parent():
    # DP root 0 with two 3-vertex branches, a path 1-2-3 and a cherry 4-(5, 6): whichever is cut
    # first, the 7-vertex table combines the P of one branch with the P of the other, a
    # non-symmetric (a = 4, p = 3) eMA
    return np.array([-1, 0, 1, 2, 0, 4, 4], dtype=np.int32)


@pytest.mark.parametrize("case", ["spider-symmetric", "two-branch-10-colors"])
def test_register_ema_sums_like_the_vertex_tiles(case, monkeypatch):
    # the register form adds each output's terms in the split table's order: FP32 maps equal
    # the vertex-tile kernel's bit for bit, and the oracle's within the tolerance (the spider's
    # combine is kept apart from the last step here, as with the vertex tiles)
    monkeypatch.setenv("SGC_NO_FUSE", "1")
    sgc.build()
    rp, ci = sgcgen.rmat(13, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=8)
    g = sgc.Graph(rp, ci)
    if case == "spider-symmetric":
        parent, colors, root = sgcgen.spider_tree([3, 3, 3]), 0, -1
    else:
        parent, colors, root = _two_branch_parent(), 10, 0
    t = sgc.Template(parent)
    opt = sgc.sgc_options_init(precision=sgc.SGC_FP32, batch=8, colors=colors, root=root)
    rep = sgc.sgc_autotune(g.handle, t.handle, opt)
    emas = [e for e in rep[:-1] if e["name"] == "ema" and 103 in e["shapes"]]
    assert any(e["t"] == 7 and e["a"] == 4 and e["p"] == 3 for e in emas), rep
    seeds = np.arange(60, 76, dtype=np.uint64)
    a = sgc.count(g, t, seeds, precision="fp32", batch=8, ema_rows=101, colors=colors, root=root)
    b = sgc.count(g, t, seeds, precision="fp32", batch=8, ema_rows=103, colors=colors, root=root)
    assert np.array_equal(a.maps, b.maps)
    ref = oracle.estimate(rp, ci, parent, [int(s) for s in seeds], ncolors=colors or len(parent))
    assert np.allclose(b.maps, np.array(ref.maps, dtype=np.float64), rtol=FP32_RTOL, atol=0)


def test_fused_combine_and_last_step(monkeypatch):
    # the spider's symmetric register-form combine fused with the last step: every row's term is
    # the unfused path's, bit for bit; the rows' FP64 sums run over another grid, so the maps
    # agree to FP64 rounding, and with the oracle within the FP32 tolerance
    sgc.build()
    rp, ci = sgcgen.rmat(13, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=13)
    parent = sgcgen.spider_tree([3, 3, 3])
    for batch, seeds in ((8, np.arange(200, 216, dtype=np.uint64)), (4, np.arange(300, 305, dtype=np.uint64)),
                         (16, np.arange(400, 416, dtype=np.uint64)), (32, np.arange(500, 532, dtype=np.uint64))):
        fused = sgc.count(sgc.Graph(rp, ci), sgc.Template(parent), seeds, precision="fp32", batch=batch)
        monkeypatch.setenv("SGC_NO_FUSE", "1")
        apart = sgc.count(sgc.Graph(rp, ci), sgc.Template(parent), seeds, precision="fp32", batch=batch)
        monkeypatch.delenv("SGC_NO_FUSE")
        assert np.allclose(fused.maps, apart.maps, rtol=1e-12, atol=0), (fused.maps, apart.maps)
        check(fused.maps, oracle_maps(rp, ci, parent, seeds), "fp32")


FINAL_SHAPE_TREES = {  # template -> the last step's (K, p) on R-MAT 13 (seed 12) with the planner's root
    "spider10": (sgcgen.spider_tree([3, 3, 3]), (9, 3)),
    "pruefer7": (sgcgen.pruefer_tree(7, 1007), (6, 1)),
    "pruefer8": (sgcgen.pruefer_tree(8, 1008), (7, 3)),
    "pruefer9": (sgcgen.pruefer_tree(9, 1009), (8, 4)),
    "pruefer11": (sgcgen.pruefer_tree(11, 1011), (10, 2)),
    "pruefer15": (sgcgen.pruefer_tree(15, 9), (14, 1)),
}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(FINAL_SHAPE_TREES))
def test_final_compile_time_form_matches_table_form(monkeypatch, precision, name):
    # the last step with compile-time complement indices sums every row in the table-driven
    # kernel's order: identical maps in either precision, for each (K, p) shape compiled in
    sgc.build()
    rp, ci = sgcgen.rmat(13, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=12)
    parent, _ = FINAL_SHAPE_TREES[name]
    seeds = np.arange(90, 101 if len(parent) < 12 else 92, dtype=np.uint64)
    monkeypatch.setenv("SGC_NO_FUSE", "1")  # the last step as its own kernel
    got = sgc.count(sgc.Graph(rp, ci), sgc.Template(parent), seeds, precision=precision)
    monkeypatch.setenv("SGC_FINAL_TABLE", "1")
    tab = sgc.count(sgc.Graph(rp, ci), sgc.Template(parent), seeds, precision=precision)
    assert np.array_equal(got.maps, tab.maps)
    check(got.maps, oracle_maps(rp, ci, parent, seeds), precision)


def test_autotune_report_and_tuned_counts():
    sgc.build()
    rp, ci = sgcgen.rmat(13, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=5)
    g = sgc.Graph(rp, ci)
    parent = sgcgen.pruefer_tree(8, 1008)
    t = sgc.Template(parent)
    opt = sgc.sgc_options_init(precision=sgc.SGC_FP64, batch=8)
    rep = sgc.sgc_autotune(g.handle, t.handle, opt)
    assert rep and rep[-1]["kind"] == -1
    assert rep[-1]["shapes"][rep[-1]["chosen"]] in (8, 4)
    for e in rep[:-1]:
        assert e["kind"] in (2, 4)
        assert len(e["shapes"]) >= 2 and 0 <= e["chosen"] < len(e["shapes"])
        assert all(ms > 0 for ms in e["ms"])
    # a second call reads the cached report
    assert sgc.sgc_autotune(g.handle, t.handle, opt) == rep
    seeds = np.arange(1, 12, dtype=np.uint64)
    tuned = sgc.count(g, t, seeds, precision="fp64", batch=8, autotune=True)
    check(tuned.maps, oracle_maps(rp, ci, parent, seeds), "fp64")


def test_fused_combine_takes_no_table_workspace(monkeypatch):
    # the 10-vertex spider's last combine runs fused with the last step: its 7-vertex table is never
    # stored, so it takes no workspace and no HBM bytes (the same counts either way)
    sgc.build()
    rp, ci = sgcgen.rmat(12, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1)
    parent = sgcgen.spider_tree([3, 3, 3])
    fused = sgc.plan(sgc.Graph(rp, ci), sgc.Template(parent), batch=8)
    seeds = np.arange(1, 9, dtype=np.uint64)
    a = sgc.count(sgc.Graph(rp, ci), sgc.Template(parent), seeds, batch=8)
    monkeypatch.setenv("SGC_NO_FUSE", "1")
    g2 = sgc.Graph(rp, ci)
    apart = sgc.plan(g2, sgc.Template(parent), batch=8)
    b = sgc.count(g2, sgc.Template(parent), seeds, batch=8)
    assert fused["workspace_bytes"] < apart["workspace_bytes"], (fused, apart)
    assert fused["est_bytes"] < apart["est_bytes"]
    assert np.allclose(a.maps, b.maps, rtol=1e-5, atol=0)


@pytest.mark.parametrize("batch", [8, 16, 32])
def test_register_ema_shapes_of_the_batched_trees(batch):
    # the register-form combines compiled in for the 7-, 8- and 11-vertex Pruefer trees (seeds 1007,
    # 1008, 1011): the vertex tiles' sums (FP32 rounding apart) and the oracle's counts
    sgc.build()
    rp, ci = sgcgen.rmat(12, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=5)
    g = sgc.Graph(rp, ci)
    for k in (7, 8, 11):
        parent = sgcgen.pruefer_tree(k, 1000 + k)
        t = sgc.Template(parent)
        seeds = np.arange(200, 200 + batch, dtype=np.uint64)
        a = sgc.count(g, t, seeds, precision="fp32", batch=batch, ema_rows=103)
        b = sgc.count(g, t, seeds, precision="fp32", batch=batch, ema_rows=101)
        assert np.allclose(a.maps, b.maps, rtol=1e-6, atol=0), (k, a.maps, b.maps)
        check(a.maps[:4], oracle_maps(rp, ci, parent, seeds[:4]), "fp32")
