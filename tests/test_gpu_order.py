"""Row numbering (Section 4.3's locality pre-processing): the reverse Cuthill-McKee
order of SGC_GRAPH_ORDER_RCM changes only which row a vertex lands in.  Colors are
drawn from the original ids, so every coloring's count is the same as under the
default degree order and as the oracle's: FP64 bit-exact (while below 2^53), FP32
within the parity tolerance (neighbour lists are summed in another order)."""
import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    sgc.build()


def _oracle(rp, ci, parent, seeds):
    res = [oracle.count(rp, ci, parent, oracle.colors(int(s), len(rp) - 1, len(parent))) for s in seeds]
    return np.array([float(r.maps) for r in res]), max(r.max_intermediate for r in res)


GRAPHS = {
    # hubs split into segments (rows > 256) plus many light rows and isolated vertices
    "rmat13": lambda: sgcgen.rmat(13, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=3),
    # no heavy row at all: the whole graph in RCM order, several components
    "er": lambda: sgcgen.er(3000, 6000, 17),
    # a path: the RCM order is a path order
    "path": lambda: _path_graph(500),
}


def _path_graph(n):
    rows = [[v - 1] if v > 0 else [] for v in range(n)]
    for v in range(n - 1):
        rows[v].append(v + 1)
    rp = np.zeros(n + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([u for r in rows for u in sorted(r)], dtype=np.int32)
    return rp, ci


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rcm_order_counts_match_degree_order_and_oracle(name, precision):
    rp, ci = GRAPHS[name]()
    g0 = sgc.Graph(rp, ci)
    g1 = sgc.Graph(rp, ci, rcm=True)
    s0, s1 = g0.stats(), g1.stats()
    assert s0["ordering"] == 0 and s1["ordering"] == 1
    for key in ("n_active", "nnz", "max_degree", "n_heavy", "n_segments"):
        assert s0[key] == s1[key], key
    seeds = np.arange(7, 17, dtype=np.uint64)
    for parent in (sgcgen.spider_tree([2, 2, 2]), sgcgen.pruefer_tree(8, 1008), sgcgen.path_tree(5)):
        t = sgc.Template(parent)
        want, mx = _oracle(rp, ci, parent, seeds)
        a = sgc.count(g0, t, seeds, precision=precision).maps
        b = sgc.count(g1, t, seeds, precision=precision).maps
        if precision == "fp64" and mx < 2 ** 53:
            assert np.array_equal(a, want) and np.array_equal(b, want)
        else:
            nz = want > 0
            assert np.all(b[~nz] == 0)
            assert np.all(np.abs(b[nz] - want[nz]) <= FP32_RTOL * want[nz]), (b, want)


def test_rcm_order_from_device_csr():
    torch = pytest.importorskip("torch")
    rp, ci = sgcgen.rmat(12, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=9)
    d_rp = torch.from_numpy(rp).cuda()
    d_ci = torch.from_numpy(ci).cuda()
    torch.cuda.synchronize()
    g = sgc.Graph.from_device(len(rp) - 1, len(ci), d_rp.data_ptr(), d_ci.data_ptr(), rcm=True)
    assert g.stats()["ordering"] == 1
    parent = sgcgen.spider_tree([3, 3])
    seeds = np.arange(3, 11, dtype=np.uint64)
    want, mx = _oracle(rp, ci, parent, seeds)
    assert mx < 2 ** 53
    got = sgc.count(g, sgc.Template(parent), seeds, precision="fp64").maps
    assert np.array_equal(got, want)


def test_rcm_order_rejects_bad_columns_like_the_degree_order():
    # an out-of-range column is skipped by the host-side ordering and reported by the relabelling
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([1, 7], dtype=np.int32)
    with pytest.raises(sgc.SgcError):
        sgc.Graph(rp, ci, validate=False, rcm=True)
