"""The batched configuration at reduced scale against the exact oracle: an Erdos-Renyi graph of
average degree 24 and an R-MAT graph (a=.57 b=.19 c=.19), the six Pruefer trees of 5, 7, 8, 10, 11
and 12 vertices (seeds 1000 + size), 7 colorings each - passes of 4, 2 and 1 - counted by one
sgc_count_many call recorded as one CUDA graph, with autotuned launch shapes.  FP32 maps within
1e-5 of the oracle per coloring; a replay with new seeds too."""
import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu

SIZES = (5, 7, 8, 10, 11, 12)


def graphs():
    yield "er", sgcgen.er(5000, 60000, seed=1)
    yield "rmat", sgcgen.rmat(12, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1)


@pytest.mark.parametrize("name,graph", list(graphs()))
def test_batched_reduced_matches_oracle(name, graph):
    sgc.build()
    rp, ci = graph
    n = len(rp) - 1
    g = sgc.Graph(rp, ci)
    parents = [sgcgen.pruefer_tree(k, 1000 + k) for k in SIZES]
    ts = [sgc.Template(p) for p in parents]
    n_iter = 7
    for call in range(2):
        seeds = (np.arange(len(ts) * n_iter, dtype=np.uint64).reshape(len(ts), n_iter)
                 + np.uint64(1 + 100 * call))
        k0 = g.stats()["kernel_launches"]
        est, maps = sgc.count_many(g, ts, seeds, precision="fp32", batch=4, use_graph=True, autotune=True)
        assert g.stats()["kernel_launches"] > k0
        for j, p in enumerate(parents):
            want = np.array([float(oracle.count(rp, ci, p, oracle.colors(int(s), n, len(p))).maps)
                             for s in seeds[j]])
            assert np.allclose(maps[j], want, rtol=1e-5, atol=0), (name, len(p), maps[j], want)
