"""The R-MAT scale-21 templates (12-vertex path, 13- and 15-vertex Pruefer trees with seeds 7 and 9,
k = |T|) at reduced scale against the exact oracle: R-MAT scale 16 with the same parameters and the
benchmark's coloring seeds 1..4.  The expected counts come from tests/golden/make_c3_golden.py
(the oracle only; the 15-vertex tree's counts pass 2^128 and were computed with 192-bit integers).

FP32 tables run as the benchmark runs them: 4 colorings per pass with autotuned launch shapes
(relative error <= 1e-5 per coloring).  FP64 tables with the planner's shapes are compared at
relative 1e-12: every count here is far above 2^53, where FP64 sums round (Section 7.4).
"""
import json
import os

import numpy as np
import pytest

import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "c3_rmat16.json")


@pytest.fixture(scope="module")
def c3():
    sgc.build()
    with open(GOLDEN) as f:
        gold = json.load(f)
    gp = gold["graph"]
    rp, ci = sgcgen.rmat(gp["scale"], edge_factor=gp["edge_factor"], a=gp["a"], b=gp["b"], c=gp["c"],
                         seed=gp["seed"])
    assert (len(rp) - 1, len(ci)) == (gp["n"], gp["nnz"])
    return gold, sgc.Graph(rp, ci)


def parent_of(spec):
    return sgcgen.path_tree(spec[1]) if spec[0] == "path" else sgcgen.pruefer_tree(spec[1], spec[2])


NAMES = ["path12", "pruefer13", "pruefer15"]


@pytest.mark.parametrize("name", NAMES)
def test_fp32_autotuned_matches_oracle(c3, name):
    gold, g = c3
    rec = gold["templates"][name]
    t = sgc.Template(parent_of(rec["spec"]))
    assert t.automorphisms == rec["aut"]
    seeds = np.array(gold["seeds"], dtype=np.uint64)
    want = np.array([float(int(r["maps"])) for r in rec["results"]])
    r = sgc.count(g, t, seeds, precision="fp32", batch=4, autotune=True)
    assert np.allclose(r.maps, want, rtol=1e-5, atol=0), (r.maps, want)
    # the tuned plan again (cached on the graph), with the estimate of Section 2.1
    r2 = sgc.count(g, t, seeds, precision="fp32", batch=4, autotune=True)
    assert np.allclose(r2.maps, want, rtol=1e-5, atol=0)
    k = rec["k"]
    scale = 1.0
    for i in range(1, k + 1):
        scale *= k / i
    assert r2.estimate == pytest.approx(float(np.mean(want)) / rec["aut"] * scale, rel=1e-5)


@pytest.mark.parametrize("name", NAMES)
def test_fp64_matches_oracle(c3, name):
    gold, g = c3
    rec = gold["templates"][name]
    t = sgc.Template(parent_of(rec["spec"]))
    seeds = np.array(gold["seeds"], dtype=np.uint64)
    want = np.array([float(int(r["maps"])) for r in rec["results"]])
    assert all(int(r["max_intermediate"]) >= 2 ** 53 for r in rec["results"])
    r = sgc.count(g, t, seeds, precision="fp64")
    assert np.allclose(r.maps, want, rtol=1e-12, atol=0), (r.maps, want)


@pytest.mark.parametrize("shape", [8, 15, 16, 17])
def test_wide_shapes_match_oracle(c3, shape):
    # the forms the autotuner chooses between on these templates' wide rows, each forced
    gold, g = c3
    for name in ("pruefer13", "pruefer15"):
        rec = gold["templates"][name]
        t = sgc.Template(parent_of(rec["spec"]))
        seeds = np.array(gold["seeds"][:2], dtype=np.uint64)
        want = np.array([float(int(r["maps"])) for r in rec["results"][:2]])
        r = sgc.count(g, t, seeds, precision="fp32", batch=2, spmm_shape=shape)
        assert np.allclose(r.maps, want, rtol=1e-5, atol=0), (name, shape, r.maps, want)


def test_scheduled_ema_matches_oracle(c3):
    # the scheduled eMA (bank-conflict-free rounds, rows staged by bulk copies; with up to 8 rows per
    # block, and with half as many so that two blocks share an SM) on the 13- and 15-vertex trees'
    # wide combines, one coloring per pass
    gold, g = c3
    for name in ("pruefer13", "pruefer15"):
        rec = gold["templates"][name]
        t = sgc.Template(parent_of(rec["spec"]))
        seeds = np.array(gold["seeds"][:2], dtype=np.uint64)
        want = np.array([float(int(r["maps"])) for r in rec["results"][:2]])
        for precision, tol in (("fp32", 1e-5), ("fp64", 1e-12)):
            for shape in (104, 105):
                r = sgc.count(g, t, seeds, precision=precision, batch=1, ema_rows=shape)
                assert np.allclose(r.maps, want, rtol=tol, atol=0), (name, precision, shape, r.maps, want)


@pytest.mark.parametrize("shape", [18, 19])
def test_staged_spmm_matches_oracle(c3, shape):
    # the grouped SpMM with neighbour rows copied into shared-memory rings (one coloring per pass) on
    # all three templates' SpMMs wider than 128 columns; narrower ones keep the planner's shapes
    gold, g = c3
    for name in NAMES:
        rec = gold["templates"][name]
        t = sgc.Template(parent_of(rec["spec"]))
        seeds = np.array(gold["seeds"][:2], dtype=np.uint64)
        want = np.array([float(int(r["maps"])) for r in rec["results"][:2]])
        r = sgc.count(g, t, seeds, precision="fp32", batch=1, spmm_shape=shape)
        assert np.allclose(r.maps, want, rtol=1e-5, atol=0), (name, shape, r.maps, want)
