"""The C-ABI library (no GPU needed): it builds for sm_103a, loads, exports
every symbol include/sgc.h declares, and its host-only template code agrees
with independent checks."""
import math
import os
import re

import numpy as np
import pytest

import paper_1903_04395_gb300 as sgc
import sgcgen
from tests import pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    sgc.build()
    return sgc.lib()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "sgc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgc_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("sgc_graph_create", "sgc_template_create", "sgc_count", "sgc_count_device",
                     "sgc_graph_destroy", "sgc_template_destroy", "sgc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    for name in _declared_functions():
        assert hasattr(built, name), name
    assert set(sgc.SIGNATURES) == set(_declared_functions())


def test_version_and_options(built):
    assert sgc.sgc_version() >= 100
    o = sgc.sgc_options_init()
    assert o.precision == sgc.SGC_FP32 and o.root == -1 and o.batch == 0


@pytest.mark.parametrize("parent", [sgcgen.path_tree(1), sgcgen.path_tree(2), sgcgen.path_tree(7), sgcgen.star_tree(6),
                                    sgcgen.spider_tree([3, 3, 3]), sgcgen.spider_tree([2, 2]),
                                    sgcgen.spider_tree([1, 2, 3])]
                         + [sgcgen.pruefer_tree(k, s) for k in (5, 6, 7, 8) for s in (1, 2, 3)])
def test_template_automorphisms_match_brute_force(built, parent):
    t = sgc.Template(parent)
    assert t.automorphisms == pins.aut_brute(parent)


def test_template_automorphisms_closed_forms(built):
    assert sgc.Template(sgcgen.spider_tree([3, 3, 3])).automorphisms == 6
    for k in range(3, 17):
        assert sgc.Template(sgcgen.path_tree(k)).automorphisms == 2
    for k in range(3, 13):
        assert sgc.Template(sgcgen.star_tree(k)).automorphisms == math.factorial(k - 1)


@pytest.mark.parametrize("parent,why", [
    ([-1, -1, 0], "two roots"),
    ([1, 2, 0], "no root"),
    ([-1, 0, 5], "parent out of range"),
    ([-1, 2, 1], "cycle"),
    ([-1, 1], "self parent"),
    ([], "empty"),
    (list(range(-1, 18)), "k above the maximum"),
])
def test_template_rejects_invalid(built, parent, why):
    with pytest.raises(sgc.SgcError) as ei:
        sgc.sgc_template_create(len(parent), np.array(parent if parent else [0], dtype=np.int32))
    assert ei.value.status == sgc.SGC_ERR_INVALID, why


def test_null_arguments_rejected(built):
    L = sgc.lib()
    assert L.sgc_count(None, None, None, 0, None, None, None) == sgc.SGC_ERR_INVALID
    assert L.sgc_graph_stats_get(None, None) == sgc.SGC_ERR_INVALID
    assert L.sgc_template_create(3, None, None) == sgc.SGC_ERR_INVALID
    sgc.sgc_graph_destroy(None)
    sgc.sgc_template_destroy(None)


def test_iterations_bound_is_the_lemma_count():
    # the lemma after Lemma 1 (Section 5.1): O(e^k log(1/delta) / eps^2) colorings, constant 1
    import math
    sgc.build()
    for k, eps, delta in [(5, 0.1, 0.05), (10, 0.05, 0.01), (1, 1.0, 0.5), (16, 0.2, 0.1), (18, 0.2, 0.1)]:
        want = math.ceil(math.exp(k) * math.log(1 / delta) / eps ** 2)
        got = sgc.sgc_iterations_bound(k, eps, delta)
        assert abs(got - want) <= 1, (k, eps, delta, got, want)
    for bad in [(0, 0.1, 0.1), (19, 0.1, 0.1), (5, 0.0, 0.1), (5, 0.1, 0.0), (5, 0.1, 1.0)]:
        assert sgc.sgc_iterations_bound(*bad) == -1


def test_binding_rejects_unknown_precision():
    # the binding maps only 'fp32' and 'fp64'; anything else is an error before any call
    with pytest.raises(ValueError):
        sgc._precision("fp16")
    assert sgc._precision("fp32") == sgc.SGC_FP32 and sgc._precision("fp64") == sgc.SGC_FP64


def test_estimate_from_maps_matches_the_oracle_estimator(built):
    # Section 2.1: mean of maps / |Aut(T)| / P(colorful), P = k!/k^k, or k!/((k-|T|)! k^|T|) with more colors
    import oracle
    rp, ci = sgcgen.er(60, 200, 9)
    for parent, colors in ((sgcgen.pruefer_tree(5, 2), 0), (sgcgen.spider_tree([2, 1]), 0), (sgcgen.path_tree(4), 6)):
        t = sgc.Template(parent)
        seeds = list(range(1, 9))
        ref = oracle.estimate(rp, ci, parent, seeds, ncolors=colors or None)
        got = sgc.sgc_estimate_from_maps(t.handle, np.array(ref.maps, dtype=np.float64), colors)
        assert got == pytest.approx(ref.mean, rel=1e-13)
    t = sgc.Template(sgcgen.path_tree(3))
    assert sgc.sgc_estimate_from_maps(t.handle, np.zeros(0)) == 0.0
    # 3-path, k = 3: P(colorful) = 3!/3^3 = 2/9, |Aut| = 2: 36 maps -> 36 / 2 * 9 / 2 = 81
    assert sgc.sgc_estimate_from_maps(t.handle, np.array([36.0])) == pytest.approx(81.0, rel=1e-15)
    with pytest.raises(sgc.SgcError):
        sgc.sgc_estimate_from_maps(t.handle, np.array([-1.0]))
    with pytest.raises(sgc.SgcError):
        sgc.sgc_estimate_from_maps(t.handle, np.array([1.0]), sgc.SGC_MAX_K + 1)


def test_templates_up_to_eighteen_vertices(built):
    # k <= 18: every relative color set (subsets of the other 17 colors) has a 16-bit index
    assert sgc.SGC_MAX_K == 18
    assert sgc.Template(sgcgen.path_tree(18)).automorphisms == 2
    assert sgc.Template(sgcgen.star_tree(18)).automorphisms == math.factorial(17)
    assert sgc.Template(sgcgen.pruefer_tree(17, 3)).automorphisms >= 1
    with pytest.raises(sgc.SgcError):
        sgc.Template(sgcgen.path_tree(19))
