"""Host-side helpers of bench.py: the traffic record is matched to a kernel by the hash of its
definition (no GPU)."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_kernel_source_sha_finds_each_recorded_function():
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for r in rec["kernels"]:
        sha = b.kernel_source_sha(r["function"])
        assert sha is not None and len(sha) == 16
    assert b.kernel_source_sha("no_such_kernel_anywhere") is None


def test_recorded_traffic_follows_the_function_hash(monkeypatch):
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    r = rec["kernels"][0]
    # with the recorded hash the record is used; with any other hash it reads as unmeasured
    monkeypatch.setattr(b, "kernel_source_sha", lambda fn: r["function_sha"])
    assert b.recorded_traffic(r["op"], r["k"], r["batch"], r["shape"]) == r["dram_bytes_per_launch"]
    # another number of colors, colorings per pass or launch shape is another launch
    assert b.recorded_traffic(r["op"], r["k"] + 1, r["batch"], r["shape"]) is None
    assert b.recorded_traffic(r["op"], r["k"], r["batch"] * 2, r["shape"]) is None
    assert b.recorded_traffic(r["op"], r["k"], r["batch"], r["shape"] + 1) is None
    assert b.recorded_traffic(r["op"], r["k"], r["batch"], None) is None
    monkeypatch.setattr(b, "kernel_source_sha", lambda fn: "0" * 16)
    assert b.recorded_traffic(r["op"], r["k"], r["batch"], r["shape"]) is None
    assert b.recorded_traffic("no such op", r["k"], r["batch"], r["shape"]) is None


def test_survey_bytes_formulas():
    # the survey's algorithmic bytes: SpMM 4(n+1+nnz) + 2 b n C(k,p) per coloring, eMA b n (C_a+C_p+C_t)
    import math
    b = _bench()
    n, nnz = 1000, 5000
    assert b.survey_bytes({"kind": "spmm", "t": 0, "a": 0, "p": 3}, n, nnz, 10, 4, 2) == \
        4 * (n + 1 + nnz) + 2 * 2 * 4 * n * math.comb(10, 3)
    assert b.survey_bytes({"kind": "ema", "t": 6, "a": 3, "p": 3}, n, nnz, 10, 4, 1) == \
        4 * n * (math.comb(10, 3) + math.comb(10, 3) + math.comb(10, 6))
    assert b.survey_bytes({"kind": "final", "t": 10, "a": 7, "p": 3}, n, nnz, 10, 4, 1) == \
        4 * n * (math.comb(10, 7) + math.comb(10, 3))
