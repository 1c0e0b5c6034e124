"""Benchmark: color-coding tree counting on GB300.

Default workload: R-MAT scale 21 (2^21 vertices, edge factor 16,
a=0.57 b=0.19 c=0.19 d=0.05, seed 1, duplicates and self-loops removed;
63.5 M stored entries) with three templates - the 12-vertex path and the 13-
and 15-vertex Pruefer trees (seeds 7 and 9) - k = |T| colors, FP32 count
tables with FP64 final reduction.  One step counts 4 colorings of each
template (12 colorings).  `--workload rmat20-spider10` runs the 10-vertex
spider on R-MAT scale 20 (8 colorings per step, FP64 tables timed beside it);
`batched`, `serving` and `ablation` run the other configurations.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sgc|reference]

Under torchrun (N > 1) every rank counts its own colorings on its own GPU
(colorings are independent: weak scaling, no data-path collective); the
timed region is bracketed by barriers and the max over ranks is taken.
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "colorings/sec and SpMM+eMA HBM GB/s (vs ~8 TB/s) per template; p50/p99 query latency"
WORKLOADS = {
    "rmat20-spider10": dict(scale=20, templates=[("spider10", ("spider", [3, 3, 3]))], batch=8,
                            cpu_scale=20, cpu_scale_1t=16, ref_scale=20,
                            desc="R-MAT scale 20 (edge factor 16, a=.57 b=.19 c=.19, seed 1), 10-vertex spider "
                                 "(legs 3,3,3), k=10, 8 colorings per step"),
    "serving": dict(scale=21, templates=[("pruefer3..14", ("pruefer", 8, 1))], batch=1, fp64=False,
                    desc="R-MAT scale 21 resident; Poisson stream (200 queries/s) of Pruefer trees with 3..14 "
                         "vertices and 1..32 colorings per query; admission under a 120 GB budget"),
    "batched": dict(scale=20, templates=[(f"pruefer{k}", ("pruefer", k, 1000 + k)) for k in (5, 7, 8, 10, 11, 12)],
                    batch=256, fp64=False, steps=1, warmup=3,
                    desc="Erdos-Renyi G(n=500,000, m=6,000,000; seed 1) and R-MAT scale 20; Pruefer trees of "
                         "5, 7, 8, 10, 11, 12 vertices (seeds 1000+size), 256 colorings each, all templates of a "
                         "graph in one sgc_count_many call = one CUDA-graph launch; autotuned launch shapes"),
    "ablation": dict(scale=16, templates=[("spider10", ("spider", [3, 3, 3])), ("pruefer8", ("pruefer", 8, 1008))],
                     batch=8, fp64=False, steps=3, warmup=3,
                     desc="the paper's three variants on the same colorings: SpMM + eMA (PGBSC), pruned neighbour "
                          "sums one column at a time (PFASCIA), Algorithm 1's loop order (FASCIA), R-MAT scale 16"),
    "rmat21-trees": dict(scale=21, templates=[("path12", ("path", 12)), ("pruefer13", ("pruefer", 13, 7)),
                                              ("pruefer15", ("pruefer", 15, 9))], batch=4, fp64=False,
                         steps=8, warmup=3, cpu_scale=14, cpu_scale_1t=11, ref_scale=13,
                         desc="R-MAT scale 21 (edge factor 16, a=.57 b=.19 c=.19, seed 1); 12-vertex path, "
                              "13- and 15-vertex Pruefer trees (seeds 7, 9), k = |T|, 4 colorings per step each"),
}


WORKLOAD_SCALE = {name: wl["scale"] for name, wl in WORKLOADS.items()}
WORKLOAD_TEMPLATES = {name: [n for n, _ in wl["templates"]] for name, wl in WORKLOADS.items()}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 30; batched workload 1)")
    ap.add_argument("--warmup", type=int, default=None, help="warm-up steps (default 5; batched workload 3)")
    ap.add_argument("--impl", choices=["sgc", "reference"], default="sgc")
    ap.add_argument("--workload", default="rmat21-trees", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--queries", type=int, default=32, help="serving workload: queries in the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serving workload: offered queries per second")
    ap.add_argument("--sweep", default="", help="serving workload: comma-separated offered rates to sweep")
    ap.add_argument("--sweep-queries", type=int, default=64, help="serving workload: queries per swept rate")
    ap.add_argument("--no-autotune", action="store_true", help="planner launch shapes instead of the autotuner's")
    ap.add_argument("--scale", type=int, default=None,
                    help="R-MAT scale override (small cases for profiling; not a bench configuration)")
    ap.add_argument("--batch", type=int, default=None, help="colorings per pass override")
    ap.add_argument("--spmm-shape", type=int, default=0, help="force an SpMM launch shape (sgc_options.spmm_shape)")
    ap.add_argument("--ema-rows", type=int, default=0, help="force an eMA launch shape (sgc_options.ema_rows)")
    ap.add_argument("--root", type=int, default=-1,
                    help="force the DP root (sgc_options.root; profiling a small graph with a large one's plan)")
    ap.add_argument("--template", action="append", default=None,
                    help="only these templates of the workload (profiling small cases; not a bench configuration)")
    ap.add_argument("--rcm", action="store_true",
                    help="number the graph's rows in reverse Cuthill-McKee order (SGC_GRAPH_ORDER_RCM)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.scale is not None:
        wl["scale"] = args.scale
    if args.batch is not None:
        wl["batch"] = args.batch
    if args.template:
        wl["templates"] = [(n, sp) for n, sp in wl["templates"] if n in args.template]
        if not wl["templates"]:
            ap.error("--template names none of the workload's templates")
    if args.steps is None:
        args.steps = wl.get("steps", 30)
    if args.warmup is None:
        args.warmup = wl.get("warmup", 5)
    return args


def make_graph(wl):
    import sgcgen
    return sgcgen.rmat(wl["scale"], edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1)


def make_parent(spec):
    import sgcgen
    if spec[0] == "spider":
        return sgcgen.spider_tree(spec[1])
    if spec[0] == "path":
        return sgcgen.path_tree(spec[1])
    return sgcgen.pruefer_tree(spec[1], spec[2])


def make_template(wl):
    """The workload's first template (the one the CPU baseline times)."""
    return make_parent(wl["templates"][0][1])


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_sha(function: str):
    """Hash of one kernel's definition in kernels.cu: from the template line above
    `__global__ ... <function>(` to the closing brace at the start of a line."""
    with open(os.path.join(ROOT, "paper_1903_04395_gb300", "csrc", "kernels.cu")) as f:
        src = f.read()
    m = re.search(r"\n(template <[^\n]*>\n__global__ void[^\n]*\b" + re.escape(function) + r"\()", src)
    if not m:
        return None
    end = src.find("\n}\n", m.start(1))
    if end < 0:
        return None
    return hashlib.sha256(src[m.start(1):end + 3].encode()).hexdigest()[:16]


def recorded_traffic(op_name: str, k: int, batch: int, shape=None):
    """DRAM bytes per launch of an op from the committed ncu summary (profiles/traffic.json), if they were
    taken on the kernel's current source (the record keeps a hash of the kernel function's definition) for
    the same op, number of colors, colorings per pass and launch shape (None: the shape is unknown, and no
    record applies)."""
    if shape is None:
        return None
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    for r in rec.get("kernels", []):
        if r.get("op") == op_name and r.get("k") == k and r.get("batch") == batch and r.get("shape") == shape and \
                r.get("function") and \
                r.get("function_sha") == kernel_source_sha(r["function"]):
            return r.get("dram_bytes_per_launch")
    return None


def templ_k_of(e, templates):
    """Colors k of the template a profiled op belongs to (the op's own k when the library reports it)."""
    if e.get("k"):
        return int(e["k"])
    return max(len(t.parent) for _, t in templates) if templates else 0


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_rate(wl, full_n, full_nnz, scale, threads=None, seed=1):
    """The oracle (exact CPU DP) on one coloring of every template of the workload on R-MAT `scale`.
    Each template's time is scaled to the full graph by the ratio of the oracle's Lemma-1 work, and the
    rate is colorings/s of the workload's step (wl["batch"] colorings of every template)."""
    import oracle
    import sgcgen
    oracle.build()
    old = oracle.set_threads(threads) if threads else None
    try:
        rp, ci = sgcgen.rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1)
        n, nnz = len(rp) - 1, len(ci)
        secs, full, ratios = {}, {}, {}
        for name, spec in wl["templates"]:
            parent = make_parent(spec)
            k = len(parent)
            cols = oracle.colors(seed, n, k)
            t0 = time.perf_counter()
            oracle.count(rp, ci, parent, cols)
            secs[name] = time.perf_counter() - t0
            ratios[name] = oracle_work(full_n, full_nnz, parent, k) / oracle_work(n, nnz, parent, k)
            full[name] = secs[name] * ratios[name]
        used = oracle.threads()
    finally:
        if old:
            oracle.set_threads(old)
    step_s = sum(wl["batch"] * full[name] for name, _ in wl["templates"])
    return {"value": wl["batch"] * len(wl["templates"]) / step_s, "cores": used, "sample_s": sum(secs.values()),
            "sample_scale": scale, "sample_n": n, "sample_nnz": nnz, "per_template_s": secs, "work_ratio": ratios}


def survey_bytes(op, n, nnz, k, elem, batch):
    """Algorithmic bytes of one op over one pass of `batch` colorings, as the survey's measurement
    section defines them for the dense formulation (tables of C(k, x) columns over all n vertices, each
    read or written once; CSR read once): SpMM 4(n+1+nnz) + 2 b n C(k,p); eMA b n (C(k,a)+C(k,p)+C(k,t));
    fused last step b n (C(k,a)+C(k,p)); neighbour color histogram as an SpMM with p = 1."""
    C = math.comb
    kind, t, a, p = op["kind"], op["t"], op["a"], op["p"]
    if kind in ("spmm", "hist"):
        per = 2.0 * elem * n * C(k, p)
        return 4.0 * (n + 1 + nnz) + batch * per
    if kind == "ema":
        return batch * elem * n * float(C(k, a) + C(k, p) + C(k, t))
    if kind == "final":
        return batch * elem * n * float(C(k, a) + C(k, p))
    if kind == "final_leaf":
        return batch * elem * n * float(C(k, p))
    return 0.0


def oracle_work(n, nnz, parent, k):
    """Pruned-DP work of the oracle: sum over steps of nnz*C(k,p) + n*C(k,t)*C(t,p) (Lemma 1)."""
    import sgcgen  # noqa: F401
    kids = {i: [] for i in range(len(parent))}
    root = int(np.where(np.asarray(parent) < 0)[0][0])
    for i, p in enumerate(parent):
        if p >= 0:
            kids[int(p)].append(i)
    size = {}

    def sub(x):
        size[x] = 1 + sum(sub(c) for c in kids[x])
        return size[x]
    sub(root)
    work = 0.0
    for x in range(len(parent)):
        a = 1
        for c in reversed(sorted(kids[x])):
            p = size[c]
            t = a + p
            work += nnz * math.comb(k, p) + n * math.comb(k, t) * math.comb(t, p)
            a = t
    return work


def run_reference(args, wl, rank, world):
    """The oracle timed on the host cores: each step one coloring of the workload's template on an R-MAT
    scale-17 sample, scaled to the full workload by the ratio of the oracle's Lemma-1 work."""
    if rank != 0:
        return
    if args_workload_name(wl) == "batched":
        graphs = batched_graphs()
        sizes = [(len(rp) - 1, len(ci)) for _, rp, ci in graphs]
        for s in range(args.warmup):
            batched_oracle_rate(wl, sizes, seed=1 + s)
        rates, samples = [], []
        for s in range(args.steps):
            r = batched_oracle_rate(wl, sizes, seed=1 + args.warmup + s)
            rates.append(r["value"])
            samples.append(r)
        value = len(rates) / sum(1.0 / r for r in rates)
        cb = dict(samples[-1])
        cb["value"] = value
        colorings = 2 * len(wl["templates"]) * wl["batch"]
        out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "colorings/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * colorings / value,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u128",
               "data": "synthetic", "config": {"workload": "batched"}, "cpu_baseline": cb,
               "e2e": {"value": value, "unit": "colorings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return
    import oracle
    oracle.build()
    full_rp, full_ci = make_graph(wl)
    full_n, full_nnz = len(full_rp) - 1, len(full_ci)
    del full_rp, full_ci
    sc = wl.get("ref_scale", wl["scale"])
    for s in range(args.warmup):
        oracle_rate(wl, full_n, full_nnz, sc, seed=1 + s)
    step_s, rates, last = [], [], None
    for s in range(args.steps):
        last = oracle_rate(wl, full_n, full_nnz, sc, seed=1 + args.warmup + s)
        step_s.append(last["sample_s"])
        rates.append(last["value"])
    value = len(rates) / sum(1.0 / r for r in rates)
    full_size = sc == wl["scale"]
    sample = (f"each step one coloring of each template ({', '.join(n for n, _ in wl['templates'])}) on "
              + (f"the full R-MAT scale-{sc} graph" if full_size else
                 f"R-MAT scale {sc} ({last['sample_n']} vertices, {last['sample_nnz']} entries)")
              + ", exact unsigned 128/192-bit counts"
              + ("" if full_size else "; value = the workload's colorings/s at scale "
                 f"{wl['scale']} from the oracle's Lemma-1 work ratio per template (work_ratio)"))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "colorings/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(step_s) / len(step_s),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u128", "data": "synthetic",
        "config": config_of(wl, world),
        "cpu_baseline": {"value": value, "unit": "colorings/s", "cores": last["cores"], "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
        "ms_per_step_note": "host time of the sample step that ran (one coloring of each template)",
        "sample_scale": sc, "work_ratio": last["work_ratio"], "extrapolated": not full_size,
        "e2e": {"value": value, "unit": "colorings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def config_of(wl, world):
    name = args_workload_name(wl)
    subset = [n for n, _ in wl["templates"]] != WORKLOAD_TEMPLATES.get(name)
    return {"workload": name + ("" if wl["scale"] == WORKLOAD_SCALE.get(name) else f" (scale {wl['scale']} override)")
            + (f" (templates {','.join(n for n, _ in wl['templates'])} only)" if subset else ""),
            "graph": "R-MAT scale %d, edge factor 16, a=.57 b=.19 c=.19, seed 1"
            % wl["scale"], "templates": [name for name, _ in wl["templates"]], "k": "|T|",
            "colorings_per_step_per_gpu": wl["batch"] * len(wl["templates"]),
            "tables": "fp32 (power-of-two scaled), fp64 final reduction",
            "parallelism": f"colorings sharded over {world} GPU(s), no collective in the data path",
            "l2": "inputs larger than L2 (count tables of several GB per step)"}


_WL_NAME = {}


def args_workload_name(wl):
    return _WL_NAME.get(id(wl), "rmat20-spider10")


def serve_stream(sgc, g, Q, rate, base, warm=True):
    """One Poisson stream of Q queries (Pruefer trees of 3..14 vertices, 1..32 colorings) offered at `rate`
    queries/s to a fresh server (120 GB budget, 8 slots); returns the stream's measurements."""
    import sgcgen
    sizes = sgcgen.uniform_ints(3, 14, Q, seed=base + 11)
    ncol = sgcgen.uniform_ints(1, 32, Q, seed=base + 12)
    arrivals = sgcgen.poisson_arrivals(rate, Q, seed=base + 5)
    tpls = [sgc.Template(sgcgen.pruefer_tree(int(sizes[q]), base + q)) for q in range(Q)]
    if warm:
        # one small query of every size (plans, tables, module loading)
        srv = sgc.Server(g, 120 << 30, 8)
        for kk in range(3, 15):
            w = sgc.Template(sgcgen.pruefer_tree(kk, 77))
            srv.wait(srv.submit(w, [1]), 1)
        srv.close()
    srv = sgc.Server(g, 120 << 30, 8)
    t0 = time.perf_counter()
    tickets = []
    for q in range(Q):
        now = time.perf_counter() - t0
        if arrivals[q] > now:
            time.sleep(arrivals[q] - now)
        seeds = np.arange(int(ncol[q]), dtype=np.uint64) + np.uint64(10_000 * q + 1)
        tickets.append(srv.submit(tpls[q], seeds))
    lat = []
    for q, tk in enumerate(tickets):
        _, _, l = srv.wait(tk, int(ncol[q]))
        lat.append(l)
    span = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    colorings = int(np.sum(ncol))
    return {"offered_qps": rate, "queries": Q, "achieved_qps": Q / span, "colorings_per_s": colorings / span,
            "latency_p50_ms": float(np.percentile(lat, 50)), "latency_p99_ms": float(np.percentile(lat, 99)),
            "queue_p50_ms": st["queue_p50_ms"], "peak_inflight": st["peak_inflight"], "peak_bytes": st["peak_bytes"],
            "colorings": colorings, "span_s": span, "kernel_launches": st["kernel_launches"]}


def run_serving(args, wl, rank, world, local):
    """Continuous-batching server over a resident graph fed by Poisson query streams: the configured
    stream (--queries at --rate), and with --sweep a stream of --sweep-queries at each of several offered
    rates (offered vs achieved rate and p50 / p99 latency per rate; the sustainable rate is the highest
    offered rate the server keeps up with, achieved >= 90% of offered)."""
    import torch
    import paper_1903_04395_gb300 as sgc
    torch.cuda.set_device(local)
    if rank == 0:
        sgc.build()
    sgc.lib()
    rp, ci = make_graph(wl)
    n, nnz = len(rp) - 1, len(ci)
    d_rp = torch.from_numpy(rp).cuda()
    d_ci = torch.from_numpy(ci).cuda()
    g = sgc.Graph.from_device(n, nnz, d_rp.data_ptr(), d_ci.data_ptr())
    base = 1000 * (rank + 1)
    main = serve_stream(sgc, g, args.queries, args.rate, base)
    sweep = []
    if args.sweep:
        for i, r in enumerate(float(x) for x in args.sweep.split(",")):
            sweep.append(serve_stream(sgc, g, args.sweep_queries, r, base + 7919 * (i + 1), warm=False))
    span = main["span_s"]
    value = main["colorings"] / span
    res = {"metric": METRIC, "value": value * world, "unit": "colorings/s", "n_gpus": world, "steps": args.queries,
           "warmup": 12, "ms_per_step": 1e3 * span / args.queries, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "serving", "graph": "R-MAT scale 21, edge factor 16, a=.57 b=.19 c=.19, seed 1",
                      "templates": "Pruefer trees, 3..14 vertices (uniform)", "colorings_per_query": "uniform 1..32",
                      "arrivals": f"Poisson, {args.rate:g} queries/s", "budget_bytes": 120 << 30, "max_inflight": 8,
                      "queries": args.queries, "parallelism": f"one server per GPU ({world})"},
           "serving": main, "gpu_launches": main["kernel_launches"]}
    if sweep:
        ok = [x["offered_qps"] for x in sweep if x["achieved_qps"] >= 0.9 * x["offered_qps"]]
        res["sweep"] = sweep
        res["sustainable_qps"] = max(ok) if ok else None
        res["capacity_qps"] = max(x["achieved_qps"] for x in sweep)
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_ablation(args, wl, rank, world, local):
    """The paper's three variants on the GPU, same colorings (Section 6.1 and 7.1-7.2): Algorithm 1's loop
    order with no pruning (FASCIA order), the pruned neighbour sums of Eq. 2 taken one column at a time
    (PFASCIA: pruning without the row-wise SpMM), and the SpMM + eMA path (PGBSC).  pruning_speedup =
    PFASCIA / FASCIA, vectorization_speedup = PGBSC / PFASCIA."""
    import torch
    import paper_1903_04395_gb300 as sgc
    torch.cuda.set_device(local)
    if rank == 0:
        sgc.build()
    sgc.lib()
    stream = torch.cuda.Stream()
    rp, ci = make_graph(wl)
    g = sgc.Graph(rp, ci)
    B, K, W = wl["batch"], args.steps, args.warmup
    modes = (("pgbsc", 0), ("pfascia", 2), ("fascia", 1))
    out = []
    for name, spec in wl["templates"]:
        t = sgc.Template(make_parent(spec))
        row = {"template": name}
        for mode, code in modes:
            opt = sgc.sgc_options_init(precision=sgc.SGC_FP32, batch=B, stream=stream.cuda_stream, unpruned=code)
            seeds = np.arange(1, 1 + B * (W + K), dtype=np.uint64)
            for s_ in range(W):
                sgc.sgc_count(g.handle, t.handle, seeds[s_ * B:(s_ + 1) * B], opt)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            maps = []
            e0.record(stream)
            for s_ in range(W, W + K):
                maps.append(sgc.sgc_count(g.handle, t.handle, seeds[s_ * B:(s_ + 1) * B], opt)[1].copy())
            e1.record(stream)
            torch.cuda.synchronize()
            row[mode] = {"colorings_per_s": K * B / (e0.elapsed_time(e1) / 1e3), "maps_first": float(maps[0][0])}
        row["pruning_speedup"] = row["pfascia"]["colorings_per_s"] / row["fascia"]["colorings_per_s"]
        row["vectorization_speedup"] = row["pgbsc"]["colorings_per_s"] / row["pfascia"]["colorings_per_s"]
        row["total_speedup"] = row["pgbsc"]["colorings_per_s"] / row["fascia"]["colorings_per_s"]
        first = row["pgbsc"]["maps_first"]
        row["same_counts"] = all(abs(row[m]["maps_first"] - first) <= 1e-5 * abs(first) for m, _ in modes)
        out.append(row)
    res = {"metric": METRIC, "value": out[0]["pgbsc"]["colorings_per_s"], "unit": "colorings/s", "n_gpus": world,
           "steps": K, "warmup": W, "ms_per_step": 1e3 * B / out[0]["pgbsc"]["colorings_per_s"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "ablation", "graph": "R-MAT scale %d, edge factor 16, a=.57 b=.19 c=.19, seed 1"
                      % wl["scale"], "colorings_per_step": B},
           "ablation": out}
    if rank == 0:
        print(json.dumps(res), flush=True)


def batched_graphs():
    """The batched workload's graphs: (name, row_ptr, col_idx)."""
    import sgcgen
    er = sgcgen.er(500_000, 6_000_000, seed=1)
    rm = sgcgen.rmat(20, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1)
    return [("er500k-d24", *er), ("rmat20", *rm)]


def run_batched(args, wl, rank, world, local):
    """Six templates x 256 colorings on two resident graphs; per graph one sgc_count_many call, recorded and
    replayed as one CUDA graph (one launch for every pass of every template)."""
    import torch
    import paper_1903_04395_gb300 as sgc
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        sgc.build()
    if dist:
        dist.barrier()
    sgc.lib()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    NC = wl["batch"]
    parents = [make_parent(spec) for _, spec in wl["templates"]]
    NT = len(parents)
    graphs = []
    for name, rp, ci in batched_graphs():
        d_rp = torch.from_numpy(rp).cuda()
        d_ci = torch.from_numpy(ci).cuda()
        g = sgc.Graph.from_device(len(rp) - 1, len(ci), d_rp.data_ptr(), d_ci.data_ptr(), stream=stream.cuda_stream)
        graphs.append((name, g, len(rp) - 1, len(ci), rp, ci))
        del d_rp, d_ci
    templates = [sgc.Template(p) for p in parents]
    handles = [t.handle for t in templates]
    opt = sgc.sgc_options_init(precision=sgc.SGC_FP32, batch=0, stream=stream.cuda_stream, use_graph=1,
                               autotune=0 if args.no_autotune else 1)
    K, W = args.steps, args.warmup

    def seeds_for(step, gi):
        base = 1 + rank * 100_000_000 + (step * len(graphs) + gi) * NT * NC
        return np.arange(base, base + NT * NC, dtype=np.uint64).reshape(NT, NC)

    t_tune = time.perf_counter()
    for gi, (_, g, *_r) in enumerate(graphs):
        if not args.no_autotune:
            for h in handles:
                sgc.sgc_autotune(g.handle, h, sgc.sgc_options_init(precision=sgc.SGC_FP32, batch=NC,
                                                                   stream=stream.cuda_stream))
    t_tune = time.perf_counter() - t_tune
    for s in range(W):
        for gi, (_, g, *_r) in enumerate(graphs):
            sgc.sgc_count_many(g.handle, handles, seeds_for(s, gi), opt)
    torch.cuda.synchronize()
    launches0 = sum(g.stats()["kernel_launches"] for _, g, *_r in graphs)
    per_graph = [0.0] * len(graphs)
    sampler = ClockSampler(local)
    sampler.__enter__()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e_all0 = torch.cuda.Event(enable_timing=True)
    e_all1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_batched")
    e_all0.record(stream)
    for s in range(W, W + K):
        for gi, (_, g, *_r) in enumerate(graphs):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sgc.sgc_count_many(g.handle, handles, seeds_for(s, gi), opt)
            b.record(stream)
            b.synchronize()
            per_graph[gi] += a.elapsed_time(b)
    e_all1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    sampler.__exit__()
    ms = e_all0.elapsed_time(e_all1)
    if dist:
        from paper_1903_04395_gb300 import shard
        ms = shard.max_over_ranks(ms)
    launches = sum(g.stats()["kernel_launches"] for _, g, *_r in graphs) - launches0
    colorings = len(graphs) * NT * NC
    res = {"metric": METRIC, "value": world * K * colorings / (ms / 1e3), "unit": "colorings/s", "n_gpus": world,
           "steps": K, "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batched", "graphs": ["Erdos-Renyi n=500,000 m=6,000,000 seed 1",
                                                        "R-MAT scale 20, edge factor 16, a=.57 b=.19 c=.19, seed 1"],
                      "templates": [n for n, _ in wl["templates"]], "colorings_per_template": NC,
                      "launch": "one sgc_count_many per graph = one CUDA-graph launch (recorded in warm-up)",
                      "autotune": not args.no_autotune, "tables": "fp32 (power-of-two scaled), fp64 final reduction",
                      "parallelism": f"colorings sharded over {world} GPU(s), no collective in the data path",
                      "l2": "inputs larger than L2 (count tables of many GB per step)"},
           "per_graph": [{"graph": graphs[i][0], "ms_per_step": per_graph[i] / K,
                          "colorings_per_s": K * NT * NC / (per_graph[i] / 1e3)} for i in range(len(graphs))],
           "autotune_s": t_tune, "gpu_launches": launches, "clocks": sampler.summary()}
    if not args.no_autotune:
        res["tuned_shapes"] = {}
        for _, g, *_r in graphs[1:]:
            for (name, _), h in zip(wl["templates"], handles):
                rep = sgc.sgc_autotune(g.handle, h, sgc.sgc_options_init(precision=sgc.SGC_FP32, batch=NC,
                                                                         stream=stream.cuda_stream))
                res["tuned_shapes"][name] = [
                    (f"{e['name']}(t={e['t']},a={e['a']},p={e['p']})" if e["kind"] >= 0 else "batch") + ": " +
                    ", ".join(f"{sh}={m:.2f}ms" for sh, m in zip(e["shapes"], e["ms"])) +
                    f" -> {e['shapes'][e['chosen']]}" for e in rep]

    # roofline: one profiled step per graph after the timed region (op by op, CUDA events per op)
    peak, peak_kind = measured_peak()
    ops = {}
    popt = sgc.sgc_options_init(precision=sgc.SGC_FP32, batch=0, stream=stream.cuda_stream, use_graph=0,
                                autotune=opt.autotune)
    for gi, (gname, g, gn, gnnz, *_r) in enumerate(graphs):
        sgc.sgc_profile_enable(g.handle, True)
        sgc.sgc_count_many(g.handle, handles, seeds_for(W + K, gi), popt)
        for e in sgc.sgc_profile_read(g.handle):
            key = f"{gname}:{e['name']}(t={e['t']},a={e['a']},p={e['p']},B={e['batch']},k={e['k']})"
            sv = survey_bytes({"kind": e["name"], "t": e["t"], "a": e["a"], "p": e["p"]}, gn, gnnz, e["k"], 4,
                              e["batch"])
            ops[key] = {"op": key, "kind": e["name"], "ms": e["ms"], "passes": e["passes"],
                        "bytes": sv * e["passes"], "compulsory_bytes": e["bytes"] * e["passes"]}
        sgc.sgc_profile_enable(g.handle, False)
    tot = sum(o["ms"] for o in ops.values()) or 1e-9
    lst = sorted(ops.values(), key=lambda o: -o["ms"])
    for o in lst:
        o["share"] = o["ms"] / tot
        o["gbs"] = o["bytes"] / (o["ms"] * 1e-3) / 1e9 if o["ms"] > 0 else 0.0
        o["compulsory_gbs"] = o["compulsory_bytes"] / (o["ms"] * 1e-3) / 1e9 if o["ms"] > 0 else 0.0
    dom = lst[0]
    res["roofline"] = {"bound": "hbm", "achieved": dom["gbs"], "peak": peak, "unit": "GB/s",
                       "frac": dom["gbs"] / peak, "traffic": None, "kernel": dom["op"],
                       "compulsory_gbs": dom["compulsory_gbs"],
                       "bytes_definition": "survey measurement section (dense tables, n = all vertices, b = 4)",
                       "peak_source": f"{peak_kind} ({'MEASURED_PEAKS.json hbm_gbs' if peak_kind == 'measured' else '6.8 TB/s'})",
                       "note": "from one op-by-op profiled step per graph after the timed region"}
    res["ops"] = [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in o.items()} for o in lst[:12]]

    if not args.no_e2e:
        # end to end through the public API with host buffers: graph upload from pinned host memory, every
        # template's colorings from host seeds, results read back, graph released (planner shapes: tuning a
        # freshly created graph would be timed too)
        eopt = sgc.sgc_options_init(precision=sgc.SGC_FP32, batch=0, use_graph=1)
        pinned = [(torch.from_numpy(rp).pin_memory(), torch.from_numpy(ci).pin_memory(), n, nnz)
                  for _, _, n, nnz, rp, ci in graphs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for gi, (h_rp, h_ci, n, nnz) in enumerate(pinned):
            gh = sgc.sgc_graph_create(n, nnz, h_rp.data_ptr(), h_ci.data_ptr(), sgc.SGC_GRAPH_VALIDATE)
            try:
                sgc.sgc_count_many(gh, handles, seeds_for(W + K + 1, gi), eopt)
            finally:
                sgc.sgc_graph_destroy(gh)
        dt = time.perf_counter() - t0
        res["e2e"] = {"value": world * colorings / dt, "unit": "colorings/s", "steps": 1,
                      "h2d_bytes_per_step": sum(4 * (n + 1) + 4 * nnz + 8 * NT * NC for _, _, n, nnz in pinned),
                      "d2h_bytes_per_step": 8 * NT * NC * len(pinned),
                      "includes": "graph upload + validation + renumbering, planning, recording, counting, "
                                  "read-back, release"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = batched_oracle_rate(wl, [(n, nnz) for _, _, n, nnz, _, _ in graphs])
    if rank == 0:
        print(json.dumps(res), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def batched_oracle_rate(wl, full_sizes, sample_scale=15, seed=1):
    """The oracle on one coloring of every template on an R-MAT sample, scaled to the whole batched job by
    the oracle's Lemma-1 work ratio per (graph, template)."""
    import oracle
    import sgcgen
    oracle.build()
    rp, ci = sgcgen.rmat(sample_scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1)
    sn, snnz = len(rp) - 1, len(ci)
    NC = wl["batch"]
    job_s, sample_s, colorings = 0.0, 0.0, 0
    for _, spec in wl["templates"]:
        parent = make_parent(spec)
        k = len(parent)
        t0 = time.perf_counter()
        oracle.count(rp, ci, parent, oracle.colors(seed, sn, k))
        dt = time.perf_counter() - t0
        sample_s += dt
        for n, nnz in full_sizes:
            job_s += NC * dt * oracle_work(n, nnz, parent, k) / oracle_work(sn, snnz, parent, k)
            colorings += NC
    return {"value": colorings / job_s, "unit": "colorings/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"one coloring of each of the {len(wl['templates'])} templates on R-MAT scale {sample_scale} "
                      f"({sn} vertices, {snnz} entries), {sample_s:.1f} s in all, scaled per graph and template by "
                      f"the oracle's Lemma-1 work ratio to {colorings} colorings"}


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    _WL_NAME[id(wl)] = args.workload
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return
    if args.workload == "serving":
        run_serving(args, wl, rank, world, local)
        return
    if args.workload == "batched":
        run_batched(args, wl, rank, world, local)
        return
    if args.workload == "ablation":
        run_ablation(args, wl, rank, world, local)
        return

    import torch
    import paper_1903_04395_gb300 as sgc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        sgc.build()
    if dist:
        dist.barrier()
    sgc.lib()

    def barrier():
        if dist:
            dist.barrier()

    rp, ci = make_graph(wl)
    n, nnz = len(rp) - 1, len(ci)
    B = wl["batch"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    d_rp = torch.from_numpy(rp).cuda()
    d_ci = torch.from_numpy(ci).cuda()
    g = sgc.Graph.from_device(n, nnz, d_rp.data_ptr(), d_ci.data_ptr(), stream=stream.cuda_stream, rcm=args.rcm)
    templates = [(name, sgc.Template(make_parent(spec))) for name, spec in wl["templates"]]
    NT = len(templates)
    K, W = args.steps, args.warmup
    # warm-up, timed steps, then steps of their own for per-template rates, the profiled pass and FP64
    total_steps = W + K + max(2, K // 4) + 2 + 1 + max(2, K // 6)
    # distinct seeds for every (rank, step, template, coloring): each rank counts its own contiguous range
    from paper_1903_04395_gb300 import shard
    seeds = torch.from_numpy(shard.rank_seeds(1, world * total_steps * NT * B, rank, world).astype(np.int64)).cuda()
    out = torch.zeros(total_steps * NT * B, dtype=torch.float64, device="cuda")
    tpl_events = []  # per timed step and template: (template index, start, stop)

    def run_steps(opt, s0, s1, record=False):
        for s in range(s0, s1):
            for ti, (_, t) in enumerate(templates):
                off = (s * NT + ti) * B
                if record:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                sgc.sgc_count_device(g.handle, t.handle, seeds[off:].data_ptr(), B, opt, out[off:].data_ptr())
                if record:
                    e1.record(stream)
                    tpl_events.append((ti, e0, e1))

    def timed(opt, s0, steps, clocks=False):
        """Device time of `steps` steps from step s0 on: nothing but the counting calls between the two
        events (no per-op or per-template events)."""
        l0 = g.stats()["kernel_launches"]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.__enter__()
        barrier()
        torch.cuda.synchronize()
        # an NVTX range marks the timed region (ncu --nvtx --nvtx-include "timed_<precision>/")
        torch.cuda.nvtx.range_push("timed_" + ("fp64" if opt.precision == sgc.SGC_FP64 else "fp32"))
        e0.record(stream)
        run_steps(opt, s0, s0 + steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier()
        if sampler:
            sampler.__exit__()
        ms = e0.elapsed_time(e1)
        if dist:
            ms = shard.max_over_ranks(ms)
        return ms, g.stats()["kernel_launches"] - l0, (sampler.summary() if sampler else None)

    tune = 0 if (args.no_autotune or args.spmm_shape or args.ema_rows) else 1
    opt32 = sgc.sgc_options_init(precision=sgc.SGC_FP32, batch=B, stream=stream.cuda_stream, root=args.root,
                                 spmm_shape=args.spmm_shape, ema_rows=args.ema_rows, autotune=tune)
    t_w = time.perf_counter()
    run_steps(opt32, 0, W)  # warm-up: plans, autotuning (first call per template), CUDA-graph recording
    torch.cuda.synchronize()
    warm_s = time.perf_counter() - t_w
    ms, launches, clocks = timed(opt32, W, K, clocks=True)
    value = world * K * B * NT / (ms / 1e3)
    res = {"metric": METRIC, "value": value, "unit": "colorings/s", "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": config_of(wl, world), "warmup_s": warm_s}
    res["config"]["autotune"] = bool(tune)
    res["config"]["row_order"] = "reverse Cuthill-McKee after the rows longer than 256" if args.rcm else "degree"
    res["gpu_launches"] = launches
    res["clocks"] = clocks
    # the remaining measurements run after the timed region, on steps of their own
    extra = W + K
    chosen = {}  # (k, op, colorings per pass) -> the launch shape the autotuner kept
    if tune:
        res["tuned_shapes"] = {}
        for (name, t), (_, spec) in zip(templates, wl["templates"]):
            rep = sgc.sgc_autotune(g.handle, t.handle, opt32)
            for e in rep:
                if e["kind"] >= 0:
                    chosen[(len(make_parent(spec)), f"{e['name']}(t={e['t']},a={e['a']},p={e['p']})", e["batch"])] = \
                        e["shapes"][e["chosen"]]
            res["tuned_shapes"][name] = [
                (f"{e['name']}(t={e['t']},a={e['a']},p={e['p']},B={e['batch']})" if e["kind"] >= 0 else "batch") +
                ": " + ", ".join(f"{sgc.SHAPE_NAMES.get(sh, sh) if e['kind'] == 2 else sh}={m:.2f}ms"
                                 for sh, m in zip(e["shapes"], e["ms"])) +
                f" -> {e['shapes'][e['chosen']]}" for e in rep]
    if NT > 1:
        # per-template rates: events around each template's call, on steps of their own
        kt = max(2, K // 4)
        tpl_events.clear()
        torch.cuda.synchronize()
        run_steps(opt32, extra, extra + kt, record=True)
        torch.cuda.synchronize()
        extra += kt
        per = {}
        for ti, a, b_ in tpl_events:
            per[ti] = per.get(ti, 0.0) + a.elapsed_time(b_)
        res["per_template"] = [{"template": templates[ti][0], "colorings_per_s": kt * B / (per[ti] / 1e3),
                                "ms_per_step": per[ti] / kt, "steps": kt} for ti in sorted(per)]

    # roofline of the dominant op: a profiled step after the timed region (CUDA events around every op,
    # recorded on the stream the op's kernels are launched on)
    sgc.sgc_profile_enable(g.handle, True)
    kp = 1 if NT > 1 else 2
    run_steps(opt32, extra, extra + kp)
    prof = sgc.sgc_profile_read(g.handle)
    sgc.sgc_profile_enable(g.handle, False)
    extra += kp
    peak, peak_kind = measured_peak()
    ops = []
    tot_ms = max(sum(x["ms"] for x in prof), 1e-9)
    for e in prof:
        avg_ms = e["ms"] / max(e["passes"], 1)
        sv = survey_bytes({"kind": e["name"], "t": e["t"], "a": e["a"], "p": e["p"]}, n, nnz,
                          e.get("k") or templ_k_of(e, templates), 4, e["batch"])
        ops.append({"op": f"{e['name']}(t={e['t']},a={e['a']},p={e['p']})", "kind": e["name"], "k": templ_k_of(e, templates),
                    "batch": e["batch"], "passes": e["passes"], "kernels": e["kernels"], "ms_per_pass": avg_ms,
                    "survey_bytes_per_pass": sv, "gbs": sv / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0,
                    "compulsory_bytes_per_pass": e["bytes"],
                    "compulsory_gbs": e["bytes"] / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0,
                    "gather_bytes_per_pass": e["gather_bytes"],
                    "gather_gbs": e["gather_bytes"] / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0,
                    "share": e["ms"] / tot_ms})
    ops.sort(key=lambda o: -o["share"])
    dom = ops[0]
    res["roofline"] = {"bound": "hbm", "achieved": dom["gbs"], "peak": peak, "unit": "GB/s", "frac": dom["gbs"] / peak,
                       "traffic": recorded_traffic(dom["op"], dom["k"], dom["batch"],
                                                   chosen.get((dom["k"], dom["op"], dom["batch"]))),
                       "kernel": dom["op"], "launch_shape": chosen.get((dom["k"], dom["op"], dom["batch"])),
                       "k": dom["k"], "colorings_per_launch": dom["batch"],
                       "peak_source": f"{peak_kind} ({'MEASURED_PEAKS.json hbm_gbs' if peak_kind == 'measured' else '6.8 TB/s'}, burst copy)",
                       "bytes_per_launch": dom["survey_bytes_per_pass"],
                       "bytes_definition": "survey measurement section: SpMM 4(n+1+nnz) + 2 b n C(k,p) per coloring, "
                                           "eMA b n (C(k,a)+C(k,p)+C(k,t)); n = all vertices, b = 4",
                       "compulsory_gbs": dom["compulsory_gbs"], "gather_gbs": dom["gather_gbs"],
                       "note": "from a profiled step after the clean timed region; compulsory_gbs counts the "
                               "relative-color tables this library moves (each entry once); gather_gbs the "
                               "neighbour rows an SpMM gathers (once per stored entry, served by L2 and HBM)"}
    se = [o for o in ops if o["kind"] in ("spmm", "hist", "ema", "final", "final_leaf")]
    se_bytes = sum(o["survey_bytes_per_pass"] * o["passes"] for o in se)
    se_ms = sum(o["ms_per_pass"] * o["passes"] for o in se)
    res["spmm_ema_gbs"] = se_bytes / (se_ms * 1e-3) / 1e9 if se_ms else None
    res["spmm_ema_frac"] = res["spmm_ema_gbs"] / peak if se_ms else None
    res["ops"] = [{k_: (round(v, 4) if isinstance(v, float) else v) for k_, v in o.items()} for o in ops]
    # bytes an op actually has to move cannot stream faster than the copy peak: an op above it counts
    # bytes its kernels do not move
    above = [o["op"] for o in ops if o["compulsory_gbs"] > 1.05 * peak]
    res["ops_compulsory_above_peak"] = above
    if above:
        print(f"warning: compulsory bytes above the copy peak for {above}", file=sys.stderr)

    if not args.no_fp64 and wl.get("fp64", True):
        opt64 = sgc.sgc_options_init(precision=sgc.SGC_FP64, batch=B, stream=stream.cuda_stream)
        k64 = max(2, K // 6)
        run_steps(opt64, extra, extra + 1)
        torch.cuda.synchronize()
        ms64, _, _ = timed(opt64, extra + 1, k64)
        extra += 1 + k64
        res["fp64"] = {"value": world * k64 * B * NT / (ms64 / 1e3), "unit": "colorings/s", "steps": k64,
                       "ms_per_step": ms64 / k64, "dtype": "f64"}

    if not args.no_e2e:
        # the user-facing call with host buffers: graph upload from pinned host memory, counting with host
        # seeds, result read back to the host, graph released - every step
        h_rp = torch.from_numpy(rp).pin_memory()
        h_ci = torch.from_numpy(ci).pin_memory()
        maps_host = np.zeros(B, dtype=np.float64)
        k_e2e = max(2, K // 4)

        def e2e_step(s):
            gh = sgc.sgc_graph_create(n, nnz, h_rp.data_ptr(), h_ci.data_ptr(),
                                      sgc.SGC_GRAPH_VALIDATE | (sgc.SGC_GRAPH_ORDER_RCM if args.rcm else 0))
            try:
                for ti, (_, t) in enumerate(templates):
                    sd = np.arange(B, dtype=np.uint64) + np.uint64(50_000_000 + rank * 1_000_000 + (s * NT + ti) * B)
                    # the user's call with default options: the library picks the colorings per pass
                    sgc.sgc_count(gh, t.handle, sd, sgc.sgc_options_init(precision=sgc.SGC_FP32),
                                  maps_out=maps_host)
            finally:
                sgc.sgc_graph_destroy(gh)

        e2e_step(0)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for s in range(k_e2e):
            e2e_step(s + 1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist:
            dt = shard.max_over_ranks(dt)
        res["e2e"] = {"value": world * k_e2e * B * NT / dt, "unit": "colorings/s", "steps": k_e2e,
                      "h2d_bytes_per_step": 4 * (n + 1) + 4 * nnz + 8 * B * NT, "d2h_bytes_per_step": 8 * B * NT,
                      "includes": "graph upload + validation + renumbering, planning, counting (default options: "
                                  "planner launch shapes and colorings per pass; a new graph handle is not tuned), "
                                  "read-back, release"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cs = wl.get("cpu_scale", wl["scale"])
        c1 = wl.get("cpu_scale_1t", cs)
        multi = oracle_rate(wl, n, nnz, cs, seed=1)
        single = oracle_rate(wl, n, nnz, c1, threads=1, seed=1)

        def where(r):
            return ("the full graph" if r["sample_scale"] == wl["scale"] else
                    f"R-MAT scale {r['sample_scale']} ({r['sample_n']} vertices, {r['sample_nnz']} entries), "
                    f"scaled to the workload by the oracle's Lemma-1 work ratio per template")
        res["cpu_baseline"] = {
            "value": multi["value"], "unit": "colorings/s", "cores": multi["cores"], "kind": "oracle",
            "cpu_model": cpu_model(), "value_1thread": single["value"],
            "sample": f"{multi['cores']} threads: one coloring (seed 1) of each template on {where(multi)}, "
                      f"{multi['sample_s']:.1f} s; 1 thread: the same on {where(single)}, {single['sample_s']:.1f} s; "
                      "exact unsigned 128/192-bit counts"}

    if rank == 0:
        print(json.dumps(res), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
