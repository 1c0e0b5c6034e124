"""Python binding of libsgc, the GB300 implementation of color-coding tree
counting (Chen et al., "A GraphBLAS Approach for Subgraph Counting").

Argument marshalling only: every step of the counting path runs in the CUDA
kernels of ``libsgc.so`` (see ``include/sgc.h`` for the C ABI this mirrors).
The functions keep the C names (``sgc_graph_create``, ``sgc_count``, ...);
``Graph``, ``Template`` and ``count`` are small conveniences on top.

There is no CPU fallback: if ``libsgc.so`` has not been built, or no CUDA
device is usable, calls raise ``SgcError``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from ._build import LIB, build  # noqa: F401

SGC_OK, SGC_ERR_INVALID, SGC_ERR_OOM, SGC_ERR_CUDA = 0, 1, 2, 3
SGC_ERR_TIMEOUT, SGC_ERR_OVERFLOW, SGC_ERR_INTERNAL, SGC_ERR_UNSUPPORTED = 4, 5, 6, 7
SGC_FP32, SGC_FP64 = 0, 1
SGC_GRAPH_VALIDATE = 1
SGC_GRAPH_ORDER_RCM = 2
SGC_MAX_K = 18

_STATUS = {0: "SGC_OK", 1: "SGC_ERR_INVALID", 2: "SGC_ERR_OOM", 3: "SGC_ERR_CUDA", 4: "SGC_ERR_TIMEOUT",
           5: "SGC_ERR_OVERFLOW", 6: "SGC_ERR_INTERNAL", 7: "SGC_ERR_UNSUPPORTED"}


class SgcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class sgc_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("batch", ctypes.c_int32), ("mem_limit", ctypes.c_int64),
                ("stream", ctypes.c_void_p), ("root", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("spmm_shape", ctypes.c_int32), ("ema_rows", ctypes.c_int32),
                ("colors", ctypes.c_int32), ("unpruned", ctypes.c_int32)]


class sgc_graph_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_active", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("max_degree", ctypes.c_int32), ("n_heavy", ctypes.c_int32), ("n_segments", ctypes.c_int32),
                ("device", ctypes.c_int32), ("kernel_launches", ctypes.c_int64), ("ordering", ctypes.c_int32)]


class sgc_plan_info(ctypes.Structure):
    _fields_ = [("root", ctypes.c_int32), ("n_tables", ctypes.c_int32), ("n_spmm", ctypes.c_int32),
                ("n_ema", ctypes.c_int32), ("batch", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64),
                ("est_bytes", ctypes.c_double), ("est_spmm_bytes", ctypes.c_double), ("est_fma", ctypes.c_double)]


class sgc_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("inflight", ctypes.c_int32), ("peak_inflight", ctypes.c_int32), ("peak_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("latency_p50_ms", ctypes.c_double),
                ("latency_p99_ms", ctypes.c_double), ("queue_p50_ms", ctypes.c_double), ("span_s", ctypes.c_double)]


class sgc_op_profile(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("t", ctypes.c_int32), ("a", ctypes.c_int32), ("p", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("passes", ctypes.c_int64), ("kernels", ctypes.c_int64),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double), ("flops", ctypes.c_double),
                ("gather_bytes", ctypes.c_double), ("k", ctypes.c_int32)]


class sgc_tune_entry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("t", ctypes.c_int32), ("a", ctypes.c_int32), ("p", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("n_candidates", ctypes.c_int32), ("chosen", ctypes.c_int32),
                ("shapes", ctypes.c_int32 * 8), ("ms", ctypes.c_double * 8)]


OP_KINDS = {0: "color", 1: "hist", 2: "spmm", 4: "ema", 5: "final_leaf", 6: "final", 7: "final_sum", 8: "unpruned"}

# exported symbols with their ctypes signatures (restype, argtypes)
_P = ctypes.POINTER
_vp = ctypes.c_void_p
SIGNATURES = {
    "sgc_options_init": (None, [_P(sgc_options)]),
    "sgc_last_error": (ctypes.c_char_p, []),
    "sgc_version": (ctypes.c_int32, []),
    "sgc_graph_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _P(ctypes.c_int32), _P(ctypes.c_int32),
                                        ctypes.c_uint32, _P(_vp)]),
    "sgc_graph_create_device": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _vp, _vp, ctypes.c_uint32, _vp,
                                               _P(_vp)]),
    "sgc_graph_stats_get": (ctypes.c_int, [_vp, _P(sgc_graph_stats)]),
    "sgc_graph_destroy": (None, [_vp]),
    "sgc_template_create": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_int32), _P(_vp)]),
    "sgc_template_automorphisms": (ctypes.c_int, [_vp, _P(ctypes.c_uint64)]),
    "sgc_template_destroy": (None, [_vp]),
    "sgc_plan_get": (ctypes.c_int, [_vp, _vp, _P(sgc_options), _P(sgc_plan_info)]),
    "sgc_count": (ctypes.c_int, [_vp, _vp, _P(ctypes.c_uint64), ctypes.c_int32, _P(sgc_options),
                                 _P(ctypes.c_double), _P(ctypes.c_double)]),
    "sgc_count_device": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, _P(sgc_options), _vp]),
    "sgc_count_many": (ctypes.c_int, [_vp, ctypes.c_int32, _P(_vp), _P(ctypes.c_uint64), ctypes.c_int32,
                                      _P(sgc_options), _P(ctypes.c_double), _P(ctypes.c_double)]),
    "sgc_autotune": (ctypes.c_int, [_vp, _vp, _P(sgc_options), _P(sgc_tune_entry), ctypes.c_int32,
                                    _P(ctypes.c_int32)]),
    "sgc_iterations_bound": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_double, ctypes.c_double]),
    "sgc_estimate": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                                    ctypes.c_int64, _P(sgc_options), _P(ctypes.c_double), _P(ctypes.c_int64),
                                    _P(ctypes.c_double)]),
    "sgc_count_device_static": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, _P(sgc_options), _vp]),
    "sgc_estimate_from_maps": (ctypes.c_int, [_vp, ctypes.c_int32, _P(ctypes.c_double), ctypes.c_int64,
                                              _P(ctypes.c_double)]),
    "sgc_server_create": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int32, _P(_vp)]),
    "sgc_server_submit": (ctypes.c_int, [_vp, _vp, _P(ctypes.c_uint64), ctypes.c_int32, ctypes.c_int32,
                                         _P(ctypes.c_uint64)]),
    "sgc_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_int32, _P(ctypes.c_double),
                                       _P(ctypes.c_double), _P(ctypes.c_double)]),
    "sgc_server_stats_get": (ctypes.c_int, [_vp, _P(sgc_server_stats)]),
    "sgc_server_destroy": (None, [_vp]),
    "sgc_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "sgc_profile_read": (ctypes.c_int, [_vp, _P(sgc_op_profile), ctypes.c_int32, _P(ctypes.c_int32)]),
}

_lib = None


def lib():
    """Load libsgc.so (built in-tree by ``build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise SgcError(SGC_ERR_CUDA, f"{LIB} is not built; run paper_1903_04395_gb300.build()")
        handle = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(rc: int):
    if rc != SGC_OK:
        raise SgcError(rc, lib().sgc_last_error().decode(errors="replace"))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    if a.size == 0:
        a = np.zeros(1, dtype=np.int32)
    return a, a.ctypes.data_as(_P(ctypes.c_int32))


# ----------------------------------------------------------- C-named calls --

def sgc_options_init(precision=SGC_FP32, batch=0, mem_limit=0, stream=None, root=-1, use_graph=1,
                     autotune=0, spmm_shape=0, ema_rows=0, colors=0, unpruned=0) -> sgc_options:
    o = sgc_options()
    lib().sgc_options_init(ctypes.byref(o))
    o.precision, o.batch, o.mem_limit, o.root, o.use_graph = precision, batch, mem_limit, root, use_graph
    o.autotune, o.spmm_shape, o.ema_rows, o.colors = autotune, spmm_shape, ema_rows, colors
    o.unpruned = unpruned
    o.stream = stream
    return o


def sgc_version() -> int:
    return int(lib().sgc_version())


def sgc_graph_create(n: int, nnz: int, row_ptr, col_idx, flags: int = SGC_GRAPH_VALIDATE) -> int:
    """row_ptr / col_idx: host arrays, or integer host addresses (e.g. pinned buffers)."""
    if isinstance(row_ptr, int) and isinstance(col_idx, int):
        rpp = ctypes.cast(row_ptr, _P(ctypes.c_int32))
        cip = ctypes.cast(col_idx, _P(ctypes.c_int32))
    else:
        rp, rpp = _i32(row_ptr)
        ci, cip = _i32(col_idx)
    out = _vp()
    _check(lib().sgc_graph_create(n, nnz, rpp, cip, flags, ctypes.byref(out)))
    return out.value


def sgc_graph_create_device(n: int, nnz: int, d_row_ptr: int, d_col_idx: int, flags: int = SGC_GRAPH_VALIDATE,
                            stream: int | None = None) -> int:
    out = _vp()
    _check(lib().sgc_graph_create_device(n, nnz, d_row_ptr, d_col_idx, flags, stream, ctypes.byref(out)))
    return out.value


def sgc_graph_stats_get(g: int) -> dict:
    s = sgc_graph_stats()
    _check(lib().sgc_graph_stats_get(g, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in sgc_graph_stats._fields_}


def sgc_graph_destroy(g: int) -> None:
    lib().sgc_graph_destroy(g)


def sgc_template_create(k: int, parent) -> int:
    p, pp = _i32(parent)
    out = _vp()
    _check(lib().sgc_template_create(k, pp, ctypes.byref(out)))
    return out.value


def sgc_template_automorphisms(t: int) -> int:
    a = ctypes.c_uint64(0)
    _check(lib().sgc_template_automorphisms(t, ctypes.byref(a)))
    return int(a.value)


def sgc_template_destroy(t: int) -> None:
    lib().sgc_template_destroy(t)


def sgc_plan_get(g: int, t: int, opt: sgc_options | None = None) -> dict:
    info = sgc_plan_info()
    _check(lib().sgc_plan_get(g, t, ctypes.byref(opt) if opt is not None else None, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in sgc_plan_info._fields_}


def sgc_count(g: int, t: int, seeds, opt: sgc_options | None = None, maps_out: np.ndarray | None = None):
    """Host-buffer count: returns (estimate, colorful maps per coloring as float64 array)."""
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    n = int(s.size)
    maps = maps_out if maps_out is not None and maps_out.size >= max(n, 1) else np.zeros(max(n, 1), dtype=np.float64)
    est = ctypes.c_double(0.0)
    _check(lib().sgc_count(g, t, s.ctypes.data_as(_P(ctypes.c_uint64)) if n else None, n,
                           ctypes.byref(opt) if opt is not None else None, ctypes.byref(est),
                           maps.ctypes.data_as(_P(ctypes.c_double))))
    return float(est.value), maps[:n]


def sgc_count_device(g: int, t: int, d_seeds: int, n_iter: int, opt: sgc_options | None, d_maps: int) -> None:
    """Device-buffer count: enqueue on opt.stream (or the graph's stream); no synchronisation."""
    _check(lib().sgc_count_device(g, t, d_seeds, n_iter, ctypes.byref(opt) if opt is not None else None, d_maps))


def sgc_count_many(g: int, templates, seeds, opt: sgc_options | None = None):
    """Several templates in one call: seeds has shape (n_templates, n_iter); returns
    (estimates[n_templates], colorful maps[n_templates, n_iter])."""
    handles = (_vp * max(len(templates), 1))(*templates)
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64).reshape(len(templates), -1))
    n_t, n_iter = s.shape
    est = np.zeros(max(n_t, 1), dtype=np.float64)
    maps = np.zeros(max(n_t * n_iter, 1), dtype=np.float64)
    _check(lib().sgc_count_many(g, n_t, handles, s.ctypes.data_as(_P(ctypes.c_uint64)) if s.size else None, n_iter,
                                ctypes.byref(opt) if opt is not None else None,
                                est.ctypes.data_as(_P(ctypes.c_double)), maps.ctypes.data_as(_P(ctypes.c_double))))
    return est[:n_t], maps[:n_t * n_iter].reshape(n_t, n_iter)


SHAPE_NAMES = {1: "direct", 2: "direct+prefetch", 3: "buckets", 4: "register-buckets", 5: "direct+packed", 6: "direct+ring2",
               7: "direct+ring4", 8: "direct-batch",
               9: "direct-batch+lane-table", 10: "buckets-batch", 11: "direct-batch-g8", 12: "direct-batch-g12",
               13: "direct-batch-private", 14: "direct-batch-unrolled", 15: "direct-batch-wide",
               16: "grouped", 17: "grouped-256",
               18: "grouped-staged", 19: "grouped-staged-2"}


def sgc_autotune(g: int, t: int, opt: sgc_options | None = None) -> list:
    """Run (or read back) the autotuner for one template: per op, the launch shapes timed (ms, one pass)
    and the one kept; the last entry (kind -1) compares batch sizes (ms per coloring)."""
    cap = 64
    buf = (sgc_tune_entry * cap)()
    n = ctypes.c_int32(0)
    _check(lib().sgc_autotune(g, t, ctypes.byref(opt) if opt is not None else None, buf, cap, ctypes.byref(n)))
    out = []
    for i in range(min(n.value, cap)):
        e = buf[i]
        m = e.n_candidates
        out.append({"kind": e.kind, "name": OP_KINDS.get(e.kind, "batch"), "t": e.t, "a": e.a, "p": e.p,
                    "batch": e.batch, "shapes": list(e.shapes[:m]), "ms": list(e.ms[:m]), "chosen": e.chosen})
    return out


def sgc_iterations_bound(k: int, eps: float, delta: float) -> int:
    """Worst-case colorings for an (eps, delta)-approximation: ceil(e^k ln(1/delta) / eps^2)."""
    return int(lib().sgc_iterations_bound(k, eps, delta))


def sgc_estimate(g: int, t: int, eps: float, delta: float, first_seed: int = 1, min_iter: int = 0,
                 max_iter: int = 0, opt: sgc_options | None = None):
    """Count colorings until the (eps, delta) stopping rule holds; returns (estimate, n_used, rel_half_width)."""
    est = ctypes.c_double(0)
    n = ctypes.c_int64(0)
    rel = ctypes.c_double(0)
    _check(lib().sgc_estimate(g, t, eps, delta, first_seed, min_iter, max_iter,
                              ctypes.byref(opt) if opt is not None else None, ctypes.byref(est), ctypes.byref(n),
                              ctypes.byref(rel)))
    return float(est.value), int(n.value), float(rel.value)


SGC_STATIC_WORKSPACE_BYTES = 64 << 20


def sgc_estimate_from_maps(t: int, maps, colors: int = 0) -> float:
    """The estimate of Section 2.1 from per-coloring colorful maps (computed by libsgc)."""
    m = np.ascontiguousarray(maps, dtype=np.float64)
    out = ctypes.c_double(0.0)
    _check(lib().sgc_estimate_from_maps(t, int(colors), m.ctypes.data_as(_P(ctypes.c_double)), int(m.size),
                                        ctypes.byref(out)))
    return float(out.value)


def sgc_count_device_static(g: int, t: int, d_seeds: int, n_iter: int, opt: sgc_options | None, d_maps: int) -> None:
    """Like sgc_count_device, but with no device allocation: all scratch comes from the library's static
    device array of SGC_STATIC_WORKSPACE_BYTES (for callers that cannot call cudaMalloc while counting).
    Waits for its work before returning; calls that overlap on the GPU race on the shared array."""
    _check(lib().sgc_count_device_static(g, t, d_seeds, n_iter, ctypes.byref(opt) if opt is not None else None,
                                         d_maps))


def sgc_profile_enable(g: int, on: bool = True) -> None:
    _check(lib().sgc_profile_enable(g, 1 if on else 0))


def sgc_profile_read(g: int) -> list:
    """Aggregated per-op device times (CUDA events) since profiling was enabled or last read."""
    cap = 64
    buf = (sgc_op_profile * cap)()
    n = ctypes.c_int32(0)
    _check(lib().sgc_profile_read(g, buf, cap, ctypes.byref(n)))
    out = []
    for i in range(min(n.value, cap)):
        e = {f: getattr(buf[i], f) for f, _ in sgc_op_profile._fields_}
        e["name"] = OP_KINDS.get(e["kind"], str(e["kind"]))
        out.append(e)
    return out


def sgc_server_create(g: int, mem_budget: int, max_inflight: int = 8) -> int:
    out = _vp()
    _check(lib().sgc_server_create(g, mem_budget, max_inflight, ctypes.byref(out)))
    return out.value


def sgc_server_submit(srv: int, t: int, seeds, precision: int = SGC_FP32) -> int:
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    ticket = ctypes.c_uint64(0)
    _check(lib().sgc_server_submit(srv, t, s.ctypes.data_as(_P(ctypes.c_uint64)), int(s.size), precision,
                                   ctypes.byref(ticket)))
    return int(ticket.value)


def sgc_server_wait(srv: int, ticket: int, n: int, timeout_ms: int = -1):
    """Returns (estimate, maps[n], latency_ms); raises SgcError (SGC_ERR_TIMEOUT if not done in time)."""
    est = ctypes.c_double(0)
    lat = ctypes.c_double(0)
    maps = np.zeros(max(n, 1), dtype=np.float64)
    _check(lib().sgc_server_wait(srv, ticket, timeout_ms, ctypes.byref(est), maps.ctypes.data_as(_P(ctypes.c_double)),
                                 ctypes.byref(lat)))
    return float(est.value), maps[:n], float(lat.value)


def sgc_server_stats_get(srv: int) -> dict:
    st = sgc_server_stats()
    _check(lib().sgc_server_stats_get(srv, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in sgc_server_stats._fields_}


def sgc_server_destroy(srv: int) -> None:
    lib().sgc_server_destroy(srv)


class Server:
    """Owning wrapper of an sgc_server handle (continuous-batching counting server)."""

    def __init__(self, graph: "Graph", mem_budget: int, max_inflight: int = 8):
        self.graph = graph  # keeps the graph alive
        self.templates = {}
        self.handle = sgc_server_create(graph.handle, mem_budget, max_inflight)

    def submit(self, template: "Template", seeds, precision: str = "fp32") -> int:
        self.templates[id(template)] = template  # keeps submitted templates alive
        return sgc_server_submit(self.handle, template.handle, seeds,
                                 _precision(precision))

    def wait(self, ticket: int, n: int, timeout_ms: int = -1):
        return sgc_server_wait(self.handle, ticket, n, timeout_ms)

    def stats(self) -> dict:
        return sgc_server_stats_get(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sgc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------- wrappers --

class Graph:
    """Owning wrapper of an sgc_graph handle."""

    def __init__(self, row_ptr, col_idx, validate: bool = True, rcm: bool = False):
        row_ptr = np.asarray(row_ptr)
        n = len(row_ptr) - 1
        flags = (SGC_GRAPH_VALIDATE if validate else 0) | (SGC_GRAPH_ORDER_RCM if rcm else 0)
        self.handle = sgc_graph_create(n, len(col_idx), row_ptr, col_idx, flags)

    @classmethod
    def from_device(cls, n: int, nnz: int, d_row_ptr: int, d_col_idx: int, validate: bool = True, stream=None,
                    rcm: bool = False):
        self = cls.__new__(cls)
        flags = (SGC_GRAPH_VALIDATE if validate else 0) | (SGC_GRAPH_ORDER_RCM if rcm else 0)
        self.handle = sgc_graph_create_device(n, nnz, d_row_ptr, d_col_idx, flags, stream)
        return self

    def stats(self) -> dict:
        return sgc_graph_stats_get(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sgc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Template:
    """Owning wrapper of an sgc_template handle."""

    def __init__(self, parent):
        parent = np.asarray(parent, dtype=np.int32)
        self.k = len(parent)
        self.handle = sgc_template_create(self.k, parent)

    @property
    def automorphisms(self) -> int:
        return sgc_template_automorphisms(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sgc_template_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class CountResult:
    estimate: float
    maps: np.ndarray


def _precision(name: str) -> int:
    """'fp32' or 'fp64' -> sgc_precision; anything else is an error (no silent default)."""
    if name == "fp32":
        return SGC_FP32
    if name == "fp64":
        return SGC_FP64
    raise ValueError(f"precision must be 'fp32' or 'fp64', not {name!r}")


def count(graph: Graph, template: Template, seeds, precision: str = "fp32", batch: int = 0, root: int = -1,
          mem_limit: int = 0, use_graph: bool = True, autotune: bool = False, spmm_shape: int = 0,
          ema_rows: int = 0, colors: int = 0, unpruned: int = 0) -> CountResult:
    """unpruned: 0 = the SpMM + eMA path; 1 = Algorithm 1's loop order (no pruning); 2 = pruned neighbour
    sums taken one column at a time (no row-wise SpMM).  True counts as 1."""
    opt = sgc_options_init(precision=_precision(precision), batch=batch, root=root,
                           mem_limit=mem_limit, use_graph=1 if use_graph else 0, autotune=1 if autotune else 0,
                           spmm_shape=spmm_shape, ema_rows=ema_rows, colors=colors,
                           unpruned=int(unpruned))
    est, maps = sgc_count(graph.handle, template.handle, seeds, opt)
    return CountResult(est, maps)


def count_many(graph: Graph, templates, seeds, precision: str = "fp32", batch: int = 0, use_graph: bool = True,
               autotune: bool = False, mem_limit: int = 0):
    """Count several templates in one call (one CUDA-graph launch when use_graph): seeds (n_templates, n_iter).
    Returns (estimates, maps[n_templates, n_iter])."""
    opt = sgc_options_init(precision=_precision(precision), batch=batch,
                           use_graph=1 if use_graph else 0, autotune=1 if autotune else 0, mem_limit=mem_limit)
    return sgc_count_many(graph.handle, [t.handle for t in templates], seeds, opt)


def plan(graph: Graph, template: Template, precision: str = "fp32", batch: int = 0, root: int = -1) -> dict:
    opt = sgc_options_init(precision=_precision(precision), batch=batch, root=root)
    return sgc_plan_get(graph.handle, template.handle, opt)
