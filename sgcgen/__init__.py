"""Seeded synthetic inputs: simple undirected graphs (CSR) and tree templates.

This module only makes inputs.  It holds none of the counting method's
arithmetic, so the CPU oracle and the CUDA library are both fed from it
without sharing any of the method's code.  Graph generation runs in the small
C library ``sgcgen.c`` (compiled in-tree with gcc on first use); the tree
helpers are plain Python.

Recipes (all integer arithmetic on SplitMix64 draws, identical on x86-64 and
aarch64):

* ``rmat(scale, ...)``: R-MAT, ``2**scale * edge_factor`` samples, quadrant
  probabilities a, b, c (d = 1 - a - b - c), no noise, no vertex permutation,
  symmetrised, self-loops and duplicates dropped.
* ``er(n, m, seed)``: Erdos-Renyi G(n, m) with m distinct non-loop edges.
* ``pruefer_tree(k, seed)``: uniform labelled tree from a Pruefer sequence,
  rooted at vertex 0.
* ``path_tree``, ``spider_tree``, ``star_tree``: fixed template shapes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgcgen.c")
_LIB_PATH = os.path.join(_HERE, "libsgcgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libsgcgen.so`` next to its source (gcc, -O2, position independent)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            i32pp = P(P(ctypes.c_int32))
            lib.sgcgen_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_uint64, i32pp, i32pp, P(ctypes.c_int64)]
            lib.sgcgen_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32pp, i32pp,
                                      P(ctypes.c_int64)]
            lib.sgcgen_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, P(ctypes.c_int32),
                                              P(ctypes.c_int32), i32pp, i32pp, P(ctypes.c_int64)]
            lib.sgcgen_pruefer_tree.argtypes = [ctypes.c_int32, ctypes.c_uint64, P(ctypes.c_int32)]
            lib.sgcgen_splitmix64_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.sgcgen_splitmix64_draw.restype = ctypes.c_uint64
            lib.sgcgen_free.argtypes = [ctypes.c_void_p]
            for f in (lib.sgcgen_rmat, lib.sgcgen_er, lib.sgcgen_from_edges, lib.sgcgen_pruefer_tree):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _take_csr(lib, rc, n, rp, ci, nnz):
    if rc != 0:
        raise RuntimeError(f"sgcgen: generator failed with code {rc}")
    try:
        row_ptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
        col_idx = np.ctypeslib.as_array(ci, shape=(max(int(nnz.value), 1),))[: int(nnz.value)].copy()
    finally:
        lib.sgcgen_free(ctypes.cast(rp, ctypes.c_void_p))
        lib.sgcgen_free(ctypes.cast(ci, ctypes.c_void_p))
    return row_ptr.astype(np.int32), col_idx.astype(np.int32)


def _thr(p: float) -> int:
    return min(int(round(p * 4294967296.0)), 4294967296)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1):
    """R-MAT graph with 2**scale vertices as (row_ptr, col_idx) int32 arrays."""
    lib = _load()
    rp = ctypes.POINTER(ctypes.c_int32)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64(0)
    rc = lib.sgcgen_rmat(scale, edge_factor, _thr(a), _thr(a + b), _thr(a + b + c), seed,
                         ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nnz))
    return _take_csr(lib, rc, 1 << scale, rp, ci, nnz)


def er(n: int, m: int, seed: int = 1):
    """Erdos-Renyi G(n, m) as (row_ptr, col_idx) int32 arrays."""
    lib = _load()
    rp = ctypes.POINTER(ctypes.c_int32)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64(0)
    rc = lib.sgcgen_er(n, m, seed, ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nnz))
    return _take_csr(lib, rc, n, rp, ci, nnz)


def from_edges(n: int, edges) -> tuple:
    """Symmetric CSR of an undirected edge list (self-loops and repeats dropped)."""
    lib = _load()
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    eu = np.ascontiguousarray(e[:, 0])
    ev = np.ascontiguousarray(e[:, 1])
    rp = ctypes.POINTER(ctypes.c_int32)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64(0)
    i32p = ctypes.POINTER(ctypes.c_int32)
    rc = lib.sgcgen_from_edges(n, len(e), eu.ctypes.data_as(i32p), ev.ctypes.data_as(i32p),
                               ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nnz))
    return _take_csr(lib, rc, n, rp, ci, nnz)


def complete_graph(n: int):
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def tree_graph(parent) -> tuple:
    """The template tree itself as a host graph (CSR over its k vertices)."""
    parent = list(parent)
    return from_edges(len(parent), [(i, p) for i, p in enumerate(parent) if p >= 0])


def pruefer_tree(k: int, seed: int) -> np.ndarray:
    """Uniform labelled tree on k vertices (Pruefer sequence), parent array rooted at 0."""
    lib = _load()
    out = np.zeros(k, dtype=np.int32)
    rc = lib.sgcgen_pruefer_tree(k, seed, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise RuntimeError(f"sgcgen: pruefer_tree failed with code {rc}")
    return out


def path_tree(k: int) -> np.ndarray:
    """Path 0-1-...-(k-1) rooted at vertex 0."""
    return np.array([-1] + list(range(k - 1)), dtype=np.int32)


def star_tree(k: int) -> np.ndarray:
    """Star K_{1,k-1} with centre 0."""
    return np.array([-1] + [0] * (k - 1), dtype=np.int32)


def spider_tree(legs) -> np.ndarray:
    """Centre 0 with legs of the given lengths; leg vertices are numbered consecutively."""
    parent = [-1]
    for length in legs:
        prev = 0
        for _ in range(length):
            parent.append(prev)
            prev = len(parent) - 1
    return np.array(parent, dtype=np.int32)


def splitmix64_draw(seed: int, j: int) -> int:
    """j-th SplitMix64 output of the stream keyed by ``seed`` (input-side copy)."""
    return int(_load().sgcgen_splitmix64_draw(seed, j))


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: exponential gaps from SplitMix64 draws."""
    lib = _load()
    u = np.array([(lib.sgcgen_splitmix64_draw(seed, j) >> 11) for j in range(count)], dtype=np.float64)
    u = (u + 0.5) / float(1 << 53)
    return np.cumsum(-np.log(u) / rate_per_s)


def uniform_ints(lo: int, hi: int, count: int, seed: int) -> np.ndarray:
    """count integers uniform in [lo, hi] from SplitMix64 draws."""
    lib = _load()
    span = hi - lo + 1
    return np.array([lo + (((lib.sgcgen_splitmix64_draw(seed, j) >> 32) * span) >> 32)
                     for j in range(count)], dtype=np.int64)
