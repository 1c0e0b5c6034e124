"""TEST INFRASTRUCTURE ONLY: the exact CPU oracle for color-coding tree counting.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it (``sgc_oracle.c`` is its own implementation of the
paper's Section 2.1 color coding, Eq. 1 index, Eq. 2 pruning and the
pre-computed neighbour traversal of Section 4.2).

Counts are exact unsigned integers, 128 bits wide; a count that needs more
is recomputed by the same source compiled with 192-bit limbs
(``-DORACLE_WIDE``), and only past 192 bits is an overflow reported (never
wrapped).  Python receives them as ``int``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libsgc_oracle.so")
_WIDE_PATH = os.path.join(_HERE, "libsgc_oracle_wide.so")
_lock = threading.Lock()
_lib = None
_wide = None

OK, OVERFLOW, EINVAL, ENOMEM = 0, 1, -1, -2


class OracleOverflow(ArithmeticError):
    """A count exceeded the build's range (2**128 - 1, or 2**192 - 1 for the wide build)."""


def _build_one(path: str, extra, force: bool) -> str:
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC", *extra, "-o", tmp, _SRC])
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile ``libsgc_oracle.so`` (128-bit counts) and ``libsgc_oracle_wide.so`` (192-bit counts)
    in place (gcc -O2 -fopenmp)."""
    _build_one(_WIDE_PATH, ["-DORACLE_WIDE"], force)
    return _build_one(_LIB_PATH, [], force)


def _load(wide: bool = False):
    global _lib, _wide
    with _lock:
        if (_wide if wide else _lib) is None:
            build()
            lib = ctypes.CDLL(_WIDE_PATH if wide else _LIB_PATH)
            P = ctypes.POINTER
            lib.oracle_color.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_uint8)]
            lib.oracle_count.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int32,
                                         P(ctypes.c_int32), P(ctypes.c_uint8), ctypes.c_int32, ctypes.c_int32,
                                         P(ctypes.c_uint64), P(ctypes.c_uint64), P(ctypes.c_uint64)]
            lib.oracle_count_colors.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32),
                                                ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32),
                                                P(ctypes.c_uint8), ctypes.c_int32, ctypes.c_int32,
                                                P(ctypes.c_uint64), P(ctypes.c_uint64), P(ctypes.c_uint64)]
            lib.oracle_automorphisms.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_uint64)]
            lib.oracle_colorset_index.argtypes = [P(ctypes.c_int32), ctypes.c_int32]
            lib.oracle_colorset_index.restype = ctypes.c_int64
            lib.oracle_colorset_unindex.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                    P(ctypes.c_int32)]
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            for f in (lib.oracle_color, lib.oracle_count, lib.oracle_count_colors, lib.oracle_automorphisms,
                      lib.oracle_colorset_unindex, lib.oracle_threads, lib.oracle_words, lib.oracle_set_threads):
                f.restype = ctypes.c_int
            if wide:
                _wide = lib
            else:
                _lib = lib
    return _wide if wide else _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _check(rc):
    if rc == OVERFLOW:
        raise OracleOverflow("oracle: a count exceeded the build's unsigned integer range")
    if rc == EINVAL:
        raise ValueError("oracle: invalid argument")
    if rc == ENOMEM:
        raise MemoryError("oracle: out of host memory")
    if rc != OK:
        raise RuntimeError(f"oracle: error {rc}")


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> int:
    """Use n OpenMP threads in later calls (both builds); returns the previous count."""
    _load(True).oracle_set_threads(int(n))
    return int(_load().oracle_set_threads(int(n)))


def colors(seed: int, n: int, k: int) -> np.ndarray:
    """Counter-based coloring: SplitMix64 draw v of stream ``seed``, hi32 scaled to [0, k)."""
    out = np.empty(max(n, 1), dtype=np.uint8)
    _check(_load().oracle_color(seed, n, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return out[:n]


def colorset_index(cols) -> int:
    """Eq. 1 index of an ascending color list."""
    a, p = _i32(cols)
    return int(_load().oracle_colorset_index(p, len(a)))


def colorset_unindex(idx: int, h: int, k: int) -> list:
    out = np.zeros(max(h, 1), dtype=np.int32)
    _check(_load().oracle_colorset_unindex(idx, h, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return [int(x) for x in out[:h]]


@dataclass
class CountResult:
    maps: int               # colorful injective maps T -> G  (sum_v N(v, T, all colors))
    max_intermediate: int   # largest value in any table, buffer or the final sum
    per_vertex: list | None = None


def _words(x, w) -> int:
    return sum(int(x[i]) << (64 * i) for i in range(w))


def count(row_ptr, col_idx, parent, cols, mode: str = "pruned", root: int | None = None,
          per_vertex: bool = False, ncolors: int | None = None, wide: bool | None = None) -> CountResult:
    """Exact colorful maps of tree ``parent`` in graph (row_ptr, col_idx) under coloring ``cols``
    (colors in [0, ncolors), ncolors >= |T|, default |T|: Section 2.1 allows k >= |T| colors).
    wide=None: 128-bit counts, recomputed with 192-bit counts when they overflow; True / False
    forces one build."""
    if wide is None:
        try:
            return count(row_ptr, col_idx, parent, cols, mode, root, per_vertex, ncolors, wide=False)
        except OracleOverflow:
            return count(row_ptr, col_idx, parent, cols, mode, root, per_vertex, ncolors, wide=True)
    lib = _load(wide)
    w = int(lib.oracle_words())
    rp, rpp = _i32(row_ptr)
    ci, cip = _i32(col_idx if len(col_idx) else np.zeros(1, np.int32))
    par, parp = _i32(parent)
    col = np.ascontiguousarray(cols, dtype=np.uint8)
    colp = (col if len(col) else np.zeros(1, np.uint8)).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    n = len(rp) - 1
    maps = (ctypes.c_uint64 * w)()
    mx = (ctypes.c_uint64 * w)()
    pv = np.zeros((max(n, 1), w), dtype=np.uint64) if per_vertex else None
    pvp = pv.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if per_vertex else None
    rc = lib.oracle_count_colors(n, rpp, cip, len(par), len(par) if ncolors is None else int(ncolors), parp, colp,
                                 {"pruned": 0, "literal": 1}[mode], -1 if root is None else int(root), maps, mx, pvp)
    _check(rc)
    res = CountResult(maps=_words(maps, w), max_intermediate=_words(mx, w))
    if per_vertex:
        res.per_vertex = [_words(row, w) for row in pv[:n]]
    return res


def automorphisms(parent) -> int:
    """|Aut(T)| as the colorful maps of T into itself under the identity coloring."""
    par, parp = _i32(parent)
    out = ctypes.c_uint64(0)
    _check(_load().oracle_automorphisms(len(par), parp, ctypes.byref(out)))
    return int(out.value)


@dataclass
class Estimate:
    seeds: list
    maps: list          # per coloring
    copies: list        # maps / |Aut(T)| per coloring (exact)
    estimates: list     # copies * k^k / k!  per coloring (float)
    mean: float         # mean of the per-coloring estimates
    aut: int
    max_intermediate: int


def colorful_probability(t: int, k: int) -> Fraction:
    """Probability that t vertices get t distinct colors out of k uniform ones: k! / ((k - t)! k^t)."""
    return Fraction(math.factorial(k), math.factorial(k - t) * k ** t)


def estimate(row_ptr, col_idx, parent, seeds, mode: str = "pruned", ncolors: int | None = None) -> Estimate:
    """Per-coloring colorful counts and the color-coding estimate copies / P(colorful), averaged
    (k^k / k! * copies for k = |T| colors, Section 2.1)."""
    t = len(parent)
    k = t if ncolors is None else int(ncolors)
    n = len(row_ptr) - 1
    aut = automorphisms(parent)
    scale = 1 / colorful_probability(t, k)
    maps, copies, ests = [], [], []
    mx = 0
    for s in seeds:
        r = count(row_ptr, col_idx, parent, colors(int(s), n, k), mode=mode, ncolors=k)
        if r.maps % aut != 0:
            raise ArithmeticError("oracle: maps not divisible by |Aut(T)|")
        maps.append(r.maps)
        copies.append(r.maps // aut)
        ests.append(float(copies[-1] * scale))
        mx = max(mx, r.max_intermediate)
    mean = float(sum(Fraction(c) for c in copies) * scale / len(seeds)) if seeds else 0.0
    return Estimate(list(seeds), maps, copies, ests, mean, aut, mx)
