"""Write the exact colorful maps of the 12-vertex path and the 13- and 15-vertex Pruefer trees
(seeds 7 and 9) on reduced-scale R-MAT graphs, for the GPU parity tests of those templates.

Calls only the CPU oracle (``oracle/``) and the seeded input generators (``sgcgen/``): the graph is
R-MAT with edge factor 16, a=.57 b=.19 c=.19, seed 1, the templates and colorings are the
benchmark's (k = |T| colors, coloring seeds 1..4).  Exact counts of the 15-vertex tree pass 2^128
from scale 16 on; the oracle then recomputes them with 192-bit counts.

    python tests/golden/make_c3_golden.py 16 > tests/golden/c3_rmat16.json
"""
from __future__ import annotations

import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import oracle  # noqa: E402
import sgcgen  # noqa: E402

TEMPLATES = [("path12", ("path", 12)), ("pruefer13", ("pruefer", 13, 7)), ("pruefer15", ("pruefer", 15, 9))]
SEEDS = [1, 2, 3, 4]


def parent_of(spec):
    return sgcgen.path_tree(spec[1]) if spec[0] == "path" else sgcgen.pruefer_tree(spec[1], spec[2])


def main():
    scale = int(sys.argv[1])
    names = sys.argv[2:] or [n for n, _ in TEMPLATES]
    rp, ci = sgcgen.rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1)
    n = len(rp) - 1
    out = {"graph": {"kind": "rmat", "scale": scale, "edge_factor": 16, "a": 0.57, "b": 0.19, "c": 0.19,
                     "seed": 1, "n": n, "nnz": int(len(ci))},
           "seeds": SEEDS, "templates": {}}
    for name, spec in TEMPLATES:
        if name not in names:
            continue
        parent = parent_of(spec)
        k = len(parent)
        rows = []
        for s in SEEDS:
            t0 = time.perf_counter()
            r = oracle.count(rp, ci, parent, oracle.colors(s, n, k))
            rows.append({"seed": s, "maps": str(r.maps), "max_intermediate": str(r.max_intermediate),
                         "oracle_s": round(time.perf_counter() - t0, 2)})
            print(f"{name} seed {s}: {r.maps.bit_length()} bits, {rows[-1]['oracle_s']} s", file=sys.stderr)
        out["templates"][name] = {"spec": list(spec), "k": k, "aut": oracle.automorphisms(parent), "results": rows}
    json.dump(out, sys.stdout, indent=1)
    print()


if __name__ == "__main__":
    main()
