"""Checkpoint and resume of long counting runs.

Colorings are independent iterations of the estimator (Section 2.1), so the
whole state of a run is the list of (seed, colorful maps) pairs counted so
far: no table is ever checkpointed.  A RunLog appends one JSON line per
counted chunk (flushed and fsynced before the next chunk starts); a resumed
run reads the lines back and counts only the seeds that are missing.
"""
from __future__ import annotations

import json
import os

import numpy as np


class RunLog:
    """Append-only log of counted colorings for one (graph, template, options) run."""

    def __init__(self, path: str, run_key: str):
        self.path = path
        self.run_key = run_key
        self.done: dict[int, float] = {}
        if os.path.exists(path):
            with open(path) as f:
                for line in f:
                    line = line.strip()
                    if not line:
                        continue
                    try:
                        rec = json.loads(line)
                    except json.JSONDecodeError:
                        continue  # a line cut short by a crash: its chunk is counted again
                    if rec.get("run") != run_key:
                        raise ValueError(f"{path} belongs to run {rec.get('run')!r}, not {run_key!r}")
                    for s, m in zip(rec["seeds"], rec["maps"]):
                        self.done[int(s)] = float(m)

    def missing(self, seeds) -> list[int]:
        return [int(s) for s in seeds if int(s) not in self.done]

    def record(self, seeds, maps) -> None:
        rec = {"run": self.run_key, "seeds": [int(s) for s in seeds], "maps": [float(m) for m in maps]}
        torn = False
        if os.path.exists(self.path) and os.path.getsize(self.path) > 0:
            with open(self.path, "rb") as f:
                f.seek(-1, os.SEEK_END)
                torn = f.read(1) != b"\n"
        with open(self.path, "a") as f:
            f.write(("\n" if torn else "") + json.dumps(rec) + "\n")
            f.flush()
            os.fsync(f.fileno())
        for s, m in zip(rec["seeds"], rec["maps"]):
            self.done[s] = m

    def maps(self, seeds) -> np.ndarray:
        return np.array([self.done[int(s)] for s in seeds], dtype=np.float64)


def count_resumable(count_fn, seeds, log: RunLog, chunk: int = 64) -> np.ndarray:
    """Count the colorings of `seeds` with count_fn(seed_array) -> maps, chunk by chunk, skipping the
    seeds the log already holds; returns the maps of all seeds in seed order."""
    todo = log.missing(seeds)
    for i in range(0, len(todo), chunk):
        part = np.asarray(todo[i:i + chunk], dtype=np.uint64)
        log.record(part, count_fn(part))
    return log.maps(seeds)


def run_key(graph_stats: dict, parent, options: dict) -> str:
    """A key naming a run: graph size and degree summary, template, options."""
    g = {k: graph_stats[k] for k in ("n", "n_active", "nnz", "max_degree")}
    return json.dumps({"graph": g, "parent": [int(x) for x in parent], "options": options}, sort_keys=True)
