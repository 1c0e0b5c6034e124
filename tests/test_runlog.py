"""Checkpoint / resume of counting runs (host logic, no GPU): a run interrupted
after some chunks and resumed from its log returns the same maps as an
uninterrupted run, counts every seed exactly once, and rejects another run's log."""
import json

import numpy as np
import pytest

import oracle
import sgcgen
from paper_1903_04395_gb300 import runlog


class Crash(Exception):
    pass


def make_counter(rp, ci, parent, calls, crash_after=None):
    n = len(rp) - 1

    def count(seeds):
        if crash_after is not None and len(calls) >= crash_after:
            raise Crash()
        calls.append([int(s) for s in seeds])
        return [oracle.count(rp, ci, parent, oracle.colors(int(s), n, len(parent))).maps for s in seeds]
    return count


def test_resume_after_interruption(tmp_path):
    rp, ci = sgcgen.er(300, 900, 4)
    parent = sgcgen.pruefer_tree(5, 1005)
    seeds = list(range(1000, 1037))
    key = "er300/pruefer5"
    calls_a = []
    full = runlog.count_resumable(make_counter(rp, ci, parent, calls_a), seeds,
                                  runlog.RunLog(str(tmp_path / "a.jsonl"), key), chunk=8)
    path = str(tmp_path / "b.jsonl")
    calls_b = []
    with pytest.raises(Crash):
        runlog.count_resumable(make_counter(rp, ci, parent, calls_b, crash_after=3), seeds,
                               runlog.RunLog(path, key), chunk=8)
    assert len(calls_b) == 3
    # a line cut short by the crash is ignored
    with open(path, "a") as f:
        f.write('{"run": "er300/pru')
    calls_c = []
    resumed = runlog.count_resumable(make_counter(rp, ci, parent, calls_c), seeds, runlog.RunLog(path, key), chunk=8)
    assert np.array_equal(resumed, full)
    counted = sorted(s for c in calls_b + calls_c for s in c)
    assert counted == seeds  # every seed exactly once
    # the records appended after the torn line survive a reload
    again = runlog.RunLog(path, key)
    assert again.missing(seeds) == [] and np.array_equal(again.maps(seeds), full)


def test_log_of_another_run_rejected(tmp_path):
    path = tmp_path / "c.jsonl"
    path.write_text(json.dumps({"run": "other", "seeds": [1], "maps": [2.0]}) + "\n")
    with pytest.raises(ValueError):
        runlog.RunLog(str(path), "mine")
