"""Summaries of ncu output for the profiles kept with the repository.

    python -m paper_1903_04395_gb300.ncu_summary launches <launches.csv>
        per kernel (template arguments kept): launches, total device time, share
        and mean time, from a `--metrics gpu__time_duration.sum --csv` launch list.
        ncu serialises launches and runs them cold: compare shares, not times.
    python -m paper_1903_04395_gb300.ncu_summary report <capture.ncu-rep> ...
        the memory, occupancy and stall counters of each captured launch, read with
        `ncu -i <capture> --page raw --csv`.
"""
from __future__ import annotations

import collections
import csv
import re
import subprocess
import sys

REPORT_METRICS = [
    "gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
    "dram__throughput.avg.pct_of_peak_sustained_elapsed", "lts__t_sector_hit_rate.pct",
    "l1tex__t_sector_hit_rate.pct", "l1tex__throughput.avg.pct_of_peak_sustained_active",
    "l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum", "lts__throughput.avg.pct_of_peak_sustained_elapsed",
    "sm__throughput.avg.pct_of_peak_sustained_elapsed", "sm__warps_active.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active",
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "launch__registers_per_thread",
    "launch__occupancy_limit_registers", "launch__occupancy_limit_shared_mem", "launch__occupancy_limit_warps",
    "launch__grid_size", "launch__block_size", "launch__shared_mem_per_block_dynamic",
]


_TIME_MS = {"nsecond": 1e-6, "ns": 1e-6, "usecond": 1e-3, "us": 1e-3, "msecond": 1.0, "ms": 1.0}
_BYTES = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}


def launch_table(path: str) -> dict:
    """Per kernel (name with template arguments): launches, total ms and, when the capture has them,
    total DRAM bytes read and written."""
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ki, mi, vi, ui = (h.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    agg = collections.defaultdict(lambda: {"launches": 0, "ms": 0.0, "read": 0.0, "write": 0.0})
    for r in rows[hi + 1:]:
        if len(r) <= vi:
            continue
        m = re.search(r"(k_\w+)(<[^()]*>)?", r[ki])
        key = (m.group(1) + (m.group(2) or "")) if m else r[ki][:60]
        v = float(r[vi].replace(",", ""))
        if r[mi] == "gpu__time_duration.sum":
            agg[key]["launches"] += 1
            agg[key]["ms"] += v * _TIME_MS.get(r[ui], 1e-6)
        elif r[mi] == "dram__bytes_read.sum":
            agg[key]["read"] += v * _BYTES.get(r[ui], 1.0)
        elif r[mi] == "dram__bytes_write.sum":
            agg[key]["write"] += v * _BYTES.get(r[ui], 1.0)
    return dict(agg)


def launches(path: str) -> None:
    agg = launch_table(path)
    tot = sum(v["ms"] for v in agg.values())
    dram = any(v["read"] or v["write"] for v in agg.values())
    head = f"{'kernel':48s} {'launches':>8s} {'total ms':>10s} {'share':>7s} {'avg ms':>9s}"
    print(head + (f" {'read GB':>9s} {'write GB':>9s} {'GB/s':>8s}" if dram else ""))
    for k, v in sorted(agg.items(), key=lambda x: -x[1]["ms"]):
        n, ms = v["launches"], v["ms"]
        line = f"{k:48s} {n:8d} {ms:10.2f} {100 * ms / tot:6.1f}% {ms / n:9.3f}"
        if dram:  # per launch, and their sum over the launch's time
            line += f" {v['read'] / n / 1e9:9.3f} {v['write'] / n / 1e9:9.3f} {(v['read'] + v['write']) / ms / 1e6:8.0f}"
        print(line)
    print(f"{'total':48s} {sum(v['launches'] for v in agg.values()):8d} {tot:10.2f}")


def report(paths) -> None:
    for path in paths:
        out = subprocess.run(["ncu", "-i", path, "--page", "raw", "--csv"], capture_output=True, text=True).stdout
        rows = list(csv.reader(out.splitlines()))
        h, units = rows[0], rows[1]
        for vals in rows[2:]:
            print("==", path, vals[h.index("Kernel Name")][:90])
            for i, name in enumerate(h):
                stall = name.startswith("smsp__average_warps_issue_stalled") and name.endswith("per_issue_active.ratio")
                if name not in REPORT_METRICS and not stall:
                    continue
                try:
                    v = float(vals[i].replace(",", ""))
                except ValueError:
                    continue
                if stall and v < 0.3:
                    continue
                print(f"  {name:75s} {units[i]:10s} {vals[i]}")


if __name__ == "__main__":
    if len(sys.argv) < 3 or sys.argv[1] not in ("launches", "report"):
        sys.exit(__doc__)
    launches(sys.argv[2]) if sys.argv[1] == "launches" else report(sys.argv[2:])
