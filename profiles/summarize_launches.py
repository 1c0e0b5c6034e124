"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel.

    python profiles/summarize_launches.py <launches.csv>

Prints launches, total device time and share per kernel (template arguments
kept), sorted by time.  ncu serialises launches and runs them cold, so the
shares - not the absolute times - are what compare with bench.py.
"""
import collections
import csv
import re
import sys


def main(path):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ki, mi, vi, ui = (h.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        m = re.search(r"(k_\w+)(<[^()]*>)?", r[ki])
        key = (m.group(1) + (m.group(2) or "")) if m else r[ki][:60]
        v = float(r[vi].replace(",", ""))
        scale = {"nsecond": 1e-6, "ns": 1e-6, "usecond": 1e-3, "us": 1e-3, "msecond": 1.0, "ms": 1.0}.get(r[ui], 1e-6)
        agg[key][0] += 1
        agg[key][1] += v * scale
    tot = sum(v[1] for v in agg.values())
    print(f"{'kernel':48s} {'launches':>8s} {'total ms':>10s} {'share':>7s} {'avg ms':>9s}")
    for k, (n, ms) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"{k:48s} {n:8d} {ms:10.2f} {100 * ms / tot:6.1f}% {ms / n:9.3f}")
    print(f"{'total':48s} {sum(v[0] for v in agg.values()):8d} {tot:10.2f}")


if __name__ == "__main__":
    main(sys.argv[1])
