"""Summarises an ncu CSV launch list (gpu__time_duration.sum per launch).

    python -m paper_1911_11906_gb300.ncu_summary launches.csv [more.csv ...]

Prints, per kernel, the number of launches, the total device time and its
share of the listed total, largest first.  ncu serialises launches and runs
them cold, so the shares are what compares with a live run, not the times.
"""
from __future__ import annotations

import csv
import re
import sys
from collections import defaultdict


def _short(name: str) -> str:
    name = re.sub(r"\(.*$", "", name)              # drop the argument list
    name = re.sub(r"^void\s+", "", name)
    name = name.replace("<unnamed>::", "").replace("unnamed>::", "").replace("fraclap::", "")
    return name.strip()


def summarize(paths):
    tot = defaultdict(float)
    cnt = defaultdict(int)
    for path in paths:
        with open(path) as fh:
            lines = [ln for ln in fh if ln.startswith('"')]
        for row in csv.DictReader(lines):
            if row.get("Metric Name") != "gpu__time_duration.sum":
                continue
            k = _short(row["Kernel Name"])
            v = float(row["Metric Value"].replace(",", ""))
            unit = row.get("Metric Unit", "ns")
            scale = {"ns": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "nsecond": 1e-6}.get(unit, 1e-6)
            tot[k] += v * scale
            cnt[k] += 1
    total = sum(tot.values())
    rows = sorted(tot.items(), key=lambda kv: -kv[1])
    out = [f"{'kernel':60s} {'launches':>9s} {'total ms':>12s} {'share':>7s}"]
    for k, v in rows:
        out.append(f"{k[:60]:60s} {cnt[k]:9d} {v:12.3f} {100 * v / total:6.2f}%")
    out.append(f"{'TOTAL':60s} {sum(cnt.values()):9d} {total:12.3f} 100.00%")
    return "\n".join(out)


if __name__ == "__main__":
    print(summarize(sys.argv[1:]))
