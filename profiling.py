"""Summaries of Nsight Compute output for the profiles/ notes.

    python profiling.py launches <launches.csv>
    python profiling.py raw <report.ncu-rep>

``launches``: per kernel name, the number of launches, total device time and
share of the listed time (from a ``--metrics gpu__time_duration.sum --csv``
capture; per-launch times there are cold-cache and serialised, so only the
shares are comparable with a live run). ``raw``: the DRAM, occupancy and stall
counters of each captured launch (``ncu -i <rep> --page raw --csv``).
"""
from __future__ import annotations

import csv
import io
import re
import subprocess
import sys
from collections import defaultdict

RAW_METRICS = [
    "gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
    "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "dram__cycles_active.avg.pct_of_peak_sustained_elapsed",
    "sm__warps_active.avg.pct_of_peak_sustained_active", "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "launch__registers_per_thread", "launch__shared_mem_per_block_dynamic", "launch__grid_size",
    "launch__block_size", "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio",
    "smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio",
    "smsp__inst_executed.sum", "lts__t_sector_hit_rate.pct", "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active",
]


def _short(name: str) -> str:
    name = re.sub(r"^void ", "", name)
    name = re.sub(r"\(.*$", "", name)
    return name.replace("<unnamed>::", "")


def summarize_launches(path: str) -> str:
    text = open(path).read()
    start = text.find('"ID"')
    rows = list(csv.DictReader(io.StringIO(text[start:])))
    per = defaultdict(lambda: [0, 0.0])
    for r in rows:
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        v = float(r["Metric Value"].replace(",", ""))
        unit = r.get("Metric Unit", "")
        scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}
        us = v * scale.get(unit, 1.0)
        k = _short(r["Kernel Name"])
        per[k][0] += 1
        per[k][1] += us
    total = sum(t for _, t in per.values()) or 1.0
    out = [f"{'kernel':70s} {'launches':>8s} {'total us':>12s} {'share':>7s}"]
    for k, (n, t) in sorted(per.items(), key=lambda kv: -kv[1][1]):
        out.append(f"{k[:70]:70s} {n:8d} {t:12.1f} {100 * t / total:6.1f}%")
    return "\n".join(out)


def summarize_raw(rep: str) -> str:
    csv_text = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True,
                              text=True, check=True).stdout
    rows = list(csv.reader(io.StringIO(csv_text)))
    hdr, units = rows[0], rows[1]
    out = []
    for r in rows[2:]:
        out.append(f"launch: {_short(r[hdr.index('Kernel Name')])}")
        for m in RAW_METRICS:
            if m in hdr:
                i = hdr.index(m)
                out.append(f"  {m:80s} {r[i]} {units[i]}")
    return "\n".join(out)


if __name__ == "__main__":
    mode, path = sys.argv[1], sys.argv[2]
    print(summarize_launches(path) if mode == "launches" else summarize_raw(path))
