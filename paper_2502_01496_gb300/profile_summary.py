"""Summarises an Nsight Compute launch list (``ncu --metrics
gpu__time_duration.sum --csv --log-file ...``) per kernel: launches, total
device time and share.  Usage: python -m paper_2502_01496_gb300.profile_summary
launches.csv [--per-step K]."""
from __future__ import annotations

import collections
import csv
import re
import sys


def summarise(path: str, per_step: int | None = None) -> str:
    rows = [l for l in open(path) if l.startswith('"')]
    recs = list(csv.DictReader(rows))
    tot = collections.OrderedDict()
    for r in recs:
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = re.sub(r"\(.*", "", r["Kernel Name"]).replace("kdfmm::<unnamed>::", "")
        name = name.replace("void ", "").strip()
        t = float(r["Metric Value"])
        n, s = tot.get(name, (0, 0.0))
        tot[name] = (n + 1, s + t)
    grand = sum(s for _, s in tot.values())
    out = [f"{'kernel':40s} {'launches':>8s} {'total_us':>10s} {'share':>7s}"]
    for name, (n, s) in sorted(tot.items(), key=lambda kv: -kv[1][1]):
        out.append(f"{name[:40]:40s} {n:8d} {s / 1e3:10.1f} {100 * s / grand:6.1f}%")
    out.append(f"{'all':40s} {sum(n for n, _ in tot.values()):8d} {grand / 1e3:10.1f} 100.0%")
    if per_step:
        out.append(f"per step (/{per_step}): {grand / 1e3 / per_step:.1f} us")
    return "\n".join(out)


if __name__ == "__main__":
    k = None
    if "--per-step" in sys.argv:
        k = int(sys.argv[sys.argv.index("--per-step") + 1])
    print(summarise(sys.argv[1], k))
