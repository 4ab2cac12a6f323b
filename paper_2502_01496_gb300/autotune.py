"""Autotuner for forests of independent systems: leaf size per (theta, N) bin
and the walk's hand-over budget.

The leaf size n_leaf trades the walk and the M2L (more, smaller leaves: more
cells to visit and more far cells per leaf) against the P2P (fewer, larger
leaves: more particle pairs inside the near lists).  The best value depends
on the opening parameter theta (a small theta opens more cells, Eq. 4) and on
the system size, and -- because every phase processes all systems of a forest
in the same launches, sharing the GPU and its L2 -- on the rest of the batch.
The walk budget (cells one walk thread visits before its leaf goes to the
block-wide walk, which decides the leaf's system in tiles of 1024 cells)
sets which leaves are walked by a thread and which by a whole block.

So the tuner works in place, on the batch it is tuning for: systems are
grouped into (theta, N) bins; starting from the defaults, one pass of
coordinate descent (largest bin first) times the whole forest for each
candidate leaf size of one bin, then each candidate walk budget, and keeps a
change only when it beats the incumbent by more than `min_gain` (timing
noise); a last pair of timings keeps the defaults if the tuned setting is
not faster.  The result is a table that maps bins to leaf sizes plus the walk
budget; `choose` looks systems up in it.

Usage (on the GPU):  python -m paper_2502_01496_gb300.autotune [--out FILE]
(tunes on a seeded 256-system Plummer batch and writes the table).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE_PATH = os.path.join(HERE, "tuned_leaf_sizes.json")

THETA_EDGES = (0.0, 0.4, 0.55, 0.7, 0.85, 1.0)
N_EDGES = (1, 8192, 65536, 1 << 30)
CANDIDATES = (8, 12, 16, 20, 24, 32)
DEFAULT_LEAF = 16
BUDGETS = (1024, 2048, 4096, 8192)
DEFAULT_BUDGET = 0          # the library's default (4096)


def _bin(value, edges) -> int:
    for k in range(len(edges) - 1):
        if value < edges[k + 1]:
            return k
    return len(edges) - 2


def choose(sizes, thetas, table: dict | None = None) -> np.ndarray:
    """Leaf size of each system from the tuned table (DEFAULT_LEAF for bins
    the table lacks)."""
    if table is None:
        table = load()
    leaf = np.full(len(sizes), DEFAULT_LEAF, dtype=np.int32)
    if not table:
        return leaf
    te, ne = table.get("theta_edges", THETA_EDGES), table.get("n_edges", N_EDGES)
    best = table.get("best", {})
    for k, (n, th) in enumerate(zip(sizes, thetas)):
        key = f"{_bin(float(th), te)},{_bin(int(n), ne)}"
        if key in best:
            leaf[k] = int(best[key])
    return leaf


def load(path: str = TABLE_PATH) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def _time_forest(native, torch, f, x, m, off, thetas, nl, budget, a, flush, reps):
    native.tree_set_walk_budget(f.handle, budget)
    native.fmm_accel_batched(f.handle, x, m, None, off, f.params, a, None, theta=thetas,
                             n_leaf=nl)
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        native.fmm_accel_batched(f.handle, x, m, None, off, f.params, a, None, theta=thetas,
                                 n_leaf=nl)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune(systems=None, thetas=None, reps: int = 3, precision: int = 1, log=print,
         min_gain: float = 0.005, handle=None) -> dict:
    """Tunes leaf sizes per (theta, N) bin and the walk budget in place on a
    batch (default: 256 Plummer systems, N log-uniform in [2048, 262144],
    theta uniform in [0.3, 1], eps 0.01).  `handle` (a native.KdFmm) may be
    the one the batch will run on, so its buffers and graph are reused."""
    import torch
    from . import native
    from . import workloads as W
    t_start = time.perf_counter()
    if systems is None:
        B = W.plummer_batch(256, config_index=103)
        systems, thetas = B.systems, B.theta
    sizes = np.array([p.n for p in systems])
    thetas = np.asarray(thetas, dtype=np.float64)
    x = torch.tensor(np.concatenate([p.x for p in systems]), device="cuda")
    m = torch.tensor(np.concatenate([p.m for p in systems]), device="cuda")
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    a = torch.empty((int(off[-1]), 3), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    f = handle or native.KdFmm(theta=0.5, eps=0.01, n_leaf=DEFAULT_LEAF, soft_kind=0,
                               precision=precision)
    keys = np.array([f"{_bin(float(th), THETA_EDGES)},{_bin(int(n), N_EDGES)}"
                     for n, th in zip(sizes, thetas)])
    order = sorted(set(keys), key=lambda k: -int(sizes[keys == k].sum()))
    best = {k: DEFAULT_LEAF for k in order}
    nl = np.full(len(sizes), DEFAULT_LEAF, dtype=np.int32)
    budget = DEFAULT_BUDGET
    run = lambda n_leaf, b: _time_forest(native, torch, f, x, m, off, thetas, n_leaf, b, a,
                                         flush, reps)
    cur = base = run(nl, budget)
    log(f"defaults (n_leaf {DEFAULT_LEAF}, library walk budget): {base:.2f} ms "
        f"({int(off[-1])} particles)")
    times = {}
    for key in order:
        sel = keys == key
        row = {str(DEFAULT_LEAF): round(cur, 3)}
        for cand in CANDIDATES:
            if cand == best[key]:
                continue
            trial = nl.copy()
            trial[sel] = cand
            t = run(trial, budget)
            row[str(cand)] = round(t, 3)
            if t < cur * (1.0 - min_gain):
                cur, nl, best[key] = t, trial, cand
        times[key] = row
        log(f"bin {key} ({int(sel.sum())} systems, {int(sizes[sel].sum())} particles): "
            f"n_leaf {best[key]}  {row}")
    budget_ms = {}
    for b in BUDGETS:
        t = run(nl, b)
        budget_ms[str(b)] = round(t, 3)
        if t < cur * (1.0 - min_gain):
            cur, budget = t, b
    log(f"walk budget {budget or 'default'}  {budget_ms}")
    final = run(nl, budget)
    default = run(np.full(len(sizes), DEFAULT_LEAF, dtype=np.int32), DEFAULT_BUDGET)
    if final >= default:
        best = {k: DEFAULT_LEAF for k in order}
        budget = DEFAULT_BUDGET
        log(f"tuned {final:.2f} ms is not faster than the defaults {default:.2f} ms: keeping them")
        final = default
    log(f"tuned: {final:.2f} ms (defaults {default:.2f} ms)")
    native.tree_set_walk_budget(f.handle, DEFAULT_BUDGET)
    props = torch.cuda.get_device_properties(0)
    return {"theta_edges": list(THETA_EDGES), "n_edges": list(N_EDGES),
            "candidates": list(CANDIDATES), "best": best, "walk_budget": int(budget),
            "ms": times, "budget_ms": budget_ms,
            "ms_default": round(default, 3), "ms_tuned": round(final, 3),
            "tuning_s": round(time.perf_counter() - t_start, 1), "device": props.name,
            "precision": "mixed" if precision == 1 else "fp64",
            "tuned_at": time.strftime("%Y-%m-%d %H:%M:%S")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE_PATH)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    table = tune(reps=args.reps)
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1)
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
