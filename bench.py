#!/usr/bin/env python
"""Benchmark of one kd-tree FMM force evaluation (tree build + moments + walk +
M2L + L2P + P2P + assembly + total momentum) on a GB300.

Default workload: two n = 1 polytropes of 2^20 equal-mass particles each
(radius 1, separation 4), M4 kernel softening with h = 1.2 (m/rho)^(1/3),
theta = 0.5, leaves of at most 16 particles, mixed precision.  Prints one JSON
line.  `--impl reference` times the CPU oracle on a bounded sample instead.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one independent replica per GPU (the evaluation of one
particle set does not shard: no collective in the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mparticles/s per FMM force eval at θ=0.5: FP32-mixed vs FP64 GPU, same accuracy"
UNIT = "Mparticles/s"
# P2P floating-point work per particle-particle interaction (algorithmic count,
# Newtonian part: 3 sub, r^2 with 2 FMA + 1 mul + 1 add, rsqrt, 3 mul, 3 FMA,
# potential add; FMA = 2 flops); the M4 kernel softening adds 10 per interaction
P2P_FLOPS_PER_INTERACTION = {0: 20, 1: 30}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-per-star", type=int, default=1 << 20)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--n-leaf", type=int, default=16)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=12.0)
    ap.add_argument("--batched-steps", type=int, default=5,
                    help="steps of the 256-system batch (0 skips it)")
    ap.add_argument("--variant-steps", type=int, default=5,
                    help="steps of the dual-walk and standard-expansion variants (0 skips them)")
    ap.add_argument("--large-steps", type=int, default=3,
                    help="steps of the 2^24-particle uniform + clumps evaluation (0 skips it)")
    return ap.parse_args()


def workload(args):
    from paper_2502_01496_gb300 import workloads as W
    ps = W.polytrope_binary(args.n_per_star, W.seed_for(1))
    cfg = {
        "workload": f"binary_polytrope_2x{args.n_per_star}",
        "n": ps.n,
        "theta": args.theta,
        "n_leaf": args.n_leaf,
        "softening": "M4 cubic spline, R_kern=2, h=1.2*(m/rho)^(1/3)",
        "precision": args.precision,
        "l2": "flushed between timed steps (512 MiB write, outside the timed events)",
        "step": "tree_build + fmm_accel + total_momentum",
    }
    return ps, cfg


# ---------------------------------------------------------------------------
# reference arm and CPU baseline: the oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_rate(ps, args, budget_s, rng_seed=0):
    """The oracle on this workload, as it stands: full tree build (one thread),
    then forces of a random sample of leaves until the budget is spent,
    extrapolated to all leaves -- once on one thread and once with the leaves
    spread over every host core (OpenMP, same results bit for bit).  Returns
    the two baselines and the sampled leaves' forces (caller order, NaN
    outside the sample)."""
    import numpy as np
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    T = oracle.Tree(ps.x, ps.m, ps.h, theta=args.theta, n_leaf=args.n_leaf,
                    soft_kind=ps.soft_kind, eps=ps.eps)
    t_build = time.perf_counter() - t0
    c = T.cells()
    leaves = np.nonzero(c.is_leaf)[0]
    rng = np.random.default_rng(rng_seed)
    order = rng.permutation(leaves)
    a_s = np.full((ps.n, 3), np.nan)
    phi_s = np.full(ps.n, np.nan)
    out = {}
    k = 0
    for label, threads in (("single", 1), ("all_cores", oracle.max_threads())):
        done, npart, t_eval = 0, 0, 0.0
        batch_n = 16 * threads
        while t_eval < budget_s / 2 and k < len(order):
            batch = np.sort(order[k:k + batch_n])
            t1 = time.perf_counter()
            a, phi = T.eval_threads(leaves=batch, nthreads=threads)
            t_eval += time.perf_counter() - t1
            rows = ~np.isnan(phi)
            a_s[rows], phi_s[rows] = a[rows], phi[rows]
            npart += int(c.count[batch].sum())
            done += len(batch)
            k += len(batch)
        t_total = t_build + t_eval * len(leaves) / max(done, 1)
        out[label] = {
            "value": ps.n / t_total / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"oracle tree build of all {ps.n} particles ({t_build:.2f} s, one thread) + "
                       f"forces of {done} random leaves of {len(leaves)} ({npart} particles, "
                       f"{t_eval:.2f} s on {threads} thread(s)), extrapolated to all leaves")}
    return out, a_s, phi_s


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    ps, cfg = workload(args)
    per_step = max(1.0, min(6.0, 120.0 / max(1, args.steps + args.warmup)))
    rates = []
    for k in range(args.warmup + args.steps):
        r, _, _ = oracle_rate_cached(ps, args, per_step, k)
        if k >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ps.n / value / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": _REF_DESC.get("desc", "")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


_REF_CACHE = {}
_REF_DESC = {}


def oracle_rate_cached(ps, args, budget_s, seed):
    """Later reference steps reuse the oracle tree (its build time is kept in
    the extrapolation) and time a fresh leaf sample."""
    import numpy as np
    import oracle
    if "T" not in _REF_CACHE:
        t0 = time.perf_counter()
        T = oracle.Tree(ps.x, ps.m, ps.h, theta=args.theta, n_leaf=args.n_leaf,
                        soft_kind=ps.soft_kind, eps=ps.eps)
        _REF_CACHE.update(T=T, t_build=time.perf_counter() - t0, c=T.cells())
    T, t_build, c = _REF_CACHE["T"], _REF_CACHE["t_build"], _REF_CACHE["c"]
    leaves = np.nonzero(c.is_leaf)[0]
    rng = np.random.default_rng(seed)
    order = rng.permutation(leaves)
    threads = oracle.max_threads()
    done, npart, t_eval, k = 0, 0, 0.0, 0
    while t_eval < budget_s and k < len(order):
        batch = order[k:k + 16 * threads]
        t1 = time.perf_counter()
        T.eval_threads(leaves=np.sort(batch), nthreads=threads)
        t_eval += time.perf_counter() - t1
        npart += int(c.count[batch].sum())
        done += len(batch)
        k += len(batch)
    t_total = t_build + t_eval * len(leaves) / done
    _REF_DESC["desc"] = (f"per step: forces of {done} random leaves of {len(leaves)} ({npart} "
                         f"particles) on {threads} host thread(s) (OpenMP over leaves) timed and "
                         f"extrapolated to all leaves, plus the oracle's tree build of all {ps.n} "
                         f"particles ({t_build:.2f} s, one thread)")
    return ps.n / t_total / 1e6, _REF_DESC["desc"], t_total


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def __enter__(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def traffic_for(kernel_key):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_key)
    except Exception:
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2502_01496_gb300", "csrc", rec.get("source", "p2p.cu"))
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if digest != rec.get("source_sha256"):
        return None
    return rec.get("bytes_per_launch_full_size")


def rel_error_summary(a, phi, a_ref, phi_ref) -> dict:
    """Per-particle relative errors |a - a_ref| / |a_ref| and |phi - phi_ref| /
    |phi_ref|: maximum and root mean square."""
    import numpy as np
    na = np.linalg.norm(a_ref, axis=1)
    ea = np.linalg.norm(a - a_ref, axis=1) / na
    ep = np.abs(phi - phi_ref) / np.abs(phi_ref)
    i = int(np.argmax(ea))
    return {"a_max": float(ea.max()), "a_rms": float(np.sqrt(np.mean(ea ** 2))),
            "a_p99999": float(np.quantile(ea, 0.99999)),
            "a_worst_abs_a_over_median": float(na[i] / np.median(na)),
            "a_n_above_2e-5": int(np.count_nonzero(ea > 2e-5)),
            "phi_max": float(ep.max()), "phi_rms": float(np.sqrt(np.mean(ep ** 2)))}


def total_force_summary(m, a_ref, F_mix, F64) -> dict:
    """The method's uncompensated total force sum m a (Sec. 4) of both paths,
    relative to sum m |a|, and the mixed path's deviation from the float64
    one relative to |F_fp64|."""
    import numpy as np
    scale = float(np.sum(m * np.linalg.norm(a_ref, axis=1)))
    return {"mixed": [float(v) for v in F_mix], "fp64_gpu": [float(v) for v in F64],
            "fp64_rel_to_sum_m_abs_a": float(np.linalg.norm(F64) / scale),
            "mixed_minus_fp64_rel": float(np.linalg.norm(F_mix - F64) / np.linalg.norm(F64))}


def reduce_max(value: float, dev, world: int) -> float:
    """Largest value over the ranks (the slowest replica sets the job's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_per_rank: int, steps: int, max_total_ms: float, world: int) -> float:
    """Mparticles/s of the whole job: every rank evaluates its own replica of
    n_per_rank particles per step; the job takes the slowest rank's time."""
    return world * n_per_rank * steps / (max_total_ms / 1e3) / 1e6


def settle():
    """Frees what earlier legs left (handles in reference cycles, cached
    blocks) and waits for the device, so that no deferred free -- a
    synchronising cudaFree of gigabytes -- lands inside a timed region."""
    import gc
    import torch
    gc.collect()
    torch.cuda.synchronize()


def run_batched(args, dev, flush):
    """The batch of 256 independent Plummer systems (N log-uniform in
    [2048, 262144], theta uniform in [0.3, 1], eps 0.01, mixed precision) as one
    forest per step: build + walk + M2L + P2P of all systems in shared launches,
    replayed as one captured CUDA graph.  Before the timed steps the autotuner
    tunes leaf sizes per (theta, N) bin and the walk budget in place on this
    batch (its time is reported, outside the timed region); the defaults (16
    everywhere, library budget) are timed for comparison."""
    settle()
    import numpy as np
    import torch
    from paper_2502_01496_gb300 import autotune, native
    from paper_2502_01496_gb300 import workloads as W
    B = W.plummer_batch(256)
    sizes = np.array([p.n for p in B.systems])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    x = torch.tensor(np.concatenate([p.x for p in B.systems]), device=dev)
    m = torch.tensor(np.concatenate([p.m for p in B.systems]), device=dev)
    a = torch.empty((n, 3), dtype=torch.float64, device=dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    f = native.KdFmm(theta=0.5, eps=0.01, n_leaf=16, soft_kind=0, precision=native.MIXED)
    table = autotune.tune(B.systems, B.theta, reps=2, log=lambda *a: None)
    out = {"workload": "plummer_batch_256", "n": n, "n_sys": 256, "unit": UNIT,
           "tuning": {"in_place": True, "seconds": table["tuning_s"],
                      "walk_budget": table["walk_budget"] or "library default (4096)",
                      "leaf_sizes": table["best"], "ms_default": table["ms_default"],
                      "ms_tuned": table["ms_tuned"]}}
    for label, nl, budget in (("tuned", autotune.choose(sizes, B.theta, table), table["walk_budget"]),
                              ("leaf16", np.full(256, 16, dtype=np.int32), 0)):
        native.tree_set_walk_budget(f.handle, budget)

        def step():
            native.fmm_accel_batched(f.handle, x, m, None, off, f.params, a, phi, theta=B.theta,
                                     eps=B.eps, n_leaf=nl)
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        l0 = f.stats()["launches"]
        ts = []
        for _ in range(args.batched_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        st = f.stats()
        ms = statistics.mean(ts)
        out[label] = {"value": n / (ms / 1e3) / 1e6, "ms_per_step": ms,
                      "launches_per_step": (st["launches"] - l0) / args.batched_steps,
                      "p2p": st["np2p"], "m2l": st["nfar"], "nleaves": st["nleaves"]}
    out["value"] = out["tuned"]["value"]
    return out


def run_large(args, dev, flush):
    """The large single evaluation: 2^24 particles, half uniform in the unit
    cube and half in 64 Gaussian clumps (sigma 0.01), masses log-uniform over a
    decade, eps 1e-3, theta 0.5, leaves of at most 32, mixed precision; the
    same step as the headline (build + evaluation + total momentum)."""
    settle()
    import statistics
    import torch
    from paper_2502_01496_gb300 import native
    from paper_2502_01496_gb300 import workloads as W
    ps = W.uniform_clumps(1 << 24, W.seed_for(2))
    n = ps.n
    x = torch.tensor(ps.x, device=dev)
    m = torch.tensor(ps.m, device=dev)
    a = torch.empty((n, 3), dtype=torch.float64, device=dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    F = torch.empty(3, dtype=torch.float64, device=dev)
    f = native.KdFmm(theta=0.5, eps=ps.eps, n_leaf=32, soft_kind=0, precision=native.MIXED)

    def step():
        f.build(x, m)
        f.accel(a, phi)
        native.total_momentum(m, a, F)

    for _ in range(2):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    native.tree_timing(f.handle, True, read=False)
    ts, phases = [], []
    for _ in range(args.large_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
        phases.append(native.tree_timing(f.handle, True))
    native.tree_timing(f.handle, False, read=False)
    st = f.stats()
    ms = statistics.mean(ts)
    out = {"workload": "uniform_clumps_16777216", "n": n, "theta": 0.5, "n_leaf": 32,
           "precision": "mixed", "unit": UNIT, "value": n / (ms / 1e3) / 1e6, "ms_per_step": ms,
           "steps": args.large_steps,
           "phases_ms": {k: statistics.mean(p[k] for p in phases) for k in phases[0]},
           "p2p": st["np2p"], "m2l": st["nfar"], "nleaves": st["nleaves"], "ncells": st["ncells"]}
    del f, x, m, a, phi
    return out


def run_variants(args, ps, x, m, h, flush):
    """The same workload under the method's variants: the paper's leaf-only walk
    with Eq. 6 (the headline), the symmetric dual-tree walk, and the standard
    p = 3 expansion -- time per evaluation and the relative total force
    |sum m a| / sum m |a| that the leaf-only walk leaves (Sec. 4)."""
    settle()
    import torch
    from paper_2502_01496_gb300 import native
    out = {}
    n = ps.n
    a = torch.empty((n, 3), dtype=torch.float64, device=x.device)
    F = torch.empty(3, dtype=torch.float64, device=x.device)
    prec = native.MIXED if args.precision == "mixed" else native.FP64
    for label, walk, expansion in (("leaf_walk", 0, 0), ("dual_walk", 1, 0),
                                   ("standard_expansion", 0, 1)):
        f = native.KdFmm(theta=args.theta, eps=ps.eps, r_kern=2.0, n_leaf=args.n_leaf,
                         soft_kind=ps.soft_kind, precision=prec, walk=walk, expansion=expansion)
        for _ in range(2):
            f.build(x, m, h)
            f.accel(a, None, want_phi=False)
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.variant_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            f.build(x, m, h)
            f.accel(a, None, want_phi=False)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        native.total_momentum(m, a, F)
        rel = float(torch.linalg.norm(F) / (m * torch.linalg.norm(a, dim=1)).sum())
        st = f.stats()
        ms = statistics.mean(ts)
        out[label] = {"value": n / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_eval": ms,
                      "rel_total_force": rel, "p2p": st["np2p"], "m2l": st["nfar"],
                      "near": st["nnear"]}
        del f
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2502_01496_gb300 import native

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    # roofline denominators of this device: float32 peak derived from its SM
    # count and maximum clock, and float32 / float64 FMA loops measured now
    peaks = native.measure_peaks()
    ps, cfg = workload(args)
    cfg["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"
    n = ps.n
    x = torch.tensor(ps.x, device=dev)
    m = torch.tensor(ps.m, device=dev)
    h = torch.tensor(ps.h, device=dev) if ps.h is not None else None
    prec = native.MIXED if args.precision == "mixed" else native.FP64
    f = native.KdFmm(theta=args.theta, eps=ps.eps, r_kern=2.0, n_leaf=args.n_leaf,
                     soft_kind=ps.soft_kind, precision=prec)
    a = torch.empty((n, 3), dtype=torch.float64, device=dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    F = torch.empty(3, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        f.build(x, m, h)
        f.accel(a, phi)
        native.total_momentum(m, a, F)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    native.tree_timing(f.handle, True, read=False)
    launches0 = f.stats()["launches"]
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    times, p2p_ms, phases = [], [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(str(uuid) if uuid else None) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            ph = native.tree_timing(f.handle, True)
            phases.append(ph)
            p2p_ms.append(ph["p2p"])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    native.tree_timing(f.handle, False, read=False)
    st = f.stats()
    launches = st["launches"] - launches0 + 2 * args.steps      # + the two momentum kernels per step
    total_ms = reduce_max(sum(times), dev, world)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(n, args.steps, total_ms, world)

    # dominant kernel: P2P (+ L2P + assembly), one launch per step
    p2p_mean = statistics.mean(p2p_ms)
    flops = st["np2p"] * P2P_FLOPS_PER_INTERACTION[ps.soft_kind]
    achieved = flops / (p2p_mean / 1e3) / 1e12
    kernel_key = f"k_p2p_{args.precision}_{'m4' if ps.soft_kind == 1 else 'plummer'}"
    peak = peaks["fp32_derived_tflops"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_for(kernel_key),
                "kernel": kernel_key, "flops_per_launch": flops,
                "flops_per_interaction": P2P_FLOPS_PER_INTERACTION[ps.soft_kind],
                "peak_source": (f"derived: {peaks['sms']} SMs x 128 FP32 lanes x 2 flop x "
                                f"{peaks['sm_max_mhz']:.0f} MHz (SM count and clock queried)"),
                "peak_measured": peaks["fp32_tflops"],
                "frac_of_measured": achieved / peaks["fp32_tflops"],
                "peak_measured_source": "FFMA throughput loop in this run (kdfmm_measure_peaks)",
                "launch_ms": p2p_mean}
    phase_mean = {k: statistics.mean(p[k] for p in phases) for k in phases[0]}
    # the mixed result of the last timed step, for the accuracy comparison
    a_mix, phi_mix, F_mix = a.cpu().numpy(), phi.cpu().numpy(), F.cpu().numpy()

    # the plain FP64 GPU path on the same workload (the metric's comparison)
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        g = native.KdFmm(theta=args.theta, eps=ps.eps, r_kern=2.0, n_leaf=args.n_leaf,
                         soft_kind=ps.soft_kind, precision=native.FP64)
        g.build(x, m, h)
        g.accel(a, phi)
        native.total_momentum(m, a, F)
        torch.cuda.synchronize()
        native.tree_timing(g.handle, True, read=False)
        t64, ph64 = [], []
        for _ in range(args.fp64_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.build(x, m, h)
            g.accel(a, phi)
            native.total_momentum(m, a, F)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
            ph64.append(native.tree_timing(g.handle, True))
        native.tree_timing(g.handle, False, read=False)
        ms64 = statistics.mean(t64)
        phases64 = {k: statistics.mean(p[k] for p in ph64) for k in ph64[0]}
        st64 = g.stats()
        ach64 = st64["np2p"] * P2P_FLOPS_PER_INTERACTION[ps.soft_kind] / (phases64["p2p"] / 1e3) / 1e12
        fp64 = {"value": n / (ms64 / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms64,
                "steps": args.fp64_steps, "phases_ms": phases64,
                "p2p_roofline": {"bound": "alu", "achieved": ach64, "unit": "TFLOP/s",
                                 "peak": peaks["fp64_tflops"], "frac": ach64 / peaks["fp64_tflops"],
                                 "peak_source": "DFMA throughput loop in this run (kdfmm_measure_peaks)",
                                 "kernel": f"k_p2p_fp64_{'m4' if ps.soft_kind == 1 else 'plummer'}"}}
        a64, phi64, F64 = a.cpu().numpy(), phi.cpu().numpy(), F.cpu().numpy()
        del g

    # end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        xh = torch.tensor(ps.x).pin_memory()
        mh = torch.tensor(ps.m).pin_memory()
        hh = torch.tensor(ps.h).pin_memory() if ps.h is not None else None
        ah = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        Fh = torch.empty(3, dtype=torch.float64).pin_memory()
        xd, md = torch.empty_like(x), torch.empty_like(m)
        hd = torch.empty_like(h) if h is not None else None

        def e2e_step():
            xd.copy_(xh, non_blocking=True)
            md.copy_(mh, non_blocking=True)
            if hd is not None:
                hd.copy_(hh, non_blocking=True)
            f.build(xd, md, hd)
            f.accel(a, phi)
            native.total_momentum(md, a, F)
            ah.copy_(a, non_blocking=True)
            Fh.copy_(F, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        te = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e2e_step()
            e1.record(stream)
            e1.synchronize()
            te.append(e0.elapsed_time(e1))
        ems = reduce_max(sum(te), dev, world)
        e2e = {"value": whole_job_rate(n, args.steps, ems, world), "unit": UNIT,
               "h2d_bytes_per_step": int(n * (24 + 8 + (8 if h is not None else 0))),
               "d2h_bytes_per_step": int(n * 24 + 24), "ms_per_step": ems / args.steps,
               "path": ("public Python API (native.KdFmm over the C ABI) with torch copies from "
                        "pinned host memory inside the timed events")}

    batched = None
    if args.batched_steps > 0:
        batched = run_batched(args, dev, flush)
    variants = None
    if args.variant_steps > 0:
        variants = run_variants(args, ps, x, m, h, flush)
    large = None
    if args.large_steps > 0 and rank == 0 and world == 1:
        large = run_large(args, dev, flush)

    # accuracy of this run: mixed against the float64 GPU path (every
    # particle) and both against the oracle on the baseline's sampled leaves
    accuracy = None
    if fp64 is not None:
        accuracy = {"mixed_vs_fp64_gpu": rel_error_summary(a_mix, phi_mix, a64, phi64),
                    "total_force": total_force_summary(ps.m, a64, F_mix, F64)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, a_or, phi_or = oracle_rate(ps, args, args.cpu_budget_s)
        cpu = dict(base["all_cores"])
        cpu["single_thread"] = base["single"]
        if accuracy is not None:
            rows = np.nonzero(~np.isnan(phi_or))[0]
            accuracy["vs_oracle_sampled_leaves"] = {
                "particles": int(rows.size),
                "mixed": rel_error_summary(a_mix[rows], phi_mix[rows], a_or[rows], phi_or[rows]),
                "fp64_gpu": rel_error_summary(a64[rows], phi64[rows], a_or[rows], phi_or[rows])}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk.summary(), "gpu_launches": int(launches),
            "fp64_gpu": fp64,
            "mixed_over_fp64": (value / world / fp64["value"]) if fp64 else None,
            "phases_ms": phase_mean,
            "batched": batched,
            "variants": variants,
            "large": large,
            "accuracy": accuracy,
            "peaks": peaks,
            "interactions": {"p2p": st["np2p"], "m2l": st["nfar"], "nleaves": st["nleaves"],
                             "ncells": st["ncells"], "p2p_per_s": st["np2p"] / (ms_per_step / 1e3),
                             "m2l_per_s": st["nfar"] / (ms_per_step / 1e3)},
            "wall_s_timed_region": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
