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
# FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


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
    """Oracle (single thread) on this workload: full tree build, forces of a
    random sample of leaves until the budget is spent, extrapolated to all
    leaves.  Returns (Mparticles/s, sample description)."""
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
    done, npart, t_eval, k = 0, 0, 0.0, 0
    while t_eval < budget_s and k < len(order):
        batch = order[k:k + 16]
        t1 = time.perf_counter()
        T.eval(leaves=np.sort(batch))
        t_eval += time.perf_counter() - t1
        npart += int(c.count[batch].sum())
        done += len(batch)
        k += len(batch)
    t_total = t_build + t_eval * len(leaves) / done
    desc = (f"oracle tree build of all {ps.n} particles ({t_build:.2f} s) + forces of {done} of "
            f"{len(leaves)} leaves ({npart} particles, {t_eval:.2f} s), extrapolated to all leaves")
    return ps.n / t_total / 1e6, desc, t_total


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ps, cfg = workload(args)
    per_step = max(1.0, min(6.0, 120.0 / max(1, args.steps + args.warmup)))
    rates = []
    for k in range(args.warmup + args.steps):
        r, _, _ = oracle_rate_cached(ps, args, per_step, k)
        if k >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ps.n / value / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
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
    done, npart, t_eval, k = 0, 0, 0.0, 0
    while t_eval < budget_s and k < len(order):
        batch = order[k:k + 16]
        t1 = time.perf_counter()
        T.eval(leaves=np.sort(batch))
        t_eval += time.perf_counter() - t1
        npart += int(c.count[batch].sum())
        done += len(batch)
        k += len(batch)
    t_total = t_build + t_eval * len(leaves) / done
    _REF_DESC["desc"] = (f"per step: forces of {done} random leaves of {len(leaves)} ({npart} "
                         f"particles) timed and extrapolated to all leaves, plus the oracle's tree "
                         f"build of all {ps.n} particles ({t_build:.2f} s)")
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


def run_batched(args, dev, flush):
    """The batch of 256 independent Plummer systems (N log-uniform in
    [2048, 262144], theta uniform in [0.3, 1], eps 0.01, mixed precision) as one
    forest per step: build + walk + M2L + P2P of all systems in shared launches,
    leaf sizes from the autotuned table (and, for comparison, 16 everywhere)."""
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
    table = autotune.load()
    out = {"workload": "plummer_batch_256", "n": n, "n_sys": 256, "unit": UNIT,
           "tuned_table": bool(table)}
    for label, nl in (("tuned", autotune.choose(sizes, B.theta, table)),
                      ("leaf16", np.full(256, 16, dtype=np.int32))):
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
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic_for(kernel_key),
                "kernel": kernel_key, "flops_per_launch": flops,
                "flops_per_interaction": P2P_FLOPS_PER_INTERACTION[ps.soft_kind],
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "launch_ms": p2p_mean}
    phase_mean = {k: statistics.mean(p[k] for p in phases) for k in phases[0]}

    # the plain FP64 GPU path on the same workload (the metric's comparison)
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        g = native.KdFmm(theta=args.theta, eps=ps.eps, r_kern=2.0, n_leaf=args.n_leaf,
                         soft_kind=ps.soft_kind, precision=native.FP64)
        g.build(x, m, h)
        g.accel(a, phi)
        native.total_momentum(m, a, F)
        torch.cuda.synchronize()
        t64 = []
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
        ms64 = statistics.mean(t64)
        fp64 = {"value": n / (ms64 / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms64,
                "steps": args.fp64_steps}
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
               "d2h_bytes_per_step": int(n * 24 + 24), "ms_per_step": ems / args.steps}

    batched = None
    if args.batched_steps > 0:
        batched = run_batched(args, dev, flush)
    variants = None
    if args.variant_steps > 0:
        variants = run_variants(args, ps, x, m, h, flush)
    large = None
    if args.large_steps > 0 and rank == 0 and world == 1:
        large = run_large(args, dev, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, desc, _ = oracle_rate(ps, args, args.cpu_budget_s)
        cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}

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
