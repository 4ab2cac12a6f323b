"""Builds and force evaluations of a seeded workload, for profilers (a small
case of the benchmark's workload, or a centrally condensed Plummer sphere).

  python -m paper_2502_01496_gb300.profile_case [--workload binary|plummer]
      [--n-per-star 262144] [--n 1048576] [--theta 0.5] [--n-leaf 16]
      [--precision mixed|fp64] [--evals 1]
"""
from __future__ import annotations

import argparse


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["binary", "plummer"], default="binary")
    ap.add_argument("--n-per-star", type=int, default=1 << 18, help="binary: particles per star")
    ap.add_argument("--n", type=int, default=1 << 20, help="plummer: particles")
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--n-leaf", type=int, default=16)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--evals", type=int, default=1, help="build + evaluation repetitions")
    args = ap.parse_args()
    import torch
    from . import native
    from . import workloads as W
    if args.workload == "binary":
        ps = W.polytrope_binary(args.n_per_star, W.seed_for(1))
    else:
        ps = W.plummer(args.n, W.seed_for(4))
    x = torch.tensor(ps.x, device="cuda")
    m = torch.tensor(ps.m, device="cuda")
    h = None if ps.h is None else torch.tensor(ps.h, device="cuda")
    f = native.KdFmm(theta=args.theta, eps=ps.eps, n_leaf=args.n_leaf, soft_kind=ps.soft_kind,
                     precision=native.MIXED if args.precision == "mixed" else native.FP64)
    for _ in range(args.evals):
        f.build(x, m, h)
        f.accel()
    torch.cuda.synchronize()
    print(f.stats())


if __name__ == "__main__":
    main()
