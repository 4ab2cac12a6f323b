"""One build and one force evaluation of a seeded binary polytrope, for
profilers (a small case of the benchmark's workload).

  python -m paper_2502_01496_gb300.profile_case [--n-per-star 262144] [--theta 0.5]
      [--n-leaf 16] [--precision mixed|fp64]
"""
from __future__ import annotations

import argparse


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-per-star", type=int, default=1 << 18)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--n-leaf", type=int, default=16)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    args = ap.parse_args()
    import torch
    from . import native
    from . import workloads as W
    ps = W.polytrope_binary(args.n_per_star, W.seed_for(1))
    x = torch.tensor(ps.x, device="cuda")
    m = torch.tensor(ps.m, device="cuda")
    h = torch.tensor(ps.h, device="cuda")
    f = native.KdFmm(theta=args.theta, eps=ps.eps, n_leaf=args.n_leaf, soft_kind=ps.soft_kind,
                     precision=native.MIXED if args.precision == "mixed" else native.FP64)
    f.build(x, m, h)
    f.accel()
    torch.cuda.synchronize()
    print(f.stats())


if __name__ == "__main__":
    main()
