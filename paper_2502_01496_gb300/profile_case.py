"""Builds and force evaluations of a seeded workload, for profilers (a small
case of the benchmark's workload, a centrally condensed Plummer sphere, or
the batch of 256 Plummer systems as one forest: the first evaluation runs
eagerly, later ones replay its captured graph).

  python -m paper_2502_01496_gb300.profile_case [--workload binary|plummer|batch]
      [--n-per-star 262144] [--n 1048576] [--theta 0.5] [--n-leaf 16]
      [--precision mixed|fp64] [--evals 1]
"""
from __future__ import annotations

import argparse


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["binary", "plummer", "batch"], default="binary")
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
    prec = native.MIXED if args.precision == "mixed" else native.FP64
    if args.workload == "batch":
        import numpy as np
        B = W.plummer_batch(256)
        off = np.concatenate([[0], np.cumsum([p.n for p in B.systems])]).astype(np.int64)
        n = int(off[-1])
        x = torch.tensor(np.concatenate([p.x for p in B.systems]), device="cuda")
        m = torch.tensor(np.concatenate([p.m for p in B.systems]), device="cuda")
        a = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        phi = torch.empty(n, dtype=torch.float64, device="cuda")
        f = native.KdFmm(theta=0.5, eps=0.01, n_leaf=args.n_leaf, soft_kind=0, precision=prec)
        nl = np.full(len(B.systems), args.n_leaf, dtype=np.int32)
        for _ in range(args.evals):
            native.fmm_accel_batched(f.handle, x, m, None, off, f.params, a, phi, theta=B.theta,
                                     eps=B.eps, n_leaf=nl)
        torch.cuda.synchronize()
        print(f.stats())
        return
    if args.workload == "binary":
        ps = W.polytrope_binary(args.n_per_star, W.seed_for(1))
    else:
        ps = W.plummer(args.n, W.seed_for(4))
    x = torch.tensor(ps.x, device="cuda")
    m = torch.tensor(ps.m, device="cuda")
    h = None if ps.h is None else torch.tensor(ps.h, device="cuda")
    f = native.KdFmm(theta=args.theta, eps=ps.eps, n_leaf=args.n_leaf, soft_kind=ps.soft_kind,
                     precision=prec)
    for _ in range(args.evals):
        f.build(x, m, h)
        f.accel()
    torch.cuda.synchronize()
    print(f.stats())


if __name__ == "__main__":
    main()
