"""Centre-of-mass drift of the leaf-only kd-tree FMM (Sec. 4).

The walk never forms the interactions "super-cell <- leaf", so the force of
cell A on cell B is not minus the force of B on A and the total force sum m a
does not vanish: the centre of mass of an isolated system drifts.  This
study measures that drift with the GPU path:

* `--study binary`: two n = 1 polytropes on circular orbits (total momentum
  zero, so the exact centre of mass stays put), KDK leapfrog with the tree
  rebuilt every step, for each theta; records |sum m a| / sum m |a| and the
  centre-of-mass displacement per step, and fits r(T) ~ T^p (a force that
  changes at random from step to step makes the centre-of-mass velocity a
  random walk, r ~ T^(3/2)).
* `--study force`: the relative total force |sum m a| / sum m |a| of one
  evaluation against N and theta (polytrope binaries), with the fit
  |sum m a| / sum m |a| ~ c N^(-q).
* `--study gradient`: the drift's sensitivity -- the gradient of
  L = w . (com(T) - com(0)) with respect to the initial positions of a Plummer
  sphere in equilibrium, through a checkpointed leapfrog (the adjoint of
  every force evaluation, trees rebuilt as in the forward run).

Writes one JSON document (stdout, or --out).  Run on the GPU:
  python -m paper_2502_01496_gb300.drift --study binary --n-per-star 1048576
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def _rel_force(m, a) -> float:
    F = np.array([math.fsum(m * a[:, k]) for k in range(3)])
    return float(np.linalg.norm(F) / np.sum(m * np.linalg.norm(a, axis=1)))


def _fit_power(t, y):
    """Least-squares slope and prefactor of log y against log t (y > 0)."""
    sel = (t > 0) & (y > 0)
    if sel.sum() < 3:
        return None, None
    p, c = np.polyfit(np.log(t[sel]), np.log(y[sel]), 1)
    return float(p), float(math.exp(c))


def study_binary(n_per_star: int, thetas, steps: int, dt: float, precision: int, seed_sys: int = 0):
    import torch
    from . import dynamics
    from . import workloads as W
    ps = W.polytrope_binary(n_per_star, W.seed_for(1, seed_sys))
    v0 = W.binary_velocities(ps)
    out = []
    for theta in thetas:
        x = torch.tensor(ps.x, device="cuda")
        v = torch.tensor(v0, device="cuda")
        m = torch.tensor(ps.m, device="cuda")
        h = torch.tensor(ps.h, device="cuda")
        t0 = time.perf_counter()
        rec = dynamics.integrate(x, v, m, h, steps=steps, dt=dt, theta=theta, eps=ps.eps,
                                 n_leaf=16, soft_kind=1, precision=precision)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        M = float(ps.m.sum())
        disp = np.linalg.norm(rec["com"] - rec["com"][0], axis=1)
        Fn = np.linalg.norm(rec["F"], axis=1)
        t = rec["step"] * dt
        p, c = _fit_power(t[1:], disp[1:])
        out.append({
            "theta": theta, "precision": "mixed" if precision == 1 else "fp64",
            "n": ps.n, "steps": steps, "dt": dt, "wall_s": wall,
            "F_over_M_mean": float(Fn.mean() / M), "F_over_M_max": float(Fn.max() / M),
            "com_disp_final": float(disp[-1]), "com_disp_fit_exponent": p,
            "com_disp_fit_prefactor": c,
            "com_disp": disp[:: max(1, steps // 20)].tolist(),
        })
        del x, v, m, h
    return out


def study_force(n_list, thetas, precision: int):
    import torch
    from . import native
    from . import workloads as W
    rows = []
    for n_per in n_list:
        ps = W.polytrope_binary(n_per, W.seed_for(1, 200))
        x = torch.tensor(ps.x, device="cuda")
        m = torch.tensor(ps.m, device="cuda")
        h = torch.tensor(ps.h, device="cuda")
        for theta in thetas:
            f = native.KdFmm(theta=theta, eps=ps.eps, n_leaf=16, soft_kind=1, precision=precision)
            f.build(x, m, h)
            a, _ = f.accel(want_phi=False)
            rows.append({"n": ps.n, "theta": theta,
                         "rel_force": _rel_force(ps.m, a.cpu().numpy())})
    fits = {}
    for theta in thetas:
        ns = np.array([r["n"] for r in rows if r["theta"] == theta], dtype=float)
        ys = np.array([r["rel_force"] for r in rows if r["theta"] == theta])
        q, c = _fit_power(ns, ys)
        fits[str(theta)] = {"exponent": q, "prefactor": c}
    return {"rows": rows, "fits": fits}


def study_gradient(n: int, steps: int, dt: float, every: int, theta: float, precision: int):
    import torch
    from . import dynamics
    from . import workloads as W
    ps = W.plummer(n, W.seed_for(4))
    v0 = W.plummer_velocities(ps.x, W.seed_for(4, 3))
    params = dict(theta=theta, eps=ps.eps, n_leaf=16, soft_kind=0, precision=precision)
    m = torch.tensor(ps.m, device="cuda")
    w = torch.tensor([0.6, 0.0, 0.8], dtype=torch.float64, device="cuda")
    x0 = torch.tensor(ps.x, device="cuda").requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xT, _, _ = dynamics.leapfrog(x0, torch.tensor(v0, device="cuda"), m, steps=steps, dt=dt,
                                 checkpoint_every=every, **params)
    loss = (w * (dynamics.centre_of_mass(xT, m) - dynamics.centre_of_mass(x0, m))).sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = x0.grad
    # the displacement of the centre of mass does not change when every particle
    # is moved by the same vector: the gradient sums to zero (up to rounding)
    return {"n": n, "steps": steps, "dt": dt, "checkpoint_every": every, "theta": theta,
            "precision": "mixed" if precision == 1 else "fp64",
            "loss": float(loss.detach()), "grad_norm": float(g.norm()),
            "grad_max": float(g.abs().max()), "grad_sum": g.sum(0).tolist(),
            "forward_s": t1 - t0, "backward_s": t2 - t1}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--study", choices=["binary", "force", "gradient"], default="binary")
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--checkpoint-every", type=int, default=10)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--n-per-star", type=int, default=1 << 20)
    ap.add_argument("--thetas", default="0.3,0.5,0.7")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--n-list", default="4096,16384,65536,262144,1048576")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    prec = 1 if args.precision == "mixed" else 0
    thetas = [float(t) for t in args.thetas.split(",")]
    if args.study == "binary":
        res = {"study": "binary", "runs": study_binary(args.n_per_star, thetas, args.steps,
                                                       args.dt, prec)}
    elif args.study == "force":
        res = {"study": "force", **study_force([int(v) for v in args.n_list.split(",")], thetas,
                                               prec)}
    else:
        res = {"study": "gradient", **study_gradient(args.n, args.steps, args.dt,
                                                     args.checkpoint_every, args.theta, prec)}
    text = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
