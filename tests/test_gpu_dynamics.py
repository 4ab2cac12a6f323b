"""Leapfrog dynamics and the differentiable force: the kick/drift kernel, the
centre-of-mass drift and total force of a leapfrog run against the same
integrator driven by the oracle, and gradients through a checkpointed
leapfrog against finite differences."""
import math

import numpy as np
import pytest

from paper_2502_01496_gb300 import workloads as W

from gpu_common import fsum_force

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


def _cuda(a):
    import torch
    return None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")


def test_kick_drift_matches_host_arithmetic():
    import torch
    from paper_2502_01496_gb300 import native
    rng = np.random.default_rng(1)
    n = 10007
    x, v, a = (rng.standard_normal((n, 3)) for _ in range(3))
    xd, vd, ad = _cuda(x), _cuda(v), _cuda(a)
    native.kick_drift(xd, vd, ad, 0.0005, 0.001)
    native.kick_drift(xd, vd, ad, 0.0005, 0.0)
    torch.cuda.synchronize()
    v1 = v + 0.0005 * a                 # numpy: one rounding per operation, as the kernel
    x1 = x + 0.001 * v1
    v2 = v1 + 0.0005 * a
    assert np.array_equal(xd.cpu().numpy(), x1)
    assert np.array_equal(vd.cpu().numpy(), v2)


def test_leapfrog_drift_matches_oracle(oracle):
    """A polytrope binary on circular orbits (8192 particles, M4 softening,
    theta 0.5, FP64), 20 KDK steps of 1e-3: the GPU run's total force
    sum m a and centre of mass at every step against the same integrator
    whose forces come from the oracle (Sec. 4: the force does not vanish
    and the centre of mass drifts)."""
    import torch
    from paper_2502_01496_gb300 import dynamics
    ps = W.polytrope_binary(4096, W.seed_for(1, 50))
    v0 = W.binary_velocities(ps)
    steps, dt = 20, 1e-3
    params = dict(theta=0.5, eps=ps.eps, n_leaf=16, soft_kind=1, precision=FP64)
    x, v = _cuda(ps.x), _cuda(v0)
    rec = dynamics.integrate(x, v, _cuda(ps.m), _cuda(ps.h), steps=steps, dt=dt, **params)
    torch.cuda.synchronize()

    def force(xx):
        T = oracle.Tree(xx, ps.m, ps.h, theta=0.5, n_leaf=16, soft_kind=1, eps=ps.eps)
        a, _ = T.eval()
        return a

    xo, vo = ps.x.copy(), v0.copy()
    ao = force(xo)
    M = math.fsum(ps.m)
    F_o = [fsum_force(ps.m, ao)]
    com_o = [np.array([math.fsum(ps.m * xo[:, k]) for k in range(3)]) / M]
    for _ in range(steps):
        vo = vo + (0.5 * dt) * ao
        xo = xo + dt * vo
        ao = force(xo)
        vo = vo + (0.5 * dt) * ao
        F_o.append(fsum_force(ps.m, ao))
        com_o.append(np.array([math.fsum(ps.m * xo[:, k]) for k in range(3)]) / M)
    F_o, com_o = np.array(F_o), np.array(com_o)
    # the force sum is far from rounding level: the method's non-conservation
    scale = np.abs(ps.m[:, None] * ao).sum(axis=0).max()
    assert np.linalg.norm(F_o, axis=1).min() > 1e-9 * scale
    errF = np.linalg.norm(rec["F"] - F_o, axis=1) / np.linalg.norm(F_o, axis=1)
    assert errF.max() < 1e-3, errF
    drift_g = rec["com"] - rec["com"][0]
    drift_o = com_o - com_o[0]
    errc = np.linalg.norm(drift_g[-1] - drift_o[-1]) / np.linalg.norm(drift_o[-1])
    assert errc < 1e-3, (drift_g[-1], drift_o[-1])
    assert np.abs(x.cpu().numpy() - xo).max() < 1e-9


def test_autograd_function_is_the_adjoint():
    import torch
    from paper_2502_01496_gb300 import dynamics, native
    ps = W.plummer(3000, W.seed_for(4, 1))
    params = dict(theta=0.5, eps=ps.eps, n_leaf=16, soft_kind=0, precision=FP64)
    x = _cuda(ps.x).requires_grad_(True)
    m = _cuda(ps.m).requires_grad_(True)
    a = dynamics.fmm_accel(x, m, **params)
    ab = torch.randn_like(a)
    (a * ab).sum().backward()
    f = native.KdFmm(**params)
    f.build(_cuda(ps.x), _cuda(ps.m))
    a2, _ = f.accel()
    xb, mb = f.vjp(ab)
    torch.cuda.synchronize()
    assert torch.equal(a.detach(), a2)
    assert torch.allclose(x.grad, xb, rtol=1e-12, atol=1e-12 * float(xb.abs().max()))
    assert torch.allclose(m.grad, mb, rtol=1e-12, atol=1e-12 * float(mb.abs().max()))


def test_checkpointed_leapfrog_gradient():
    """Gradient of L = sum w . x_T (and of the centre-of-mass displacement)
    with respect to x0 through 6 KDK steps: checkpointed equals stored, and
    both match central differences of the full dynamics (trees rebuilt every
    step; the step is small enough that no tree decision flips)."""
    import torch
    from paper_2502_01496_gb300 import dynamics
    ps = W.plummer(512, W.seed_for(4, 2))
    v0 = W.plummer_velocities(ps.x, W.seed_for(4, 3))
    params = dict(theta=0.5, eps=ps.eps, n_leaf=8, soft_kind=0, precision=FP64)
    steps, dt = 6, 1e-3
    m = _cuda(ps.m)
    rng = np.random.default_rng(8)
    wgt = _cuda(rng.standard_normal((ps.n, 3)))

    def loss(x0, every):
        xT, _, _ = dynamics.leapfrog(x0, _cuda(v0), m, steps=steps, dt=dt, checkpoint_every=every,
                                     **params)
        return (wgt * xT).sum()

    grads = []
    for every in (0, 2):
        x0 = _cuda(ps.x).requires_grad_(True)
        loss(x0, every).backward()
        grads.append(x0.grad.detach().cpu().numpy())
    g0, g2 = grads
    assert np.abs(g0 - g2).max() <= 1e-12 * np.abs(g0).max()

    with torch.no_grad():
        for _ in range(3):
            d = rng.standard_normal((ps.n, 3))
            hs = 1e-7
            lp = float(loss(_cuda(ps.x + hs * d), 0))
            lm = float(loss(_cuda(ps.x - hs * d), 0))
            fd = (lp - lm) / (2 * hs)
            ad = float(np.sum(g0 * d))
            assert abs(fd - ad) <= 1e-6 * np.linalg.norm(g0) * np.linalg.norm(d), (fd, ad)

    # the drift's sensitivity: gradient of w . (COM_T - COM_0) exists and is finite
    x0 = _cuda(ps.x).requires_grad_(True)
    xT, _, _ = dynamics.leapfrog(x0, _cuda(v0), m, steps=steps, dt=dt, checkpoint_every=3, **params)
    w = torch.tensor([0.6, 0.0, 0.8], dtype=torch.float64, device="cuda")
    (w * (dynamics.centre_of_mass(xT, m) - dynamics.centre_of_mass(x0, m))).sum().backward()
    assert torch.isfinite(x0.grad).all()


@pytest.mark.slow
def test_vjp_million_plummer_mixed_against_fp64_differences():
    """The differentiation workload: 2^20 Plummer particles, mixed forward and
    adjoint under a seeded Gaussian cotangent, against Richardson central
    differences (step 1e-4) of the FP64 evaluation on the same lists
    (kdfmm_tree_moments), along three random directions: within 1e-4."""
    import torch
    from paper_2502_01496_gb300 import native
    ps = W.plummer(1 << 20, W.seed_for(4))
    rng = np.random.default_rng(W.seed_for(4, 7))
    ab = _cuda(rng.standard_normal((ps.n, 3)))
    x, m = _cuda(ps.x), _cuda(ps.m)
    fm = native.KdFmm(theta=0.5, eps=ps.eps, n_leaf=16, soft_kind=0, precision=MIXED)
    fm.build(x, m)
    fm.accel()
    xb, mb = fm.vjp(ab)
    f64 = native.KdFmm(theta=0.5, eps=ps.eps, n_leaf=16, soft_kind=0, precision=FP64)
    f64.build(x, m)
    f64.accel()

    def L(xx, mm):
        f64.moments(xx, mm)
        a, _ = f64.accel(want_phi=False)
        return float((a * ab).sum())

    for _ in range(3):
        d = _cuda(rng.standard_normal((ps.n, 3)))
        dm = _cuda(rng.standard_normal(ps.n) * ps.m)

        def D(s):
            return (L(x + s * d, m + s * dm) - L(x - s * d, m - s * dm)) / (2 * s)

        fd = (4 * D(0.5e-4) - D(1e-4)) / 3
        ad = float((xb * d).sum() + (mb * dm).sum())
        scale = float(xb.norm() * d.norm() + mb.norm() * dm.norm())
        assert abs(fd - ad) <= 1e-4 * scale, (fd, ad, scale)
