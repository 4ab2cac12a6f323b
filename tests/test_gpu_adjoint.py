"""Frozen-topology moments and the adjoint, through the C ABI, against the oracle.

* kdfmm_tree_moments: after a build and one evaluation at x0, moved particles
  x1 on the same cells and lists.  The refreshed cell table must equal the
  oracle's frozen-topology moments bit for bit (M, centre of mass, s, h_max;
  Q to float64 rounding) and the forces its list-driven evaluation.
* kdfmm_fmm_accel_vjp: x_bar = (da/dx)^T a_bar and m_bar = (da/dm)^T a_bar of
  the evaluation with topology and lists held fixed.  Checked against central
  differences of the oracle's evaluation on the same lists (Richardson
  extrapolated, truncation O(h^4)), along random directions and per element;
  at theta = 0 against differences of the oracle's direct sum.
"""
import numpy as np
import pytest

from paper_2502_01496_gb300 import workloads as W

from gpu_common import assert_lists_bit_exact, oracle_cell_arrays, rel_errors

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


def _cuda(a):
    import torch
    return None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")


def _moved(ps, seed, dx=1e-3):
    rng = np.random.default_rng(seed)
    x1 = ps.x + dx * rng.standard_normal(ps.x.shape)
    m1 = ps.m * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, ps.n))
    return x1, m1


CASES = {
    "plummer_fp64": (lambda: W.plummer(3000, W.seed_for(0, 11)), 0.5, 16, FP64),
    "polytrope_m4_fp64": (lambda: W.polytrope_binary(2000, W.seed_for(0, 12)), 0.5, 16, FP64),
    "polytrope_m4_mixed": (lambda: W.polytrope_binary(2000, W.seed_for(0, 13)), 0.7, 16, MIXED),
    "clumps_leaf32_fp64": (lambda: W.uniform_clumps(2501, W.seed_for(0, 14)), 0.4, 32, FP64),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_frozen_moments_parity(oracle, case):
    import torch
    from paper_2502_01496_gb300 import native
    make, theta, n_leaf, prec = CASES[case]
    ps = make()
    x1, m1 = _moved(ps, 5)
    f = native.KdFmm(theta=theta, eps=ps.eps, n_leaf=n_leaf, soft_kind=ps.soft_kind, precision=prec)
    h = _cuda(ps.h)
    f.build(_cuda(ps.x), _cuda(ps.m), h)
    f.accel()
    f.moments(_cuda(x1), _cuda(m1), h)
    a, phi = f.accel()
    torch.cuda.synchronize()
    ex = f.export(lists=True)
    ga, gphi = a.cpu().numpy(), phi.cpu().numpy()

    T = oracle.Tree(ps.x, ps.m, ps.h, theta=theta, n_leaf=n_leaf, soft_kind=ps.soft_kind, eps=ps.eps)
    L0 = T.walk()
    order0 = T.order()
    T.moments_frozen(x1, m1, ps.h)
    oa, ophi = T.eval_lists(L0)

    # lists and particle order are the ones of the walk at x0
    assert np.array_equal(ex.perm, order0)
    assert_lists_bit_exact({"ex": ex}, {"lists": L0})
    oi, orr = oracle_cell_arrays(T.cells())
    assert np.array_equal(ex.cell_ints, oi)
    np.testing.assert_array_equal(ex.cell_reals[:, :6], orr[:, :6])
    scale = (orr[:, 0] * orr[:, 4] ** 2)[:, None] + 1e-300
    assert (np.abs(ex.cell_reals[:, 6:] - orr[:, 6:]) / scale).max() < 1e-12

    ea, ep = rel_errors(ga, gphi, oa, ophi)
    tol = 1e-12 if prec == FP64 else 2e-5
    assert ea.max() < tol, (case, ea.max())
    assert ep.max() < tol, (case, ep.max())


def test_frozen_moments_requires_evaluation():
    from paper_2502_01496_gb300 import native
    ps = W.plummer(500, W.seed_for(0, 15))
    f = native.KdFmm(theta=0.5, eps=ps.eps, n_leaf=16)
    x, m = _cuda(ps.x), _cuda(ps.m)
    f.build(x, m)
    with pytest.raises(native.KdfmmError):
        f.moments(x, m)
    f.accel()
    f.moments(x, m)
    with pytest.raises(ValueError):
        f.moments(x[:10], m)


def _richardson(L, x, m, dx, dm, hs):
    def D(s):
        return (L(x + s * dx, m + s * dm) - L(x - s * dx, m - s * dm)) / (2.0 * s)
    return (4.0 * D(hs / 2.0) - D(hs)) / 3.0


VJP_CASES = {
    "plummer_fp64": (lambda: W.plummer(1500, W.seed_for(0, 21)), 0.5, 16, FP64, 1e-8),
    "polytrope_m4_fp64": (lambda: W.polytrope_binary(1000, W.seed_for(0, 22)), 0.6, 16, FP64, 1e-8),
    "clumps_leaf32_fp64": (lambda: W.uniform_clumps(1201, W.seed_for(0, 23)), 0.4, 32, FP64, 1e-8),
    "polytrope_m4_mixed": (lambda: W.polytrope_binary(1000, W.seed_for(0, 24)), 0.6, 16, MIXED, 1e-5),
    # near lists of the outskirts' leaves span several P2P segments
    "plummer4096_segments_fp64": (lambda: W.plummer(4096, W.seed_for(0, 25)), 0.5, 16, FP64, 1e-8),
}


@pytest.mark.parametrize("case", sorted(VJP_CASES))
def test_vjp_against_oracle_differences(oracle, case):
    import torch
    from paper_2502_01496_gb300 import native
    make, theta, n_leaf, prec, tol = VJP_CASES[case]
    ps = make()
    n = ps.n
    rng = np.random.default_rng(99)
    ab = rng.standard_normal((n, 3))
    f = native.KdFmm(theta=theta, eps=ps.eps, n_leaf=n_leaf, soft_kind=ps.soft_kind, precision=prec)
    f.build(_cuda(ps.x), _cuda(ps.m), _cuda(ps.h))
    f.accel()
    xb, mb = f.vjp(_cuda(ab))
    torch.cuda.synchronize()
    xb, mb = xb.cpu().numpy(), mb.cpu().numpy()
    assert np.isfinite(xb).all() and np.isfinite(mb).all()
    st = f.stats()
    assert st["nfar"] > 0 and st["nnear"] > 0

    T = oracle.Tree(ps.x, ps.m, ps.h, theta=theta, n_leaf=n_leaf, soft_kind=ps.soft_kind, eps=ps.eps)
    L0 = T.walk()

    def L(x, m):
        T.moments_frozen(x, m, ps.h)
        a, _ = T.eval_lists(L0)
        return float(np.sum(ab * a))

    norm = lambda dx, dm: np.linalg.norm(xb) * np.linalg.norm(dx) + np.linalg.norm(mb) * np.linalg.norm(dm)
    for trial in range(3):
        dx = rng.standard_normal((n, 3))
        dm = rng.standard_normal(n) * ps.m
        fd = _richardson(L, ps.x, ps.m, dx, dm, 3e-5)
        ad = float(np.sum(xb * dx) + np.sum(mb * dm))
        assert abs(fd - ad) <= tol * norm(dx, dm), (case, trial, fd, ad)
    # per element: a few particles, each coordinate and the mass
    scale_x, scale_m = np.abs(xb).max(), np.abs(mb * ps.m).max()
    for i in rng.choice(n, 4, replace=False):
        for d in range(3):
            dx = np.zeros((n, 3))
            dx[i, d] = 1.0
            fd = _richardson(L, ps.x, ps.m, dx, np.zeros(n), 1e-4)
            assert abs(fd - xb[i, d]) <= 10 * tol * scale_x, (case, i, d, fd, xb[i, d])
        dm = np.zeros(n)
        dm[i] = ps.m[i]
        fd = _richardson(L, ps.x, ps.m, np.zeros((n, 3)), dm, 1e-4)
        assert abs(fd - mb[i] * ps.m[i]) <= 10 * tol * scale_m, (case, i, fd, mb[i] * ps.m[i])


@pytest.mark.parametrize("soft", ["plummer", "m4"])
def test_vjp_direct_sum(oracle, soft):
    """theta = 0 opens every cell: the evaluation is the direct sum, whose
    derivative the oracle's direct summation gives by differences."""
    import torch
    from paper_2502_01496_gb300 import native
    ps = W.plummer(700, W.seed_for(0, 31)) if soft == "plummer" else W.polytrope_binary(350, W.seed_for(0, 32))
    n = ps.n
    rng = np.random.default_rng(7)
    ab = rng.standard_normal((n, 3))
    f = native.KdFmm(theta=0.0, eps=ps.eps, n_leaf=16, soft_kind=ps.soft_kind, precision=FP64)
    f.build(_cuda(ps.x), _cuda(ps.m), _cuda(ps.h))
    f.accel()
    assert f.stats()["nfar"] == 0
    xb, mb = f.vjp(_cuda(ab))
    torch.cuda.synchronize()
    xb, mb = xb.cpu().numpy(), mb.cpu().numpy()

    def L(x, m):
        a, _ = oracle.direct(x, m, ps.h, soft_kind=ps.soft_kind, eps=ps.eps)
        return float(np.sum(ab * a))

    for trial in range(3):
        dx = rng.standard_normal((n, 3))
        dm = rng.standard_normal(n) * ps.m
        fd = _richardson(L, ps.x, ps.m, dx, dm, 3e-5)
        ad = float(np.sum(xb * dx) + np.sum(mb * dm))
        scale = np.linalg.norm(xb) * np.linalg.norm(dx) + np.linalg.norm(mb) * np.linalg.norm(dm)
        assert abs(fd - ad) <= 1e-8 * scale, (soft, trial, fd, ad)
    # momentum conservation of the direct sum: sum_i m_i a_i = 0 for all x, so
    # with a_bar_i = m_i c the position cotangent vanishes identically
    c = np.array([0.3, -1.1, 0.7])
    xb2, mb2 = f.vjp(_cuda(ps.m[:, None] * c[None, :]))
    torch.cuda.synchronize()
    assert np.abs(xb2.cpu().numpy()).max() <= 1e-10 * np.abs(xb).max()


def test_vjp_invalid_args():
    import torch
    from paper_2502_01496_gb300 import native
    ps = W.plummer(300, W.seed_for(0, 33))
    f = native.KdFmm(theta=0.5, eps=ps.eps, n_leaf=16)
    f.build(_cuda(ps.x), _cuda(ps.m))
    ab = torch.zeros((ps.n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(native.KdfmmError):
        f.vjp(ab)                       # nothing evaluated yet
    f.accel()
    with pytest.raises(ValueError):
        f.vjp(ab[:5])
    with pytest.raises(TypeError):
        f.vjp(ab.float())


def test_vjp_standard_expansion_against_oracle_differences(oracle):
    """The adjoint of the standard p = 3 series (FP64) against Richardson
    differences of the oracle's standard-series evaluation on frozen lists."""
    import torch
    from paper_2502_01496_gb300 import native
    ps = W.plummer(1200, W.seed_for(0, 25))
    n = ps.n
    rng = np.random.default_rng(5)
    ab = rng.standard_normal((n, 3))
    f = native.KdFmm(theta=0.6, eps=ps.eps, n_leaf=16, soft_kind=0, precision=FP64, expansion=1)
    f.build(_cuda(ps.x), _cuda(ps.m))
    f.accel()
    xb, mb = f.vjp(_cuda(ab))
    torch.cuda.synchronize()
    xb, mb = xb.cpu().numpy(), mb.cpu().numpy()
    T = oracle.Tree(ps.x, ps.m, None, theta=0.6, n_leaf=16, soft_kind=0, eps=ps.eps, expansion=1)
    L0 = T.walk()

    def L(x, m):
        T.moments_frozen(x, m, None)
        a, _ = T.eval_lists(L0)
        return float(np.sum(ab * a))

    for _ in range(3):
        dx = rng.standard_normal((n, 3))
        dm = rng.standard_normal(n) * ps.m
        fd = _richardson(L, ps.x, ps.m, dx, dm, 3e-5)
        ad = float(np.sum(xb * dx) + np.sum(mb * dm))
        scale = np.linalg.norm(xb) * np.linalg.norm(dx) + np.linalg.norm(mb) * np.linalg.norm(dm)
        assert abs(fd - ad) <= 1e-8 * scale, (fd, ad)
