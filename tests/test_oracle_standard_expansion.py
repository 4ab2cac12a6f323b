"""Pins of the oracle's standard p = 3 Cartesian expansion (the multipole
section's series with p = 3 and no octupole: sink and source orders add up to
at most p - 1 for the acceleration).  It differs from Eq. 6's expansion only
in the quadrupole's higher sink orders, so it must agree with it where those
vanish, keep the third-order error decay, conserve momentum for mutually
interacting cells, and -- the paper's claim -- still leave a non-zero total
force under the leaf-only walk."""
import math

import numpy as np

from paper_2502_01496_gb300 import workloads as W

STD, PH = 1, 0


def _cluster(rng, n, centre, scale):
    return rng.normal(0.0, scale, (n, 3)) + centre, rng.uniform(0.5, 1.5, n)


def _fsum3(m, a):
    return np.array([math.fsum(m * a[:, k]) for k in range(3)])


def test_standard_equals_eq6_without_quadrupole(oracle):
    """A single-particle source has Q = 0: only the monopole remains, which
    both expansions keep to every order."""
    r = np.array([1.3, -0.4, 0.9])
    for Q in (np.zeros(6),):
        p0, a0 = oracle.m2l(r, 2.5, Q, PH)
        p1, a1 = oracle.m2l(r, 2.5, Q, STD)
        assert np.array_equal(p0, p1) and np.array_equal(a0, a1)


def test_standard_equals_eq6_at_the_sink_centre(oracle):
    """At x = 0 only order-0 acceleration (and order <= 1 potential) terms
    survive, where both keep the quadrupole; the higher orders differ."""
    rng = np.random.default_rng(21)
    y, mb = _cluster(rng, 30, np.zeros(3), 0.2)
    M, com, Q, _ = oracle.moments(y, mb)
    r = np.array([1.7, -0.9, 0.6])
    p0, a0 = oracle.m2l(r, M, Q, PH)
    p1, a1 = oracle.m2l(r, M, Q, STD)
    ac0, ph0 = oracle.l2p(p0, a0, np.zeros(3))
    ac1, ph1 = oracle.l2p(p1, a1, np.zeros(3))
    assert np.allclose(ac0, ac1, rtol=1e-15, atol=0) and abs(ph0 - ph1) <= 1e-15 * abs(ph0)
    diff = np.abs(a0 - a1).max(axis=0)
    assert diff[0] <= 1e-15 * np.abs(a0).max()
    assert diff[1:10].max() > 1e-6 * np.abs(a0).max()        # gradient / Hessian terms differ


def test_standard_cluster_pair_error_decays_as_third_power(oracle):
    rng = np.random.default_rng(22)
    ys, ms = _cluster(rng, 40, np.zeros(3), 0.05)
    xs, mt = _cluster(rng, 10, np.zeros(3), 0.05)
    M, com_b, Q, _ = oracle.moments(ys, ms)
    _, com_a0, _, _ = oracle.moments(xs, mt)
    direction = np.array([0.6, -0.64, 0.48])
    errs, dists = [], [1.0, 2.0, 4.0, 8.0]
    for dist in dists:
        shift = direction * dist
        r = com_a0 + shift - com_b
        pot, acc = oracle.m2l(r, M, Q, STD)
        e = []
        for xi in xs:
            a, _ = oracle.l2p(pot, acc, xi - com_a0)
            d = xi + shift - ys
            ex = -(ms[:, None] * d / np.linalg.norm(d, axis=1)[:, None] ** 3).sum(0)
            e.append(np.linalg.norm(a - ex) / np.linalg.norm(ex))
        errs.append(max(e))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(dists))
    assert np.all(slopes < -2.6) and np.all(slopes > -3.6), slopes


def test_standard_mutual_pair_conserves_momentum(oracle):
    """Truncating by the combined order is symmetric in sink and source, so two
    cells that interact both ways exert equal and opposite total forces."""
    rng = np.random.default_rng(23)
    xa, ma = _cluster(rng, 12, np.array([0.0, 0.0, 0.0]), 0.08)
    xb, mb = _cluster(rng, 17, np.array([1.3, -0.7, 0.4]), 0.1)
    Ma, ca, Qa, _ = oracle.moments(xa, ma)
    Mb, cb, Qb, _ = oracle.moments(xb, mb)
    potA, accA = oracle.m2l(ca - cb, Mb, Qb, STD)
    potB, accB = oracle.m2l(cb - ca, Ma, Qa, STD)
    FA = sum(mi * oracle.l2p(potA, accA, xi - ca)[0] for xi, mi in zip(xa, ma))
    FB = sum(mj * oracle.l2p(potB, accB, xj - cb)[0] for xj, mj in zip(xb, mb))
    assert np.linalg.norm(FA + FB) < 1e-13 * np.linalg.norm(FA)


def test_standard_expansion_leaf_only_walk_total_force_nonzero(oracle):
    """The paper's claim for the standard series: with the leaf-only walk the
    total force still does not vanish (the walk, not the expansion, breaks
    the symmetry); and the two expansions leave different total forces."""
    ps = W.plummer(4096, W.seed_for(0))
    T = oracle.Tree(ps.x, ps.m, theta=0.5, n_leaf=16, eps=ps.eps, expansion=STD)
    a, _ = T.eval()
    T0 = oracle.Tree(ps.x, ps.m, theta=0.5, n_leaf=16, eps=ps.eps, expansion=PH)
    a0, _ = T0.eval()
    scale = math.fsum(ps.m * np.linalg.norm(a, axis=1))
    F, F0 = _fsum3(ps.m, a), _fsum3(ps.m, a0)
    assert np.linalg.norm(F) > 1e-6 * scale
    assert np.linalg.norm(F - F0) > 1e-3 * np.linalg.norm(F0)
    # the expansions differ by far less than either differs from the direct sum
    ad, _ = oracle.direct(ps.x, ps.m, eps=ps.eps)
    err_std = np.linalg.norm(a - ad, axis=1).max()
    err_ph = np.linalg.norm(a0 - ad, axis=1).max()
    assert err_std < 10 * err_ph and err_ph < 10 * err_std
