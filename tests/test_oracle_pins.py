"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's formulas: each compares the oracle
with a closed form, an invariant, a limit the paper states, a brute-force
enumeration, numerical quadrature, or values the paper prints.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

from paper_2502_01496_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fsum3(m, a):
    return np.array([math.fsum(m * a[:, k]) for k in range(3)])


def rel_err(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def test_two_body_far_is_unsoftened_point_mass(oracle):
    """n_leaf = 1 and d > 2 eps: each leaf takes the other as a long-range
    partner with s = 0 (Eq. 4 false, Eq. 5 false), so M2L + L2P give the
    unsoftened -m r_hat / d^2 (Eq. 6 with Q = 0, Eq. 8 at x = 0)."""
    x = np.array([[0.1, -0.2, 0.3], [0.9, 0.4, -0.5]])
    m = np.array([0.25, 0.75])
    T = oracle.Tree(x, m, theta=0.5, n_leaf=1, eps=0.01)
    a, phi, parts = T.eval(parts=True)
    d = x[0] - x[1]
    dn = np.linalg.norm(d)
    assert parts["n_p2p"] == 0 and parts["n_m2l"] == 2
    np.testing.assert_allclose(a[0], -m[1] * d / dn ** 3, rtol=1e-14)
    np.testing.assert_allclose(a[1], m[0] * d / dn ** 3, rtol=1e-14)
    np.testing.assert_allclose(phi, [-m[1] / dn, -m[0] / dn], rtol=1e-14)


def test_two_body_near_is_plummer(oracle):
    """d < 2 eps: Eq. 5 opens the partner leaf, the pair is summed directly
    with Plummer softening m d / (d^2 + eps^2)^(3/2)."""
    eps = 0.01
    x = np.array([[0.0, 0.0, 0.0], [0.012, -0.005, 0.003]])
    m = np.array([0.5, 0.5])
    T = oracle.Tree(x, m, theta=0.5, n_leaf=1, eps=eps)
    a, phi, parts = T.eval(parts=True)
    d = x[0] - x[1]
    s2 = d @ d + eps * eps
    assert parts["n_m2l"] == 0 and parts["n_p2p"] == 2
    np.testing.assert_allclose(a[0], -m[1] * d / s2 ** 1.5, rtol=1e-14)
    np.testing.assert_allclose(phi[0], -m[1] / math.sqrt(s2), rtol=1e-14)


def test_single_particle_and_coincident_cut(oracle):
    T = oracle.Tree(np.zeros((1, 3)), np.ones(1), theta=0.5, n_leaf=4, eps=0.01)
    a, phi = T.eval()
    assert T.ncells == 1 and np.all(a == 0.0) and np.all(phi == 0.0)
    # all particles coincident: every cut is degenerate, position split keeps
    # leaves within n_leaf and the walk still terminates
    x = np.zeros((37, 3))
    T = oracle.Tree(x, np.full(37, 1 / 37), theta=0.5, n_leaf=4, eps=0.01)
    c = T.cells()
    assert T.nfallback > 0 and np.all(c.count[c.is_leaf] <= 4)
    a, phi = T.eval()
    assert np.all(a == 0.0)
    np.testing.assert_allclose(phi, -(36 / 37) / 0.01, rtol=1e-13)


# --------------------------------------------------------------------------
# theta -> 0 and the direct sum
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["plummer", "m4"])
def test_theta_zero_is_direct_sum(oracle, kind):
    """Sec. 2: for theta = 0 every cell is opened and a_grav = a_short, i.e.
    the method is the direct sum (equal up to summation order)."""
    if kind == "plummer":
        ps = W.plummer(3000, W.seed_for(0, 1))
    else:
        ps = W.polytrope_binary(1200, W.seed_for(1, 1))
    T = oracle.Tree(ps.x, ps.m, ps.h, theta=0.0, n_leaf=16, soft_kind=ps.soft_kind, eps=ps.eps)
    a, phi, parts = T.eval(parts=True)
    ad, pd = oracle.direct(ps.x, ps.m, ps.h, soft_kind=ps.soft_kind, eps=ps.eps)
    assert parts["n_m2l"] == 0 and parts["n_p2p"] == ps.n * (ps.n - 1)
    assert rel_err(a, ad).max() < 1e-12
    assert (np.abs(phi - pd) / np.abs(pd)).max() < 1e-13
    # the direct sum conserves momentum to rounding, so does theta = 0
    scale = math.fsum(ps.m * np.linalg.norm(ad, axis=1))
    assert np.abs(fsum3(ps.m, a)).max() < 1e-14 * scale


def test_error_shrinks_as_theta_decreases(oracle):
    ps = W.plummer(4096, W.seed_for(0))
    ad, _ = oracle.direct(ps.x, ps.m, eps=ps.eps)
    core = np.linalg.norm(ps.x, axis=1) < 3.0
    med = []
    for th in (0.9, 0.6, 0.4, 0.2, 0.1):
        T = oracle.Tree(ps.x, ps.m, theta=th, n_leaf=16, eps=ps.eps)
        a, _ = T.eval()
        med.append(np.median(rel_err(a, ad)[core]))
    assert all(med[k + 1] < med[k] for k in range(len(med) - 1)), med


# --------------------------------------------------------------------------
# the expansion (Eqs. 6 and 8) and its potential
# --------------------------------------------------------------------------

def _cluster(rng, n, centre, scale):
    return rng.normal(0.0, scale, (n, 3)) + centre, rng.uniform(0.5, 1.5, n)


def test_m2l_jets_match_finite_differences_of_eq6(oracle):
    """The first- and second-order Taylor coefficients used in Eq. 8 equal
    central finite differences of Eq. 6 evaluated with plain doubles."""
    rng = np.random.default_rng(3)
    y, mb = _cluster(rng, 30, np.zeros(3), 0.2)
    M, com, Q, _ = oracle.moments(y, mb)
    r = np.array([1.7, -0.9, 0.6])
    _, acc = oracle.m2l(r, M, Q)
    ex = oracle.monomials()
    idx = {tuple(e): k for k, e in enumerate(ex)}
    np.testing.assert_allclose(acc[:, 0], oracle.acc_node(r, M, Q), rtol=1e-14)
    h = 1e-4
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (oracle.acc_node(r + e, M, Q) - oracle.acc_node(r - e, M, Q)) / (2 * h)
        mono = [0, 0, 0]
        mono[j] = 1
        np.testing.assert_allclose(acc[:, idx[tuple(mono)]], fd, rtol=1e-7, atol=1e-9)
        fd2 = (oracle.acc_node(r + e, M, Q) - 2 * oracle.acc_node(r, M, Q)
               + oracle.acc_node(r - e, M, Q)) / h ** 2
        mono[j] = 2
        np.testing.assert_allclose(2.0 * acc[:, idx[tuple(mono)]], fd2, rtol=1e-5, atol=1e-6)


def test_potential_and_acceleration_expansions_agree(oracle):
    """Two derivations: -grad of the third-order expansion of
    Phi = -M/R - Q_jk R_j R_k / (2 R^5) equals the second-order expansion of
    Eq. 6 coefficient by coefficient."""
    rng = np.random.default_rng(4)
    y, mb = _cluster(rng, 25, np.zeros(3), 0.3)
    M, _, Q, _ = oracle.moments(y, mb)
    r = np.array([-0.8, 2.1, 1.3])
    pot, acc = oracle.m2l(r, M, Q)
    ex = oracle.monomials()
    idx = {tuple(e): k for k, e in enumerate(ex)}
    for k, e in enumerate(ex):
        if e.sum() > 2:
            continue
        for i in range(3):
            up = list(e)
            up[i] += 1
            want = -(e[i] + 1) * pot[idx[tuple(up)]]
            assert abs(acc[i, k] - want) <= 1e-14 * max(1.0, abs(want)) * 10


def test_expansion_is_harmonic(oracle):
    """Outside the source, div a = 0 and the Laplacian of every a_i is 0: the
    traces of the Taylor coefficients vanish to rounding."""
    rng = np.random.default_rng(5)
    y, mb = _cluster(rng, 40, np.zeros(3), 0.25)
    M, _, Q, _ = oracle.moments(y, mb)
    r = np.array([1.1, 0.7, -1.9])
    pot, acc = oracle.m2l(r, M, Q)
    ex = oracle.monomials()
    idx = {tuple(e): k for k, e in enumerate(ex)}
    div = sum(acc[i, idx[tuple(np.eye(3, dtype=int)[i])]] for i in range(3))
    scale = np.abs(acc[:, 1:4]).max()
    assert abs(div) < 1e-13 * scale
    for i in range(3):
        lap = sum(2.0 * acc[i, idx[tuple(2 * np.eye(3, dtype=int)[j])]] for j in range(3))
        assert abs(lap) < 1e-13 * np.abs(acc[i, 4:10]).max()
    lap_phi = sum(2.0 * pot[idx[tuple(2 * np.eye(3, dtype=int)[j])]] for j in range(3))
    assert abs(lap_phi) < 1e-13 * np.abs(pot[4:10]).max()


def test_cluster_pair_error_decays_as_third_power(oracle):
    """Monopole + quadrupole source (the dipole vanishes about the centre of
    mass) and a second-order sink expansion: the error of a well-separated
    pair falls like (size / r)^3 relative to the force."""
    rng = np.random.default_rng(6)
    ys, ms = _cluster(rng, 40, np.zeros(3), 0.05)
    xs, mt = _cluster(rng, 10, np.zeros(3), 0.05)
    M, com_b, Q, _ = oracle.moments(ys, ms)
    _, com_a0, _, _ = oracle.moments(xs, mt)
    direction = np.array([0.6, -0.64, 0.48])
    errs, dists = [], [1.0, 2.0, 4.0, 8.0]
    for dist in dists:
        shift = direction * dist
        r = com_a0 + shift - com_b
        pot, acc = oracle.m2l(r, M, Q)
        e = []
        for xi in xs:
            a, _ = oracle.l2p(pot, acc, xi - com_a0)
            d = xi + shift - ys
            ex = -(ms[:, None] * d / np.linalg.norm(d, axis=1)[:, None] ** 3).sum(0)
            e.append(np.linalg.norm(a - ex) / np.linalg.norm(ex))
        errs.append(max(e))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(dists))
    assert np.all(slopes < -2.6) and np.all(slopes > -3.6), slopes


def test_newton_third_law_for_mutual_pair(oracle):
    """Sec. 3 (Eqs. 16-17 with the modified symmetric series, Eqs. 27-29): for a
    pair of cells that interact both ways through Eqs. 6 and 8 the total forces
    are equal and opposite."""
    rng = np.random.default_rng(7)
    xa, ma = _cluster(rng, 12, np.array([0.0, 0.0, 0.0]), 0.08)
    xb, mb = _cluster(rng, 17, np.array([1.3, -0.7, 0.4]), 0.1)
    Ma, ca, Qa, _ = oracle.moments(xa, ma)
    Mb, cb, Qb, _ = oracle.moments(xb, mb)
    potA, accA = oracle.m2l(ca - cb, Mb, Qb)         # field of B about A's centre
    potB, accB = oracle.m2l(cb - ca, Ma, Qa)         # field of A about B's centre
    FA = sum(mi * oracle.l2p(potA, accA, xi - ca)[0] for xi, mi in zip(xa, ma))
    FB = sum(mj * oracle.l2p(potB, accB, xj - cb)[0] for xj, mj in zip(xb, mb))
    assert np.linalg.norm(FA + FB) < 1e-13 * np.linalg.norm(FA)


# --------------------------------------------------------------------------
# Sec. 4: the asymmetric leaf <- super-cell example and the net force
# --------------------------------------------------------------------------

def _three_body(l, phi_dir, r=1.0, Ma=1.0, Mb1=0.3, Mb2=0.7):
    q = Mb1 / Mb2
    xv = l * np.array([math.cos(phi_dir), math.sin(phi_dir), 0.0])
    pos = np.array([[r, 0.0, 0.0], xv, -q * xv])      # alpha, beta1, beta2; com_beta at 0
    return pos, np.array([Ma, Mb1, Mb2]), q, xv


def test_asymmetric_example_matches_eq31(oracle):
    g = json.load(open(os.path.join(GOLDEN, "asymmetric_pair_eq31.json")))
    for phi_dir in (0.0, 0.7, 1.9):
        ratios = []
        for l in (0.04, 0.02, 0.01):
            pos, m, q, xv = _three_body(l, phi_dir)
            T = oracle.Tree(pos, m, theta=0.5, n_leaf=1, eps=1e-7)
            a, _, parts = T.eval(parts=True)
            F = fsum3(m, a)
            fac = m[0] * (m[1] + m[2]) * q * (1.0 - q)
            x1, x2 = xv[0], xv[1]
            want = np.array([g["F1"]["prefactor"] * fac * (2 * x1 ** 2 - 3 * x2 ** 2) * x1,
                             g["F2"]["prefactor"] * fac * (x2 ** 2 - 4 * x1 ** 2) * x2, 0.0])
            assert abs(F[2]) < 1e-6 * np.linalg.norm(want)
            ratios.append(np.linalg.norm(F - want) / np.linalg.norm(want))
        # the remainder is one order higher in l / r
        assert ratios[-1] < 0.05 and ratios[0] / ratios[-1] > 2.5, ratios
    # Eq. 32: the maximum over directions, attained along axis 1
    l = 0.01
    pos, m, q, _ = _three_body(l, 0.0)
    T = oracle.Tree(pos, m, theta=0.5, n_leaf=1, eps=1e-7)
    a, _ = T.eval()
    Fmax = g["Fmax"]["prefactor"] * l ** 3 * m[0] * (m[1] + m[2]) * q * (1 - q)
    assert abs(np.linalg.norm(fsum3(m, a)) / Fmax - 1.0) < 0.05


def test_total_force_nonzero_for_fmm_zero_for_direct(oracle):
    """Sec. 4/6: the leaf-only walk leaves an uncompensated total force; the
    direct sum does not."""
    ps = W.plummer(4096, W.seed_for(0))
    T = oracle.Tree(ps.x, ps.m, theta=0.5, n_leaf=16, eps=ps.eps)
    a, _ = T.eval()
    ad, _ = oracle.direct(ps.x, ps.m, eps=ps.eps)
    scale = math.fsum(ps.m * np.linalg.norm(ad, axis=1))
    assert np.linalg.norm(fsum3(ps.m, a)) > 1e-6 * scale
    assert np.linalg.norm(fsum3(ps.m, ad)) < 1e-14 * scale


def test_plummer_field_matches_analytic(oracle):
    """Validates the generator and the direct sum: the mean radial
    acceleration in shells follows -M_enc(r)/r^2 of the truncated Plummer
    sphere within Poisson noise."""
    n = 8192
    ps = W.plummer(n, W.seed_for(0, 2), eps=0.001)
    ad, _ = oracle.direct(ps.x, ps.m, eps=ps.eps)
    r = np.linalg.norm(ps.x, axis=1)
    ar = np.sum(ad * ps.x, axis=1) / r
    for lo, hi in [(0.3, 0.5), (0.5, 0.8), (0.8, 1.2), (1.2, 2.0), (2.0, 4.0)]:
        s = (r >= lo) & (r < hi)
        rm = r[s]
        want = -(rm ** 3 / (rm ** 2 + 1.0) ** 1.5) / 0.999 / rm ** 2
        got = ar[s] / want
        assert abs(got.mean() - 1.0) < 4.0 / math.sqrt(s.sum()) + 0.01, (lo, got.mean())


# --------------------------------------------------------------------------
# tree, moments and walk against brute force
# --------------------------------------------------------------------------

def _check_tree(oracle, ps, n_leaf):
    T = oracle.Tree(ps.x, ps.m, ps.h, theta=0.5, n_leaf=n_leaf, soft_kind=ps.soft_kind, eps=ps.eps)
    c = T.cells()
    order = T.order()
    assert np.array_equal(np.sort(order), np.arange(ps.n))
    h = ps.h if ps.h is not None else np.full(ps.n, ps.eps)
    for k in range(T.ncells):
        idx = order[c.first[k]:c.first[k] + c.count[k]]
        xs, ms = ps.x[idx], ps.m[idx]
        com = (ms[:, None] * xs).sum(0) / ms.sum()
        np.testing.assert_allclose(c.com[k], com, rtol=1e-12, atol=1e-14)
        assert c.M[k] == pytest.approx(ms.sum(), rel=1e-13)
        d = np.linalg.norm(xs - c.com[k], axis=1)
        assert c.s[k] == pytest.approx(d.max(), rel=1e-14, abs=1e-300)
        assert c.hmax[k] == h[idx].max()
        y = xs - c.com[k]
        Qf = 3 * np.einsum("n,ni,nj->ij", ms, y, y) - np.eye(3) * np.sum(ms * (y * y).sum(1))
        np.testing.assert_allclose(c.Q[k], Qf[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]],
                                   atol=1e-12 * max(1.0, np.abs(Qf).max()))
        if c.left[k] < 0:
            assert c.count[k] <= n_leaf and c.skip[k] == k + 1
            # a leaf keeps ascending caller order
            assert np.all(np.diff(idx) > 0)
            continue
        assert c.count[k] > n_leaf
        L, R = c.left[k], c.right[k]
        assert L == k + 1 and R == c.skip[L] and c.skip[k] == c.skip[R]
        assert c.first[L] == c.first[k] and c.first[R] == c.first[L] + c.count[L]
        assert c.count[L] + c.count[R] == c.count[k]
        ext = xs.max(0) - xs.min(0)
        axis = int(np.argmax(ext))
        left = ps.x[order[c.first[L]:c.first[L] + c.count[L]], axis]
        right = ps.x[order[c.first[R]:c.first[R] + c.count[R]], axis]
        assert left.max() < c.com[k][axis] <= right.min()
    return T, c


def test_tree_against_definitions(oracle):
    _check_tree(oracle, W.plummer(2000, W.seed_for(0, 3)), 16)
    _check_tree(oracle, W.polytrope_binary(700, W.seed_for(1, 3)), 10)
    _check_tree(oracle, W.uniform_clumps(3001, W.seed_for(2, 3)), 32)


def _brute_open(c, a, b, theta, rk):
    d = c.com[a] - c.com[b]
    r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
    return (r2 == 0.0 or theta == 0.0 or theta * theta * r2 < c.s[b] ** 2
            or r2 < (c.s[a] + c.s[b] + rk * max(c.hmax[a], c.hmax[b])) ** 2)


def test_walk_lists_equal_brute_force_enumeration(oracle):
    """far(alpha) = cells that are not opened but whose proper ancestors all
    are; near(alpha) = opened leaves whose ancestors all are (Sec. 2, Sec. 4)."""
    ps = W.plummer(1500, W.seed_for(0, 4))
    T = oracle.Tree(ps.x, ps.m, theta=0.6, n_leaf=8, eps=0.02)
    c = T.cells()
    L = T.walk()
    assert L.ancestor_far == 0
    for li, a in enumerate(L.leaf_ids):
        opened = np.array([_brute_open(c, a, b, 0.6, 2.0) for b in range(T.ncells)])
        anc_open = np.ones(T.ncells, dtype=bool)
        for b in range(1, T.ncells):          # pre-order: parents precede children
            p = c.parent[b]
            anc_open[b] = anc_open[p] and opened[p]
        far = np.nonzero(anc_open & ~opened)[0]
        near = np.nonzero(anc_open & opened & c.is_leaf)[0]
        assert np.array_equal(L.far_idx[L.far_off[li]:L.far_off[li + 1]], far)
        assert np.array_equal(L.near_idx[L.near_off[li]:L.near_off[li + 1]], near)
        # every particle is covered exactly once by far + near cells
        covered = np.zeros(ps.n, dtype=int)
        for b in np.concatenate([far, near]):
            covered[c.first[b]:c.first[b] + c.count[b]] += 1
        assert np.all(covered == 1)


def test_opening_criterion_threshold_uses_only_s_beta(oracle):
    """Eq. 4 is strict and involves s_beta only: a two-particle source leaf of
    size s at distance r is opened iff theta r < s, whatever the sink's size
    (Eq. 5 kept inactive with a tiny eps).  The source pair has masses 3:1 at
    z = +a and z = -3a, so its centre of mass is the origin and s = 3a."""
    eps = 1e-9
    r = 1.0
    for sink_size in (0.0, 0.02, 0.2):
        for s_over_r, want_open in ((0.499, False), (0.501, True)):
            a = s_over_r * r / 3.0
            src = np.array([[0.0, 0.0, a], [0.0, 0.0, -3.0 * a]])
            sink = np.array([[r, sink_size, 0.0], [r, -sink_size, 0.0]])
            x = np.concatenate([sink, src])
            m = np.array([0.25, 0.25, 0.3, 0.1])
            T = oracle.Tree(x, m, theta=0.5, n_leaf=2, eps=eps)
            c = T.cells()
            order = T.order()
            L = T.walk()
            leaves = list(L.leaf_ids)
            assert len(leaves) == 2
            sink_leaf = [k for k in leaves if 0 in order[c.first[k]:c.first[k] + c.count[k]]][0]
            src_leaf = [k for k in leaves if k != sink_leaf][0]
            assert c.s[src_leaf] == pytest.approx(3.0 * a, rel=1e-14)
            li = leaves.index(sink_leaf)
            near = set(L.near_idx[L.near_off[li]:L.near_off[li + 1]].tolist())
            assert (src_leaf in near) == want_open


# --------------------------------------------------------------------------
# invariances (exact in FP64: power-of-two scalings are exact)
# --------------------------------------------------------------------------

def test_mass_and_length_scaling_are_exact(oracle):
    ps = W.plummer(1024, W.seed_for(0, 5))
    T0 = oracle.Tree(ps.x, ps.m, theta=0.5, n_leaf=16, eps=ps.eps)
    a0, p0 = T0.eval()
    T1 = oracle.Tree(ps.x, 2.0 * ps.m, theta=0.5, n_leaf=16, eps=ps.eps)
    a1, p1 = T1.eval()
    assert np.array_equal(T0.order(), T1.order())
    assert np.array_equal(a1, 2.0 * a0) and np.array_equal(p1, 2.0 * p0)
    T2 = oracle.Tree(2.0 * ps.x, ps.m, theta=0.5, n_leaf=16, eps=2.0 * ps.eps)
    a2, p2 = T2.eval()
    L0, L2 = T0.walk(), T2.walk()
    assert np.array_equal(T0.order(), T2.order())
    assert np.array_equal(L0.far_idx, L2.far_idx) and np.array_equal(L0.near_idx, L2.near_idx)
    assert np.array_equal(a2, 0.25 * a0) and np.array_equal(p2, 0.5 * p0)


# --------------------------------------------------------------------------
# M4 kernel softening (Sec. 3 Eq. 13, Sec. 6: cubic spline, R_kern = 2)
# --------------------------------------------------------------------------

def test_m4_kernel_against_quadrature(oracle):
    w = lambda q: oracle.m4(q)[0]
    norm, _ = integrate.quad(lambda q: 4 * math.pi * q * q * w(q), 0, 2, points=[1.0])
    assert norm == pytest.approx(1.0, abs=1e-12)
    for q in (0.05, 0.3, 0.9, 1.0, 1.2, 1.7, 1.99, 2.0, 2.5):
        F_num, _ = integrate.quad(lambda u: 4 * math.pi * u * u * w(u), 0, min(q, 2.0), points=[1.0] if q > 1 else None)
        assert oracle.m4(q)[1] == pytest.approx(F_num, abs=1e-12)
        # P(q) = int_q^inf F(u)/u^2 du  (psi = P/h, psi' = -F/r^2, psi -> 1/r)
        P_num = 1.0 / max(q, 2.0)
        if q < 2.0:
            P_num += integrate.quad(lambda u: oracle.m4(u)[1] / u ** 2, q, 2.0,
                                    points=[1.0] if q < 1 else None)[0]
        assert oracle.m4(q)[2] == pytest.approx(P_num, abs=1e-11)
    # w is C^2 at the knots and flat at the centre (the cubic B-spline)
    for k in (1.0, 2.0):
        for der in range(3):
            hh = 1e-4
            f = lambda t: np.array([w(k + t - hh), w(k + t), w(k + t + hh)])
            lo, hi = f(-2 * hh), f(2 * hh)
            dlo = [lo[1], (lo[2] - lo[0]) / (2 * hh), (lo[2] - 2 * lo[1] + lo[0]) / hh ** 2][der]
            dhi = [hi[1], (hi[2] - hi[0]) / (2 * hh), (hi[2] - 2 * hi[1] + hi[0]) / hh ** 2][der]
            assert abs(dlo - dhi) < [1e-3, 2e-3, 6e-2][der]
    assert (w(1e-4) - w(0.0)) / 1e-4 == pytest.approx(0.0, abs=1e-3)


def test_m4_pair_is_symmetric_and_newtonian_outside_support(oracle):
    rng = np.random.default_rng(8)
    for _ in range(20):
        d = rng.normal(0, 0.03, 3)
        mi, mj = rng.uniform(0.5, 2, 2)
        hi, hj = rng.uniform(0.005, 0.03, 2)
        ai, pi = oracle.pair(d, mj, hi, hj, soft_kind=1)
        aj, pj = oracle.pair(-d, mi, hj, hi, soft_kind=1)
        np.testing.assert_allclose(mi * ai, -mj * aj, rtol=1e-14, atol=1e-300)
        assert pi / mj == pytest.approx(pj / mi, rel=1e-14)
        r = np.linalg.norm(d)
        if r >= 2 * max(hi, hj):
            np.testing.assert_allclose(ai, -mj * d / r ** 3, rtol=1e-13)
            assert pi == pytest.approx(-mj / r, rel=1e-13)


# --------------------------------------------------------------------------
# frozen topology (reading: same cells and particle order, new x, m, h) and
# evaluation from given lists
# --------------------------------------------------------------------------

def _frozen_definitions(c, order, x, m, h):
    """Per-cell M, centre of mass, s, h_max and traceless Q (Sec. 2, Eq. 7)
    written out from the particles of each cell's range [first, first+count)."""
    out = []
    for k in range(len(c.first)):
        idx = order[c.first[k]:c.first[k] + c.count[k]]
        xs, ms = x[idx], m[idx]
        M = math.fsum(ms)
        com = np.array([math.fsum(ms * xs[:, d]) for d in range(3)]) / M
        y = xs - com
        s = np.sqrt((y * y).sum(1)).max()
        Qf = 3 * np.einsum("n,ni,nj->ij", ms, y, y) - np.eye(3) * np.sum(ms * (y * y).sum(1))
        out.append((M, com, s, h[idx].max(), Qf[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]))
    return out


@pytest.mark.parametrize("kind", ["polytrope_m4", "plummer"])
def test_moments_frozen_against_definitions(oracle, kind):
    """After moving every particle, changing every mass and smoothing length,
    the frozen-topology moments of each cell equal the definitions over the
    cell's unchanged particle range: M and centre of mass (Sec. 2), s = the
    largest distance from the new centre of mass, h_max, and Q (Eq. 7) about
    the new centre of mass.  A super-cell's M is exactly its children's sum.
    At unchanged inputs a leaf's moments equal the fresh build's bit for bit
    (both are the same pairwise sums over the leaf in caller order)."""
    if kind == "polytrope_m4":
        ps = W.polytrope_binary(700, W.seed_for(1, 7))
        T = oracle.Tree(ps.x, ps.m, ps.h, theta=0.5, n_leaf=10, soft_kind=oracle.SOFT_M4, eps=ps.eps)
    else:
        ps = W.plummer(2000, W.seed_for(0, 7))
        T = oracle.Tree(ps.x, ps.m, theta=0.5, n_leaf=16, eps=ps.eps)
    c0 = T.cells()
    order = T.order()
    leaf = c0.left < 0

    T.moments_frozen(ps.x, ps.m, ps.h)
    c1 = T.cells()
    for f in ("M", "com", "s", "hmax"):
        assert np.array_equal(getattr(c1, f)[leaf], getattr(c0, f)[leaf]), f
    np.testing.assert_allclose(c1.M, c0.M, rtol=1e-14)
    np.testing.assert_allclose(c1.com, c0.com, rtol=1e-13, atol=1e-15)

    rng = np.random.default_rng(77)
    x1 = ps.x + rng.normal(0.0, 0.02, ps.x.shape)
    m1 = ps.m * rng.uniform(0.5, 2.0, ps.n)
    h1 = None if ps.h is None else ps.h * rng.uniform(0.8, 1.25, ps.n)
    T.moments_frozen(x1, m1, h1)
    c2 = T.cells()
    for f in ("first", "count", "left", "right", "parent", "skip", "depth"):
        assert np.array_equal(getattr(c2, f), getattr(c0, f)), f
    assert np.array_equal(T.order(), order)
    hh = np.full(ps.n, ps.eps) if h1 is None else h1
    ref = _frozen_definitions(c2, order, x1, m1, hh)
    for k, (M, com, s, hmax, Q) in enumerate(ref):
        assert c2.M[k] == pytest.approx(M, rel=1e-13)
        np.testing.assert_allclose(c2.com[k], com, rtol=1e-12, atol=1e-14)
        assert c2.s[k] == pytest.approx(s, rel=1e-12)
        assert c2.hmax[k] == hmax
        np.testing.assert_allclose(c2.Q[k], Q, atol=1e-12 * max(1e-300, c2.M[k] * c2.s[k] ** 2))
        if c2.left[k] >= 0:
            assert c2.M[k] == c2.M[c2.left[k]] + c2.M[c2.right[k]]
    # the moved moments differ from the original ones (the call is not a no-op)
    assert not np.array_equal(c2.com, c0.com)


def test_eval_lists_reproduces_eval_and_reads_its_lists(oracle):
    """Evaluation from given lists: with the walk's own lists it is the
    evaluation bit for bit (Sec. 4's leaf walk feeds Eq. 3); with every leaf
    listing every leaf as near and nothing far it is the O(N^2) direct sum;
    and the order in which leaves are listed does not matter."""
    ps = W.polytrope_binary(600, W.seed_for(1, 8))
    T = oracle.Tree(ps.x, ps.m, ps.h, theta=0.5, n_leaf=12, soft_kind=oracle.SOFT_M4, eps=ps.eps)
    a0, p0 = T.eval()
    L = T.walk()
    assert len(L.far_idx) > 0 and len(L.near_idx) > 0
    a1, p1 = T.eval_lists(L)
    assert np.array_equal(a1, a0) and np.array_equal(p1, p0)

    # leaves listed in reverse, each with its own lists
    nl = len(L.leaf_ids)
    rev = np.arange(nl)[::-1]
    fo = np.concatenate([[0], np.cumsum(np.diff(L.far_off)[rev])])
    no = np.concatenate([[0], np.cumsum(np.diff(L.near_off)[rev])])
    fi = np.concatenate([L.far_idx[L.far_off[k]:L.far_off[k + 1]] for k in rev])
    ni = np.concatenate([L.near_idx[L.near_off[k]:L.near_off[k + 1]] for k in rev])
    Lr = oracle.Lists(L.leaf_ids[rev].copy(), fo, fi.astype(np.int32), no, ni.astype(np.int32), 0)
    a2, p2 = T.eval_lists(Lr)
    assert np.array_equal(a2, a0) and np.array_equal(p2, p0)

    # all near, nothing far: the direct sum (j != i, same pair interaction)
    leaves = L.leaf_ids.astype(np.int32)
    Ld = oracle.Lists(leaves, np.zeros(nl + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                      np.arange(nl + 1, dtype=np.int64) * nl, np.tile(leaves, nl), 0)
    a3, p3 = T.eval_lists(Ld)
    ad, pd = oracle.direct(ps.x, ps.m, ps.h, soft_kind=oracle.SOFT_M4, eps=ps.eps)
    assert np.max(rel_err(a3, ad)) < 1e-13
    np.testing.assert_allclose(p3, pd, rtol=1e-13)


def test_frozen_lists_on_moved_particles_at_theta_zero_are_direct(oracle):
    """theta = 0 opens every cell (Sec. 2), so the frozen lists are all near;
    after moving the particles and changing their masses, the evaluation
    from those lists on the frozen-topology moments is the direct sum of the
    moved system."""
    ps = W.plummer(900, W.seed_for(0, 9))
    T = oracle.Tree(ps.x, ps.m, theta=0.0, n_leaf=16, eps=ps.eps)
    L = T.walk()
    assert len(L.far_idx) == 0
    rng = np.random.default_rng(5)
    x1 = ps.x + rng.normal(0.0, 0.05, ps.x.shape)
    m1 = ps.m * rng.uniform(0.5, 2.0, ps.n)
    T.moments_frozen(x1, m1, None)
    a, p = T.eval_lists(L)
    ad, pd = oracle.direct(x1, m1, eps=ps.eps)
    assert np.max(rel_err(a, ad)) < 1e-13
    np.testing.assert_allclose(p, pd, rtol=1e-13)
