"""Pins of the oracle's symmetric dual-tree walk (a separate mode, the
correction the paper's conclusions call for): every pair of particles is
covered exactly once; the lists are mutual; far pairs satisfy the symmetric
criteria and near pairs do not; theta = 0 is the direct sum; and the total
force vanishes to rounding, where the leaf-only walk leaves it."""
import math

import numpy as np
import pytest

from paper_2502_01496_gb300 import workloads as W


def _fsum3(m, a):
    return np.array([math.fsum(m * a[:, k]) for k in range(3)])


def _leaf_ranks(cells):
    is_leaf = cells.left < 0
    rank = np.full(cells.left.size, -1)
    rank[is_leaf] = np.arange(is_leaf.sum())
    return rank


@pytest.mark.parametrize("theta", [0.4, 0.8])
def test_every_particle_pair_is_covered_exactly_once(oracle, theta):
    """Brute force: for every ordered pair (i, j) the number of far entries
    (cell C holding i receives from cell B holding j) plus near entries (leaf of
    i receives from leaf of j) is exactly one."""
    ps = W.plummer(300, W.seed_for(0, 80))
    T = oracle.Tree(ps.x, ps.m, theta=theta, n_leaf=8, eps=ps.eps)
    c, order, D = T.cells(), T.order(), T.dual_walk()
    pos = np.empty(ps.n, dtype=np.int64)
    pos[order] = np.arange(ps.n)
    nc = c.first.size
    # membership[cell, particle]
    member = np.zeros((nc, ps.n), dtype=np.int64)
    for k in range(nc):
        member[k, order[c.first[k]:c.first[k] + c.count[k]]] = 1
    cover = np.zeros((ps.n, ps.n), dtype=np.int64)
    for a in range(nc):
        for e in range(D.far_off[a], D.far_off[a + 1]):
            b = D.far_idx[e]
            cover += np.outer(member[a], member[b])
    leaves = np.nonzero(c.left < 0)[0]
    for k, a in enumerate(leaves):
        for e in range(D.near_off[k], D.near_off[k + 1]):
            cover += np.outer(member[a], member[D.near_idx[e]])
    # the pairs of a pair entry are disjoint cells, so (i, i) is covered only by
    # the leaf's entry with itself (where P2P skips j = i)
    assert np.all(cover == 1), np.argwhere(cover != 1)[:5]


def test_lists_are_mutual_and_respect_the_criteria(oracle):
    ps = W.polytrope_binary(1500, W.seed_for(1, 81))
    theta, rk = 0.6, 2.0
    T = oracle.Tree(ps.x, ps.m, ps.h, theta=theta, n_leaf=16, soft_kind=1, eps=ps.eps, r_kern=rk)
    c, D = T.cells(), T.dual_walk()
    rank = _leaf_ranks(c)
    leaves = np.nonzero(c.left < 0)[0]
    far = {(a, int(b)) for a in range(c.first.size) for b in D.far_idx[D.far_off[a]:D.far_off[a + 1]]}
    near = {(int(leaves[k]), int(b)) for k in range(leaves.size)
            for b in D.near_idx[D.near_off[k]:D.near_off[k + 1]]}
    assert far and near
    assert all((b, a) in far for a, b in far)
    assert all((b, a) in near for a, b in near)
    for a, b in far:
        r = np.linalg.norm(c.com[a] - c.com[b])
        assert theta * r > c.s[a] + c.s[b]
        assert r >= c.s[a] + c.s[b] + rk * max(c.hmax[a], c.hmax[b])
    for a, b in near:
        assert rank[a] >= 0 and rank[b] >= 0
        if a != b:
            r = np.linalg.norm(c.com[a] - c.com[b])
            sep = (theta * r > c.s[a] + c.s[b]) and (r >= c.s[a] + c.s[b] + rk * max(c.hmax[a], c.hmax[b]))
            assert not sep


@pytest.mark.parametrize("kind", ["plummer", "m4"])
def test_dual_walk_conserves_momentum_and_converges(oracle, kind):
    ps = W.plummer(3000, W.seed_for(0, 82)) if kind == "plummer" else W.polytrope_binary(1500, W.seed_for(1, 83))
    ad, _ = oracle.direct(ps.x, ps.m, ps.h, soft_kind=ps.soft_kind, eps=ps.eps)
    scale = math.fsum(ps.m * np.linalg.norm(ad, axis=1))
    errs = []
    for theta in (0.0, 0.3, 0.5, 0.8):
        T = oracle.Tree(ps.x, ps.m, ps.h, theta=theta, n_leaf=16, soft_kind=ps.soft_kind, eps=ps.eps)
        a, _ = T.eval_dual()
        assert np.linalg.norm(_fsum3(ps.m, a)) < 1e-14 * scale, theta
        errs.append(np.linalg.norm(a - ad, axis=1).max() / np.linalg.norm(ad, axis=1).max())
        if theta == 0.5:
            a0, _ = T.eval()
            assert np.linalg.norm(_fsum3(ps.m, a0)) > 1e-7 * scale     # the leaf-only walk's force
    assert errs[0] < 1e-13
    assert errs[1] < errs[2] < errs[3]
