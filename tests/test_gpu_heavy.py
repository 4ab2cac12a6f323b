"""Leaves with very long walks and near lists.  In a centrally condensed
system a large leaf in the sparse outskirts fails the opening criteria
against most of the tree: its walk visits most cells and its near list holds
most leaves.  Such a walk is handed from its thread to a whole block, and
such a near list is split into segments summed by separate warps.  Neither
may change a result: the lists stay bit-exact against the oracle's walk, the
forces equal the unsplit evaluation's bits where the lists are the same, and
repeated evaluations give identical bits."""
import numpy as np
import pytest

from paper_2502_01496_gb300 import workloads as W

from gpu_common import assert_lists_bit_exact, assert_tree_bit_exact, rel_errors, split_forest

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
TOL = {FP64: 1e-12, MIXED: 2e-5}
SEG_ENTRIES = 256          # near entries per P2P segment in the library


def _cuda(a):
    import torch
    return torch.tensor(a, dtype=torch.float64, device="cuda")


def _eval(ps, theta, prec, n_leaf=16):
    import torch
    from paper_2502_01496_gb300 import native
    f = native.KdFmm(theta=theta, eps=ps.eps, n_leaf=n_leaf, soft_kind=ps.soft_kind, precision=prec)
    f.build(_cuda(ps.x), _cuda(ps.m), None if ps.h is None else _cuda(ps.h))
    a, phi = f.accel()
    torch.cuda.synchronize()
    return f, a.cpu().numpy(), phi.cpu().numpy()


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("budget", ["1", "37"])
@pytest.mark.parametrize("list_mode", ["slots", "exact", "two_pass"])
def test_block_walk_equals_thread_walk(oracle, monkeypatch, prec, budget, list_mode):
    """A budget of 1 hands every leaf to the block-wide walk, 37 about half
    of them: lists, statistics and force bits equal the thread walk's."""
    ps = W.plummer(4096, W.seed_for(0, 96))
    if list_mode != "slots":
        monkeypatch.setenv("KDFMM_LIST_MODE", list_mode)
    f0, a0, p0 = _eval(ps, 0.5, prec)
    ex0, st0 = f0.export(lists=True), f0.stats()
    monkeypatch.setenv("KDFMM_WALK_BUDGET", budget)
    f1, a1, p1 = _eval(ps, 0.5, prec)
    ex1, st1 = f1.export(lists=True), f1.stats()
    for name in ("far_off", "far_idx", "near_off", "near_idx"):
        assert np.array_equal(getattr(ex0, name), getattr(ex1, name)), name
    for key in ("nfar", "nnear", "np2p", "nexact"):
        assert st0[key] == st1[key], (key, st0[key], st1[key])
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1)
    T = oracle.Tree(ps.x, ps.m, None, theta=0.5, n_leaf=16, soft_kind=0, eps=ps.eps)
    assert_lists_bit_exact({"ex": ex1}, {"lists": T.walk()})


def test_block_walk_forest(oracle, monkeypatch):
    """Block-wide walks stay inside their own system's tree."""
    import torch
    from paper_2502_01496_gb300 import native
    monkeypatch.setenv("KDFMM_WALK_BUDGET", "5")
    systems = [W.plummer(n, W.seed_for(3, 960 + k)) for k, n in enumerate([3000, 40, 5000])]
    theta = np.array([0.4, 0.8, 0.6])
    x = np.concatenate([p.x for p in systems])
    m = np.concatenate([p.m for p in systems])
    off = np.concatenate([[0], np.cumsum([p.n for p in systems])]).astype(np.int64)
    f = native.KdFmm(theta=0.5, eps=0.01, n_leaf=16, soft_kind=0, precision=FP64)
    a = torch.empty((x.shape[0], 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(x.shape[0], dtype=torch.float64, device="cuda")
    native.fmm_accel_batched(f.handle, _cuda(x), _cuda(m), None, off, f.params, a, phi,
                             theta=theta, eps=np.full(3, 0.01), n_leaf=np.full(3, 16))
    f.n = x.shape[0]
    torch.cuda.synchronize()
    ga, gphi = a.cpu().numpy(), phi.cpu().numpy()
    parts = split_forest(f.export(lists=True), off)
    for k, ps in enumerate(systems):
        T = oracle.Tree(ps.x, ps.m, None, theta=theta[k], n_leaf=16, soft_kind=0, eps=0.01)
        assert_lists_bit_exact({"ex": parts[k]}, {"lists": T.walk()})
        oa, ophi = T.eval()
        sl = slice(off[k], off[k + 1])
        ea, ep = rel_errors(ga[sl], gphi[sl], oa, ophi)
        assert ea.max() < 1e-12 and ep.max() < 1e-12, (k, ea.max(), ep.max())


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_block_walk_in_arena_scratch(oracle, monkeypatch, prec):
    """Arena mode: a block-wide walk writes its leaf's lists into the block's
    slice of the (idle) thread-walk scratch and copies them to reserved room,
    in one pass.  Sizes: 2^15 particles, about 2900 leaves, so the arena grid
    has 23 blocks of 128 threads and a budget of 1000 gives slices of
    2944 * 1000 / (2 * 152 SMs) = 9684 entries, more than the system's ~5800
    cells; at theta = 0.5 the mean walk is longer than 1000 cells, so many leaves
    are handed on.  Lists, statistics and force bits equal the thread walk's."""
    ps = W.plummer(1 << 15, W.seed_for(0, 98))
    monkeypatch.setenv("KDFMM_LIST_MODE", "exact")
    monkeypatch.setenv("KDFMM_WALK_BUDGET", "30000")       # every leaf walks in its thread
    f0, a0, p0 = _eval(ps, 0.5, prec)
    ex0, st0 = f0.export(lists=True), f0.stats()
    assert st0["nheavy"] == 0, st0
    monkeypatch.setenv("KDFMM_WALK_BUDGET", "1000")
    f1, a1, p1 = _eval(ps, 0.5, prec)
    ex1, st1 = f1.export(lists=True), f1.stats()
    assert st1["nheavy"] > st1["nleaves"] // 10, st1
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    threads = -(-st1["nleaves"] // 128) * 128              # the arena grid (one round)
    assert st1["ncells"] <= threads * 1000 // (2 * sms), st1   # the slice holds the system
    for name in ("far_off", "far_idx", "near_off", "near_idx"):
        assert np.array_equal(getattr(ex0, name), getattr(ex1, name)), name
    for key in ("nfar", "nnear", "np2p", "nexact"):
        assert st0[key] == st1[key], (key, st0[key], st1[key])
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1)
    T = oracle.Tree(ps.x, ps.m, None, theta=0.5, n_leaf=16, soft_kind=0, eps=ps.eps)
    assert_lists_bit_exact({"ex": ex1}, {"lists": T.walk()})


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_split_near_lists_against_oracle(oracle, prec):
    """Plummer 16384 at theta = 0.5: dozens of near lists span several
    segments.  Forces match the oracle; two evaluations give identical bits."""
    ps = W.plummer(16384, W.seed_for(0, 97))
    f, a1, p1 = _eval(ps, 0.5, prec)
    ex = f.export(lists=True)
    nn = np.diff(ex.near_off)
    assert (nn > 2 * SEG_ENTRIES).sum() >= 10, nn.max()
    _, a2, p2 = _eval(ps, 0.5, prec)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
    T = oracle.Tree(ps.x, ps.m, None, theta=0.5, n_leaf=16, soft_kind=0, eps=ps.eps)
    assert_tree_bit_exact({"ex": ex}, {"order": T.order(), "cells": T.cells()})
    oa, ophi = T.eval()
    ea, ep = rel_errors(a1, p1, oa, ophi)
    assert ea.max() < TOL[prec] and ep.max() < TOL[prec], (ea.max(), ep.max())


def test_naturally_heavy_leaves_262144(oracle):
    """Plummer 2^18: the outskirts' leaves walk most of the tree (the default
    budget hands them on) and have near lists of most leaves.  The lists equal
    the oracle's; the forces on the particles of the heaviest leaves and of a
    random sample match the oracle's evaluation of those leaves."""
    ps = W.plummer(1 << 18, W.seed_for(4))
    f, ga, gphi = _eval(ps, 0.5, MIXED)
    ex = f.export(lists=True)
    T = oracle.Tree(ps.x, ps.m, None, theta=0.5, n_leaf=16, soft_kind=0, eps=ps.eps)
    L = T.walk()
    assert_lists_bit_exact({"ex": ex}, {"lists": L})
    nn = np.diff(L.near_off)
    assert nn.max() > 10000
    heavy = L.leaf_ids[np.argsort(-nn)[:6]]
    rng = np.random.default_rng(5)
    leaves = np.unique(np.concatenate([heavy, rng.choice(L.leaf_ids, 60, replace=False)]))
    oa, ophi = T.eval(leaves=leaves)
    rows = np.nonzero(np.isfinite(oa[:, 0]))[0]
    ea, ep = rel_errors(ga, gphi, oa, ophi, rows)
    assert ea.max() < TOL[MIXED] and ep.max() < TOL[MIXED], (ea.max(), ep.max())


def test_walk_budget_setting_changes_no_result():
    """kdfmm_tree_set_walk_budget only moves leaves between the thread walk
    and the block-wide walk: lists and forces are bit-identical for any
    budget, on a single system and on a captured forest (whose graph is
    captured again when the budget changes)."""
    import torch
    from paper_2502_01496_gb300 import native
    ps = W.plummer(1 << 16, W.seed_for(4, 31))
    ref_f, ref_a, ref_phi = _eval(ps, 0.5, MIXED)
    ref_ex = ref_f.export(lists=True)
    f = native.KdFmm(theta=0.5, eps=ps.eps, n_leaf=16, soft_kind=0, precision=MIXED)
    x, m = _cuda(ps.x), _cuda(ps.m)
    for budget in (3, 300, 0):
        native.tree_set_walk_budget(f.handle, budget)
        f.build(x, m)
        a, phi = f.accel()
        torch.cuda.synchronize()
        ex = f.export(lists=True)
        assert np.array_equal(ex.far_idx, ref_ex.far_idx) and np.array_equal(ex.near_idx, ref_ex.near_idx)
        assert np.array_equal(a.cpu().numpy(), ref_a) and np.array_equal(phi.cpu().numpy(), ref_phi)
    # a forest of two systems through the captured-graph path
    sizes = np.array([5000, 20000])
    systems = [W.plummer(int(k), W.seed_for(4, 40 + i)) for i, k in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    xs = _cuda(np.concatenate([p.x for p in systems]))
    ms = _cuda(np.concatenate([p.m for p in systems]))
    out = []
    for budget in (0, 5, 0):
        native.tree_set_walk_budget(f.handle, budget)
        ab = torch.empty((int(off[-1]), 3), dtype=torch.float64, device="cuda")
        for _ in range(3):                                  # eager, capture, replay
            native.fmm_accel_batched(f.handle, xs, ms, None, off, f.params, ab, None,
                                     theta=np.array([0.4, 0.8]), n_leaf=np.array([16, 12], dtype=np.int32))
        torch.cuda.synchronize()
        out.append(ab.cpu().numpy())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    with pytest.raises(native.KdfmmError):
        native.tree_set_walk_budget(f.handle, -1)
