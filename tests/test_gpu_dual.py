"""The symmetric dual-tree walk (walk = 1) on the GPU against the oracle's:
the per-cell far lists and per-leaf near lists equal as sets, forces within
the precision's bound, theta = 0 is the direct sum, and the total force sum
m a vanishes to rounding where the paper's leaf-only walk leaves it."""
import math

import numpy as np
import pytest

from paper_2502_01496_gb300 import workloads as W

from gpu_common import assert_tree_bit_exact, fsum_force, rel_errors, split_forest

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


def _cuda(a):
    import torch
    return None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")


def _gpu(ps, theta, prec, n_leaf=16):
    import torch
    from paper_2502_01496_gb300 import native
    f = native.KdFmm(theta=theta, eps=ps.eps, n_leaf=n_leaf, soft_kind=ps.soft_kind, precision=prec,
                     walk=1)
    f.build(_cuda(ps.x), _cuda(ps.m), _cuda(ps.h))
    a, phi = f.accel()
    torch.cuda.synchronize()
    return f, a.cpu().numpy(), phi.cpu().numpy()


CASES = [("plummer", 0.5, FP64), ("plummer", 0.3, FP64), ("plummer", 0.8, MIXED),
         ("plummer", 0.5, MIXED), ("polytrope_m4", 0.5, FP64), ("polytrope_m4", 0.6, MIXED)]


@pytest.mark.parametrize("case,theta,prec", CASES)
def test_dual_walk_against_oracle(oracle, case, theta, prec):
    ps = (W.plummer(4096, W.seed_for(0, 90)) if case == "plummer"
          else W.polytrope_binary(2048, W.seed_for(1, 91)))
    f, ga, gphi = _gpu(ps, theta, prec)
    ex = f.export(lists=True)
    T = oracle.Tree(ps.x, ps.m, ps.h, theta=theta, n_leaf=16, soft_kind=ps.soft_kind, eps=ps.eps)
    assert_tree_bit_exact({"ex": ex}, {"order": T.order(), "cells": T.cells()})
    D = T.dual_walk()
    assert np.array_equal(ex.far_off, D.far_off) and np.array_equal(ex.far_idx, D.far_idx)
    assert np.array_equal(ex.near_off, D.near_off) and np.array_equal(ex.near_idx, D.near_idx)
    oa, ophi = T.eval_dual()
    ea, ep = rel_errors(ga, gphi, oa, ophi)
    tol = 1e-12 if prec == FP64 else 2e-5
    assert ea.max() < tol and ep.max() < tol, (ea.max(), ep.max())
    scale = math.fsum(ps.m * np.linalg.norm(oa, axis=1))
    F = np.linalg.norm(fsum_force(ps.m, ga))
    # momentum: rounding of float64 (FP64) or of the float32 pair and expansion
    # terms (mixed), against ~1e-4 for the paper's walk
    assert F < (1e-13 if prec == FP64 else 1e-6) * scale, F / scale
    st = f.stats()
    assert st["nfar"] == len(D.far_idx) and st["nnear"] == len(D.near_idx)


def test_dual_walk_theta_zero_is_direct_sum(oracle):
    ps = W.plummer(1500, W.seed_for(0, 92))
    f, ga, gphi = _gpu(ps, 0.0, FP64)
    ad, pd = oracle.direct(ps.x, ps.m, eps=ps.eps)
    ea, ep = rel_errors(ga, gphi, ad, pd)
    assert ea.max() < 1e-12 and ep.max() < 1e-12
    assert f.stats()["nfar"] == 0


def test_dual_walk_forest(oracle):
    """A forest under the dual walk: each system's lists and forces equal the
    oracle's for that system alone."""
    import torch
    from paper_2502_01496_gb300 import native
    systems = [W.plummer(n, W.seed_for(3, 93 + k)) for k, n in enumerate([2000, 17, 3500])]
    theta = np.array([0.5, 0.7, 0.4])
    x = np.concatenate([p.x for p in systems])
    m = np.concatenate([p.m for p in systems])
    off = np.concatenate([[0], np.cumsum([p.n for p in systems])]).astype(np.int64)
    f = native.KdFmm(theta=0.5, eps=0.01, n_leaf=16, soft_kind=0, precision=FP64, walk=1)
    a = torch.empty((x.shape[0], 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(x.shape[0], dtype=torch.float64, device="cuda")
    native.fmm_accel_batched(f.handle, _cuda(x), _cuda(m), None, off, f.params, a, phi, theta=theta)
    f.n = x.shape[0]
    torch.cuda.synchronize()
    ga, gphi = a.cpu().numpy(), phi.cpu().numpy()
    st = f.stats()
    assert st["nfar"] > 0
    for k, ps in enumerate(systems):
        T = oracle.Tree(ps.x, ps.m, None, theta=theta[k], n_leaf=16, soft_kind=0, eps=ps.eps)
        oa, ophi = T.eval_dual()
        sl = slice(off[k], off[k + 1])
        ea, ep = rel_errors(ga[sl], gphi[sl], oa, ophi)
        assert ea.max() < 1e-12 and ep.max() < 1e-12, (k, ea.max(), ep.max())


def test_dual_walk_refuses_the_adjoint():
    from paper_2502_01496_gb300 import native
    ps = W.plummer(500, W.seed_for(0, 94))
    f, _, _ = _gpu(ps, 0.5, FP64)
    with pytest.raises(native.KdfmmError):
        f.vjp(_cuda(np.zeros((ps.n, 3))))
