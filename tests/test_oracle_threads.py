"""The oracle's leaf-parallel evaluation (OpenMP over target leaves, used to
time the oracle on every host core) gives the single-threaded evaluation's
result bit for bit: every leaf's walk and sums are the same steps, and each
leaf writes only its own particles."""
import numpy as np

from paper_2502_01496_gb300 import workloads as W


def test_threaded_evaluation_is_bit_identical(oracle):
    ps = W.polytrope_binary(3000, W.seed_for(1, 21))
    T = oracle.Tree(ps.x, ps.m, ps.h, theta=0.5, n_leaf=12, soft_kind=oracle.SOFT_M4, eps=ps.eps)
    a0, p0 = T.eval()
    for nthreads in (0, 1, 3):
        a1, p1 = T.eval_threads(nthreads=nthreads)
        assert np.array_equal(a0, a1) and np.array_equal(p0, p1)
    leaves = np.sort(np.random.default_rng(2).choice(T.walk().leaf_ids, 40, replace=False))
    a2, p2 = T.eval(leaves=leaves)
    a3, p3 = T.eval_threads(leaves=leaves)
    assert np.array_equal(a2, a3, equal_nan=True) and np.array_equal(p2, p3, equal_nan=True)
    assert oracle.max_threads() >= 1
