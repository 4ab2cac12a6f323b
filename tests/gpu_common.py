"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare."""
import math

import numpy as np


def run_gpu(ps, *, theta, n_leaf, precision, r_kern=2.0, lists=True):
    import torch
    from paper_2502_01496_gb300 import native
    x = torch.tensor(ps.x, dtype=torch.float64, device="cuda")
    m = torch.tensor(ps.m, dtype=torch.float64, device="cuda")
    h = None if ps.h is None else torch.tensor(ps.h, dtype=torch.float64, device="cuda")
    f = native.KdFmm(theta=theta, eps=ps.eps, r_kern=r_kern, n_leaf=n_leaf,
                     soft_kind=ps.soft_kind, precision=precision)
    f.build(x, m, h)
    a, phi = f.accel()
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    native.total_momentum(m, a, out)
    torch.cuda.synchronize()
    ex = f.export(lists=lists)
    return dict(a=a.cpu().numpy(), phi=phi.cpu().numpy(), F=out.cpu().numpy(), ex=ex,
                stats=f.stats())


def run_oracle(oracle, ps, *, theta, n_leaf, r_kern=2.0, evaluate=True, lists=True):
    T = oracle.Tree(ps.x, ps.m, ps.h, theta=theta, n_leaf=n_leaf, soft_kind=ps.soft_kind,
                    eps=ps.eps, r_kern=r_kern)
    a, phi = T.eval() if evaluate else (None, None)
    return dict(T=T, a=a, phi=phi, cells=T.cells(), order=T.order(),
                lists=T.walk() if lists else None)


def oracle_cell_arrays(c):
    ints = np.stack([c.first, c.count, c.left, c.right, c.parent, c.depth, c.skip], axis=1)
    reals = np.concatenate([c.M[:, None], c.com, c.s[:, None], c.hmax[:, None], c.Q], axis=1)
    return ints, reals


def assert_tree_bit_exact(g, o):
    ex = g["ex"]
    oi, orr = oracle_cell_arrays(o["cells"])
    assert np.array_equal(ex.perm, o["order"]), "particle order differs"
    assert ex.cell_ints.shape == oi.shape, (ex.cell_ints.shape, oi.shape)
    bad = np.nonzero(np.any(ex.cell_ints != oi, axis=1))[0]
    assert bad.size == 0, f"cell structure differs at {bad[:10]}"
    # M, centre of mass, s and h_max decide the walk: bit-exact
    np.testing.assert_array_equal(ex.cell_reals[:, :6], orr[:, :6])
    # quadrupoles: float64 rounding only, measured against M s^2, the scale at
    # which Q enters the field (Eq. 6: Q / r^4 against M / r^2 with s < r)
    scale = (orr[:, 0] * orr[:, 4] ** 2)[:, None] + 1e-300
    qerr = (np.abs(ex.cell_reals[:, 6:] - orr[:, 6:]) / scale).max()
    assert qerr < 1e-12, qerr


def assert_lists_bit_exact(g, o):
    ex, L = g["ex"], o["lists"]
    assert np.array_equal(ex.leaf_ids, L.leaf_ids)
    assert np.array_equal(ex.far_off, L.far_off)
    assert np.array_equal(ex.near_off, L.near_off)
    assert np.array_equal(ex.far_idx, L.far_idx)
    assert np.array_equal(ex.near_idx, L.near_idx)


def _rel(diff, ref):
    """|diff| / |ref| per row; 0 where both vanish, inf where only ref does."""
    with np.errstate(divide="ignore", invalid="ignore"):
        r = diff / ref
    r[(ref == 0) & (diff == 0)] = 0.0
    r[(ref == 0) & (diff != 0)] = np.inf
    return r


def rel_errors(ga, gphi, oa, ophi, rows=None):
    if rows is None:
        rows = np.arange(oa.shape[0])
    ea = _rel(np.linalg.norm(ga[rows] - oa[rows], axis=1), np.linalg.norm(oa[rows], axis=1))
    ep = _rel(np.abs(gphi[rows] - ophi[rows]), np.abs(ophi[rows]))
    return ea, ep


def fsum_force(m, a):
    return np.array([math.fsum(m * a[:, k]) for k in range(3)])


def split_forest(ex, sys_offset):
    """The export of a forest cut into one export per system, with cell ids,
    particle positions and caller indices made local to the system (the form
    the oracle gives for that system alone).  System k's cells are the
    contiguous pre-order range from its root (parent -1) to the next root."""
    from types import SimpleNamespace
    off = np.asarray(sys_offset, dtype=np.int64)
    ci = ex.cell_ints
    roots = np.nonzero(ci[:, 4] == -1)[0]
    assert roots.size == off.size - 1, (roots.size, off.size - 1)
    ends = np.append(roots[1:], ci.shape[0])
    leaf_bounds = np.searchsorted(ex.leaf_ids, np.append(roots, ci.shape[0]))
    out = []
    for k, (r0, r1) in enumerate(zip(roots, ends)):
        ints = ci[r0:r1].copy()
        ints[:, 0] -= off[k]
        for col in (2, 3, 4, 6):
            sel = ints[:, col] >= 0
            ints[sel, col] -= r0
        l0, l1 = leaf_bounds[k], leaf_bounds[k + 1]
        e = SimpleNamespace(perm=ex.perm[off[k]:off[k + 1]] - off[k], cell_ints=ints,
                            cell_reals=ex.cell_reals[r0:r1], leaf_ids=ex.leaf_ids[l0:l1] - r0,
                            far_off=None, far_idx=None, near_off=None, near_idx=None)
        if ex.far_off is not None:
            fo, no = ex.far_off[l0:l1 + 1], ex.near_off[l0:l1 + 1]
            e.far_idx = ex.far_idx[fo[0]:fo[-1]] - r0
            e.near_idx = ex.near_idx[no[0]:no[-1]] - r0
            e.far_off, e.near_off = fo - fo[0], no - no[0]
        out.append(e)
    return out
