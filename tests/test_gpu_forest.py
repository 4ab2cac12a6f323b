"""A forest of independent systems in one handle (kdfmm_forest_build /
kdfmm_fmm_accel_batched) against the oracle run on each system alone: each
system's tree and lists bit for bit, forces within the precision's bound, and
the forest's results identical to separate single-system handles."""
import numpy as np
import pytest

from paper_2502_01496_gb300 import workloads as W

from gpu_common import (assert_lists_bit_exact, assert_tree_bit_exact, fsum_force, rel_errors,
                        split_forest)

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


def _cuda(a):
    import torch
    return None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")


def _concat(systems):
    x = np.concatenate([p.x for p in systems])
    m = np.concatenate([p.m for p in systems])
    h = None if systems[0].h is None else np.concatenate([p.h for p in systems])
    off = np.concatenate([[0], np.cumsum([p.n for p in systems])]).astype(np.int64)
    return x, m, h, off


def _run_forest(systems, theta, eps, n_leaf, prec, soft_kind):
    import torch
    from paper_2502_01496_gb300 import native
    x, m, h, off = _concat(systems)
    f = native.KdFmm(theta=0.5, eps=0.01, n_leaf=16, soft_kind=soft_kind, precision=prec)
    xd, md, hd = _cuda(x), _cuda(m), _cuda(h)
    a = torch.empty((x.shape[0], 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(x.shape[0], dtype=torch.float64, device="cuda")
    native.fmm_accel_batched(f.handle, xd, md, hd, off, f.params, a, phi, theta=theta, eps=eps,
                             n_leaf=n_leaf)
    f.n = x.shape[0]
    torch.cuda.synchronize()
    return f, off, a.cpu().numpy(), phi.cpu().numpy()


RAGGED = dict(
    sizes=[1, 2, 17, 300, 2049, 5000, 4097, 33],
    theta=[0.5, 0.0, 0.3, 0.7, 1.0, 0.5, 0.4, 0.6],
    eps=[0.01, 0.02, 0.0, 0.01, 0.005, 0.01, 0.03, 0.01],
    n_leaf=[16, 1, 8, 16, 32, 12, 16, 4],
)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_forest_matches_oracle_per_system(oracle, prec):
    sizes = RAGGED["sizes"]
    systems = [W.plummer(n, W.seed_for(3, 900 + k), eps=RAGGED["eps"][k])
               for k, n in enumerate(sizes)]
    # eps = 0 needs no two particles to coincide: Plummer samples never do
    f, off, ga, gphi = _run_forest(systems, RAGGED["theta"], RAGGED["eps"], RAGGED["n_leaf"],
                                   prec, 0)
    parts = split_forest(f.export(lists=True), off)
    tol = 1e-12 if prec == FP64 else 2e-5
    for k, ps in enumerate(systems):
        T = oracle.Tree(ps.x, ps.m, None, theta=RAGGED["theta"][k], n_leaf=RAGGED["n_leaf"][k],
                        soft_kind=0, eps=RAGGED["eps"][k])
        o = dict(order=T.order(), cells=T.cells(), lists=T.walk())
        g = {"ex": parts[k]}
        assert_tree_bit_exact(g, o)
        assert_lists_bit_exact(g, o)
        oa, ophi = T.eval()
        sl = slice(off[k], off[k + 1])
        if ps.n == 1:                       # a lone particle feels nothing
            assert np.all(ga[sl] == 0.0) and np.all(gphi[sl] == 0.0)
            continue
        ea, ep = rel_errors(ga[sl], gphi[sl], oa, ophi)
        assert ea.max() < tol and ep.max() < tol, (k, ea.max(), ep.max())


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("soft", ["plummer", "m4"])
def test_forest_equals_separate_handles(prec, soft):
    """Every phase works leaf by leaf inside its own system, so a system's
    results do not depend on the other systems of the batch: bit-identical to
    a handle holding that system alone."""
    import torch
    from paper_2502_01496_gb300 import native
    if soft == "plummer":
        systems = [W.plummer(n, W.seed_for(3, 950 + k)) for k, n in enumerate([3000, 700, 9000, 64])]
        kind = 0
    else:
        systems = [W.polytrope_binary(n, W.seed_for(3, 960 + k)) for k, n in enumerate([1500, 400, 3000])]
        kind = 1
    ns = len(systems)
    theta = np.linspace(0.3, 0.9, ns)
    n_leaf = np.array([16, 8, 32, 12][:ns], dtype=np.int32)
    eps = np.full(ns, 0.01)
    f, off, ga, gphi = _run_forest(systems, theta, eps, n_leaf, prec, kind)
    for k, ps in enumerate(systems):
        g = native.KdFmm(theta=float(theta[k]), eps=0.01, n_leaf=int(n_leaf[k]), soft_kind=kind,
                         precision=prec)
        g.build(_cuda(ps.x), _cuda(ps.m), _cuda(ps.h))
        a, phi = g.accel()
        torch.cuda.synchronize()
        sl = slice(off[k], off[k + 1])
        assert np.array_equal(a.cpu().numpy(), ga[sl]), k
        assert np.array_equal(phi.cpu().numpy(), gphi[sl]), k


@pytest.mark.slow
def test_batch_of_256_plummer_systems(oracle):
    """The full batch: 256 Plummer systems, N log-uniform in [2048, 262144],
    theta uniform in [0.3, 1], mixed precision.  Four systems (the smallest,
    the largest, two drawn at random) are checked against the oracle: tree and
    lists bit for bit, sampled leaves' forces within 2e-5, and for the two
    smaller ones the total force sum m a against the oracle's within 1e-3."""
    B = W.plummer_batch(256)
    n_leaf = np.full(256, 16, dtype=np.int32)
    f, off, ga, gphi = _run_forest(B.systems, B.theta, B.eps, n_leaf, MIXED, 0)
    assert np.isfinite(ga).all() and np.isfinite(gphi).all()
    parts = split_forest(f.export(lists=True), off)
    sizes = np.diff(off)
    rng = np.random.default_rng(4)
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), *rng.choice(256, 2, replace=False)})
    for k in pick:
        ps = B.systems[k]
        T = oracle.Tree(ps.x, ps.m, None, theta=float(B.theta[k]), n_leaf=16, soft_kind=0,
                        eps=float(B.eps[k]))
        o = dict(order=T.order(), cells=T.cells(), lists=T.walk())
        g = {"ex": parts[k]}
        assert_tree_bit_exact(g, o)
        assert_lists_bit_exact(g, o)
        sl = slice(off[k], off[k + 1])
        if ps.n <= 20000:
            oa, ophi = T.eval()
            ea, ep = rel_errors(ga[sl], gphi[sl], oa, ophi)
            F_g, F_o = fsum_force(ps.m, ga[sl]), fsum_force(ps.m, oa)
            assert np.linalg.norm(F_g - F_o) <= 1e-3 * np.linalg.norm(F_o), (k, F_g, F_o)
        else:
            leaf_ids = o["lists"].leaf_ids
            leaves = np.sort(rng.choice(leaf_ids, min(leaf_ids.size, 150), replace=False))
            oa, ophi = T.eval(leaves=leaves)
            rows = np.nonzero(np.isfinite(oa[:, 0]))[0]
            ea, ep = rel_errors(ga[sl], gphi[sl], oa, ophi, rows)
        assert ea.max() < 2e-5 and ep.max() < 2e-5, (k, ea.max(), ep.max())


@pytest.mark.parametrize("mode", ["exact", "two_pass"])
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_exact_lists_match_slots(oracle, monkeypatch, prec, mode):
    """Lists placed in reserved room (arena mode, taken when a few lists are
    far longer than the rest; forced here with buffers too small at first, so
    the walk also grows them and repeats) and two-pass lists (count, scan,
    fill: the fallback when the arena walk's scratch cannot be allocated) give
    the same lists and bit-identical forces as fixed slots; the adjoint agrees
    too."""
    import torch
    sizes = [4096, 700, 2500]
    systems = [W.plummer(n, W.seed_for(3, 980 + k)) for k, n in enumerate(sizes)]
    theta = [0.3, 0.6, 1.0]
    n_leaf = [16, 8, 32]
    eps = [0.01] * 3
    f1, off, ga1, gp1 = _run_forest(systems, theta, eps, n_leaf, prec, 0)
    ex1 = f1.export(lists=True)
    rng = np.random.default_rng(3)
    ab = _cuda(rng.standard_normal((off[-1], 3)))
    xb1, mb1 = f1.vjp(ab)
    monkeypatch.setenv("KDFMM_LIST_MODE", mode)
    f2, _, ga2, gp2 = _run_forest(systems, theta, eps, n_leaf, prec, 0)
    ex2 = f2.export(lists=True)
    xb2, mb2 = f2.vjp(ab)
    torch.cuda.synchronize()
    for name in ("leaf_ids", "far_off", "far_idx", "near_off", "near_idx"):
        assert np.array_equal(getattr(ex1, name), getattr(ex2, name)), name
    assert np.array_equal(ga1, ga2) and np.array_equal(gp1, gp2)
    xb1, xb2 = xb1.cpu().numpy(), xb2.cpu().numpy()
    mb1, mb2 = mb1.cpu().numpy(), mb2.cpu().numpy()
    assert np.abs(xb1 - xb2).max() <= 1e-12 * np.abs(xb1).max()
    assert np.abs(mb1 - mb2).max() <= 1e-12 * np.abs(mb1).max()
    parts = split_forest(ex2, off)
    for k, ps in enumerate(systems):
        T = oracle.Tree(ps.x, ps.m, None, theta=theta[k], n_leaf=n_leaf[k], soft_kind=0, eps=eps[k])
        assert_lists_bit_exact({"ex": parts[k]}, {"lists": T.walk()})


def _batched(f, x, m, off, theta, n_leaf, a, phi):
    from paper_2502_01496_gb300 import native
    native.fmm_accel_batched(f.handle, x, m, None, off, f.params, a, phi, theta=theta,
                             eps=np.full(len(off) - 1, 0.01), n_leaf=n_leaf)


@pytest.mark.parametrize("list_mode", ["slots", "arena"])
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_captured_graph_replays_the_eager_evaluation(monkeypatch, prec, list_mode):
    """Repeated batched calls on the same buffers: the first runs eagerly and
    captures a graph, later ones replay it.  Replays give the eager bits, and
    a replay whose trees outgrow the graph (longer lists after theta drops,
    other system sizes) falls back to the eager path with the same results as
    a handle that never used a graph; with fixed list slots and with lists
    placed in reserved room (arena mode)."""
    import torch
    from paper_2502_01496_gb300 import native
    if list_mode == "arena":
        monkeypatch.setenv("KDFMM_LIST_MODE", "exact")
    systems = [W.plummer(n, W.seed_for(3, 990 + k)) for k, n in enumerate([5000, 3000, 1200, 6000])]
    x0, m0, _, off = _concat(systems)
    n = x0.shape[0]
    x, m = _cuda(x0), _cuda(m0)
    a = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    n_leaf = np.array([16, 12, 8, 16], dtype=np.int32)

    def reference(theta, offs):
        monkeypatch.setenv("KDFMM_GRAPH", "0")
        g = native.KdFmm(theta=0.5, eps=0.01, n_leaf=16, soft_kind=0, precision=prec)
        ar = torch.empty_like(a)
        pr = torch.empty_like(phi)
        _batched(g, x, m, offs, theta, n_leaf, ar, pr)
        torch.cuda.synchronize()
        monkeypatch.delenv("KDFMM_GRAPH")
        return ar.cpu().numpy(), pr.cpu().numpy(), g.stats()

    f = native.KdFmm(theta=0.5, eps=0.01, n_leaf=16, soft_kind=0, precision=prec)
    cases = [(np.full(4, 1.0), off), (np.full(4, 1.0), off), (np.full(4, 1.0), off),
             (np.array([0.3, 0.4, 0.35, 0.3]), off),                       # longer lists
             (np.array([0.3, 0.4, 0.35, 0.3]), off),
             (np.full(4, 0.6), np.array([0, 200, 9000, 9100, n], dtype=np.int64))]   # other sizes
    for theta, offs in cases:
        _batched(f, x, m, offs, theta, n_leaf, a, phi)
        torch.cuda.synchronize()
        ra, rp, rst = reference(theta, offs)
        assert np.array_equal(a.cpu().numpy(), ra)
        assert np.array_equal(phi.cpu().numpy(), rp)
        st = f.stats()
        for key in ("ncells", "nleaves", "depth", "nfar", "nnear", "np2p"):
            assert st[key] == rst[key], (key, st[key], rst[key])


@pytest.mark.parametrize("list_mode", ["slots", "arena"])
def test_replay_with_more_leaves_than_captured_is_redone(monkeypatch, list_mode):
    """A graph captured on a jittered 32^3 lattice (cuts through the centre of
    mass halve it exactly: 2048 leaves of 16, so the graph covers 2048 * 1.25
    + 64 = 2624) and replayed on the same buffers holding a Plummer sphere of
    the same size (2914 leaves): the walk, M2L and P2P launches of the graph
    stop at 2624 leaves, so the replay must be redone eagerly, with the bits
    of a handle that never used a graph."""
    import torch
    from paper_2502_01496_gb300 import native
    if list_mode == "arena":
        monkeypatch.setenv("KDFMM_LIST_MODE", "exact")
    g1 = np.arange(32, dtype=np.float64) / 32.0
    X, Y, Z = np.meshgrid(g1, g1, g1, indexing="ij")
    lattice = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    lattice += np.random.default_rng(3).uniform(-1e-4, 1e-4, lattice.shape)
    sphere = W.plummer(32768, W.seed_for(0, 98))
    n = 32768
    off = np.array([0, n], dtype=np.int64)
    x, m = _cuda(lattice), _cuda(np.full(n, 1.0 / n))
    a = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    theta, n_leaf = np.array([0.5]), np.array([16], dtype=np.int32)
    f = native.KdFmm(theta=0.5, eps=0.01, n_leaf=16, soft_kind=0, precision=MIXED)
    for _ in range(2):                                 # eager + capture, then a replay
        _batched(f, x, m, off, theta, n_leaf, a, phi)
    torch.cuda.synchronize()
    assert f.stats()["nleaves"] == 2048
    x.copy_(_cuda(sphere.x))                           # same buffers, another tree
    _batched(f, x, m, off, theta, n_leaf, a, phi)
    torch.cuda.synchronize()
    monkeypatch.setenv("KDFMM_GRAPH", "0")
    g = native.KdFmm(theta=0.5, eps=0.01, n_leaf=16, soft_kind=0, precision=MIXED)
    ar, pr = torch.empty_like(a), torch.empty_like(phi)
    _batched(g, x, m, off, theta, n_leaf, ar, pr)
    torch.cuda.synchronize()
    st, rst = f.stats(), g.stats()
    assert rst["nleaves"] > 2624, rst
    for key in ("ncells", "nleaves", "nfar", "nnear", "np2p"):
        assert st[key] == rst[key], (key, st[key], rst[key])
    assert torch.equal(a, ar) and torch.equal(phi, pr)
