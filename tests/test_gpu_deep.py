"""GPU parity of 63-bit keys (bh_config.max_level = 21): keys, permutation,
tree arrays and groups bit-exact against the oracle's 21-level path for both
orders; moments; group-walk, per-particle-walk and neighbour-search results
at the bars of the 30-bit suites; batched systems bit-identical to their
single evaluations; dense knots no longer leave oversized leaves."""
import numpy as np
import pytest

import workloads
from test_gpu_parity import MARGIN, _check_force, _cuda

pytestmark = pytest.mark.gpu

D = 21


@pytest.fixture(scope="module")
def bh():
    import torch
    assert torch.cuda.is_available()
    from paper_1112_4539_gb300 import _build
    _build.build()
    import paper_1112_4539_gb300 as m
    m.lib()
    return m


def _knotted(n, seed):
    # a clumpy set plus a knot of 400 particles inside 1e-4: at 10 levels the
    # knot is one oversized leaf
    rng = np.random.default_rng(seed)
    knot = np.concatenate([0.3 + 1e-4 * rng.random((400, 3)), np.full((400, 1), 1.0 / n)], 1)
    return np.concatenate([workloads.clumpy(n - 400, seed=seed), knot]).astype(np.float32)


SETS = [("plummer", 4096, 0, 8, 0), ("knotted", 30011, 2, 16, 0), ("knotted", 30011, 2, 8, 1),
        ("uniform", 65537, 7, 1, 0), ("sphere", 20001, 5, 16, 1)]


def _pos(kind, n, seed):
    return _knotted(n, seed) if kind == "knotted" else workloads.make(kind, n, seed)


@pytest.mark.parametrize("kind,n,seed,leaf,curve", SETS)
def test_keys_tree_groups_bit_exact(bh, orc, kind, n, seed, leaf, curve):
    pos = _pos(kind, n, seed)
    ctx = bh.Context(n, leaf_size=leaf, group_size=64, curve=curve, max_level=D)
    ctx.build(_cuda(pos))
    assert ctx.status() == 0
    b = orc.Built(pos, leaf, 64, 0.5, 1, curve=curve, max_level=D)
    keys = ctx.export("keys")
    assert keys.dtype == np.uint64
    np.testing.assert_array_equal(keys, b.skeys)
    np.testing.assert_array_equal(ctx.export("perm"), b.perm)
    np.testing.assert_array_equal(ctx.export("spos"), b.spos)
    t = b.tree
    np.testing.assert_array_equal(ctx.export("node_level"), t.level)
    np.testing.assert_array_equal(ctx.export("node_first"), t.first)
    np.testing.assert_array_equal(ctx.export("node_count"), t.count)
    np.testing.assert_array_equal(ctx.export("node_child"), t.child_first)
    np.testing.assert_array_equal(ctx.export("node_nchild"), t.nchild)
    np.testing.assert_array_equal(ctx.export("group_first"), b.g_first)
    np.testing.assert_array_equal(ctx.export("group_count"), b.g_count)
    st = ctx.stats()
    assert st["n_nodes"] == t.n_nodes
    assert st["max_leaf_count"] == int(t.count[t.nchild == 0].max())
    ctx.close()


def test_knot_leaves_split(bh):
    pos = _knotted(30011, 2)
    big = []
    for ml in (10, D):
        ctx = bh.Context(pos.shape[0], leaf_size=8, max_level=ml)
        ctx.build(_cuda(pos))
        big.append(ctx.stats()["max_leaf_count"])
        ctx.close()
    assert big[0] > 100 and big[1] <= 8


@pytest.mark.parametrize("order", [1, 2])
def test_moments(bh, orc, order):
    pos = _knotted(30011, 3)
    theta = 0.6
    ctx = bh.Context(pos.shape[0], leaf_size=8, group_size=64, order=order, max_level=D)
    ctx.build(_cuda(pos))
    ctx.moments(theta)
    assert ctx.status() == 0
    b = orc.Built(pos, 8, 64, theta, order, max_level=D)
    cm = ctx.export("com_m").astype(np.float64)
    ref, side = b.mom.com_m, b.mom.side
    np.testing.assert_allclose(cm[:, 3], ref[:, 3], rtol=2e-6)
    scale = np.abs(ref[:, :3]).max() + side[:, None]
    assert (np.abs(cm[:, :3] - ref[:, :3]) <= 2e-6 * scale).all()
    r_gpu = np.sqrt(ctx.export("seff").astype(np.float64))
    r_ref = np.sqrt(b.mom.s_eff)
    cscale = np.abs(ref[:, :3]).max(axis=1) + side
    assert (np.abs(r_gpu - r_ref) <= 1e-6 * r_ref + 4e-7 * cscale).all()
    if order == 2:
        q = ctx.export("quad").astype(np.float64)
        qs = b.mom.com_m[:, 3:4] * side[:, None] ** 2
        assert (np.abs(q - b.mom.quad) <= 1e-5 * qs + 1e-30).all()
    ctx.close()


@pytest.mark.parametrize("kind,n,seed,theta,eps,leaf,G,order,curve", [
    ("plummer", 4096, 0, 0.5, 0.01, 8, 64, 1, 0),
    ("knotted", 30011, 2, 0.6, 1e-3, 16, 96, 2, 0),
    ("knotted", 30011, 2, 0.5, 1e-3, 8, 64, 2, 1),
])
def test_group_walk_parity(bh, orc, kind, n, seed, theta, eps, leaf, G, order, curve):
    pos = _pos(kind, n, seed)
    ctx = bh.Context(n, leaf_size=leaf, group_size=G, order=order, curve=curve, max_level=D)
    got = ctx.evaluate(_cuda(pos), theta, eps).cpu().numpy().astype(np.float64)
    assert ctx.status() == 0
    ref, _ = orc.tree_force(pos, theta, eps, n_leaf=leaf, G=G, order=order, walk="group", curve=curve, max_level=D)
    _check_force(got, ref["out"], ref["margin"], a_abs=ref["a_abs"])
    st = ctx.stats()
    if (ref["margin"] >= MARGIN).all():
        assert st["n_pp"] == int(ref["n_pp"].sum()) and st["n_pc"] == int(ref["n_pc"].sum())
    ctx.close()


def test_particle_walk_and_neighbours(bh, orc):
    import torch
    pos = _knotted(20011, 4)
    n = pos.shape[0]
    ctx = bh.Context(n, leaf_size=8, order=2, max_level=D)
    got = ctx.evaluate(_cuda(pos), 0.5, 1e-3, walk="particle").cpu().numpy().astype(np.float64)
    assert ctx.status() == 0
    b = orc.Built(pos, 8, 32, 0.5, 2, max_level=D)
    ref = orc.force_particles(b.spos, b.perm, b.tree, b.mom, 1e-3)
    _check_force(got, ref["out"], ref["margin"], a_abs=ref["a_abs"])
    h = (0.005 + 0.05 * np.random.default_rng(4).random(n)).astype(np.float32)
    count, rho = ctx.neighbors(_cuda(pos), _cuda(h))
    c_ref, r_ref = orc.sph_density(pos, h)
    np.testing.assert_array_equal(count.cpu().numpy(), c_ref)
    np.testing.assert_allclose(rho.cpu().numpy(), r_ref, rtol=1e-5)
    ctx.close()


def test_batched_equals_single(bh):
    import torch
    sizes = [1, 2, 300, 65536, 0, 1025, 20000]
    parts = [workloads.plummer(s, seed=90 + k) if s else np.zeros((0, 4), np.float32) for k, s in enumerate(sizes)]
    pos = np.concatenate(parts)
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    x = _cuda(pos)
    ctx = bh.Context(pos.shape[0], leaf_size=8, group_size=96, order=2, max_systems=len(sizes), max_level=D)
    assert bh.bh_batch_layout(ctx.h, offs) == 0
    out = torch.full_like(x, float("nan"))
    assert bh.bh_force_batched(ctx.h, x, 0.5, 0.01, out) == 0
    assert ctx.status() == 0
    got = out.cpu().numpy()
    single = bh.Context(max(sizes), leaf_size=8, group_size=96, order=2, max_level=D)
    for k, s in enumerate(sizes):
        if s == 0:
            continue
        ref = single.evaluate(x[offs[k]:offs[k + 1]].contiguous(), 0.5, 0.01).cpu().numpy()
        np.testing.assert_array_equal(got[offs[k]:offs[k + 1]], ref)
    single.close()
    ctx.close()


def test_invalid_levels_rejected(bh):
    for ml in (0, 11, 22):
        with pytest.raises(bh.BhError):
            bh.Context(100, max_level=ml)
