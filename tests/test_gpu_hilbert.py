"""GPU parity of the Peano-Hilbert order (bh_config.curve = BH_CURVE_HILBERT).

Integer work is bit-exact against the oracle's Hilbert path: keys, sort
permutation, tree arrays and groups.  Moments follow the Morton bar (the
cell centres now come from the decoded key).  Forces of the group walk and
of the per-particle walk match the oracle at 1e-5 (margin-filtered), and the
batched path gives every system the same bits as its single evaluation.
"""
import numpy as np
import pytest

import workloads
from test_gpu_parity import MARGIN, _check_force, _cuda

pytestmark = pytest.mark.gpu

H = 1


@pytest.fixture(scope="module")
def bh():
    import torch
    assert torch.cuda.is_available()
    from paper_1112_4539_gb300 import _build
    _build.build()
    import paper_1112_4539_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("kind,n,seed,leaf", [("plummer", 4096, 0, 8), ("clumpy", 100003, 2, 16),
                                              ("uniform", 65537, 7, 1), ("sphere", 30001, 5, 8)])
def test_keys_tree_groups_bit_exact(bh, orc, kind, n, seed, leaf):
    pos = workloads.make(kind, n, seed)
    ctx = bh.Context(n, leaf_size=leaf, group_size=64, curve=H)
    ctx.build(_cuda(pos))
    assert ctx.status() == 0
    b = orc.Built(pos, leaf, 64, 0.5, 1, curve=H)
    np.testing.assert_array_equal(ctx.export("keys"), b.skeys)
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
    ctx.close()


@pytest.mark.parametrize("order", [1, 2])
def test_moments(bh, orc, order):
    pos = workloads.clumpy(60000, seed=6)
    theta = 0.6
    ctx = bh.Context(pos.shape[0], leaf_size=8, group_size=64, order=order, curve=H)
    ctx.build(_cuda(pos))
    ctx.moments(theta)
    assert ctx.status() == 0
    b = orc.Built(pos, 8, 64, theta, order, curve=H)
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


@pytest.mark.parametrize("kind,n,seed,theta,eps,leaf,G,order", [
    ("plummer", 4096, 0, 0.5, 0.01, 8, 64, 1),
    ("clumpy", 30007, 2, 0.6, 1e-3, 16, 96, 2),
    ("sphere", 10000, 4, 1.0, 0.01, 1, 32, 1),
])
def test_group_walk_parity(bh, orc, kind, n, seed, theta, eps, leaf, G, order):
    pos = workloads.make(kind, n, seed)
    ctx = bh.Context(n, leaf_size=leaf, group_size=G, order=order, curve=H)
    got = ctx.evaluate(_cuda(pos), theta, eps).cpu().numpy().astype(np.float64)
    assert ctx.status() == 0
    ref, _ = orc.tree_force(pos, theta, eps, n_leaf=leaf, G=G, order=order, walk="group", curve=H)
    _check_force(got, ref["out"], ref["margin"], a_abs=ref["a_abs"])
    st = ctx.stats()
    if (ref["margin"] >= MARGIN).all():
        assert st["n_pp"] == int(ref["n_pp"].sum()) and st["n_pc"] == int(ref["n_pc"].sum())
    ctx.close()


def test_particle_walk_parity(bh, orc):
    pos = workloads.make("clumpy", 30011, 2)
    ctx = bh.Context(pos.shape[0], leaf_size=16, order=2, curve=H)
    got = ctx.evaluate(_cuda(pos), 0.5, 1e-3, walk="particle").cpu().numpy().astype(np.float64)
    assert ctx.status() == 0
    b = orc.Built(pos, 16, 32, 0.5, 2, curve=H)
    ref = orc.force_particles(b.spos, b.perm, b.tree, b.mom, 1e-3)
    _check_force(got, ref["out"], ref["margin"], a_abs=ref["a_abs"])
    ctx.close()


def test_batched_equals_single(bh):
    import torch
    sizes = [1, 2, 300, 65536, 4096, 0, 1025, 20000]
    parts = [workloads.plummer(s, seed=70 + k) if s else np.zeros((0, 4), np.float32) for k, s in enumerate(sizes)]
    pos = np.concatenate(parts)
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    x = _cuda(pos)
    ctx = bh.Context(pos.shape[0], leaf_size=8, group_size=96, order=2, max_systems=len(sizes), curve=H)
    assert bh.bh_batch_layout(ctx.h, offs) == 0
    out = torch.full_like(x, float("nan"))
    assert bh.bh_force_batched(ctx.h, x, 0.5, 0.01, out) == 0
    assert ctx.status() == 0
    got = out.cpu().numpy()
    single = bh.Context(max(sizes), leaf_size=8, group_size=96, order=2, curve=H)
    for k, s in enumerate(sizes):
        if s == 0:
            continue
        ref = single.evaluate(x[offs[k]:offs[k + 1]].contiguous(), 0.5, 0.01).cpu().numpy()
        np.testing.assert_array_equal(got[offs[k]:offs[k + 1]], ref)
    single.close()
    ctx.close()


def test_invalid_curve_rejected(bh):
    with pytest.raises(bh.BhError):
        bh.Context(100, curve=2)
