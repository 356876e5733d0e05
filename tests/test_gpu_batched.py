"""Many independent systems in one evaluation: every system's forces equal
that system evaluated alone, bit for bit (same arithmetic at every step),
graph replay equals a direct call, and layout errors are reported."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bh():
    import torch
    assert torch.cuda.is_available()
    from paper_1112_4539_gb300 import _build
    _build.build()
    import paper_1112_4539_gb300 as m
    m.lib()
    return m


def _systems(sizes, seed=7):
    parts = [workloads.plummer(int(n), seed=seed * 1000 + k) if n > 0 else np.zeros((0, 4), np.float32)
             for k, n in enumerate(sizes)]
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    return np.concatenate(parts), offs


@pytest.mark.parametrize("order,G,leaf", [(1, 64, 8), (2, 96, 16), (1, 32, 1)])
def test_batched_equals_each_system_alone(bh, orc, order, G, leaf):
    import torch
    sizes = [1, 2, 7, 300, 65536, 4096, 0, 1025, 20000, 33, 5000, 65535]
    pos, offs = _systems(sizes)
    x = torch.from_numpy(pos).cuda()
    ctx = bh.Context(pos.shape[0], leaf_size=leaf, group_size=G, order=order, max_systems=len(sizes))
    assert bh.bh_batch_layout(ctx.h, offs) == 0
    out = torch.full_like(x, float("nan"))
    assert bh.bh_force_batched(ctx.h, x, 0.5, 0.01, out) == 0
    assert ctx.status() == 0
    st = ctx.stats()
    got = out.cpu().numpy()
    single = bh.Context(max(sizes), leaf_size=leaf, group_size=G, order=order)
    n_inter = 0
    for k, n in enumerate(sizes):
        if n == 0:
            continue
        xs = x[offs[k]:offs[k + 1]].contiguous()
        ref = single.evaluate(xs, 0.5, 0.01).cpu().numpy()
        s1 = single.stats()
        n_inter += s1["n_pp"] + s1["n_pc"]
        np.testing.assert_array_equal(got[offs[k]:offs[k + 1]], ref)
    assert st["n_pp"] + st["n_pc"] == n_inter
    single.close()
    # one system against the oracle as well
    k = 5
    sp = pos[offs[k]:offs[k + 1]]
    r, _ = orc.tree_force(sp, 0.5, 0.01, n_leaf=leaf, G=G, order=order)
    ok = r["margin"] >= 1e-5
    a = np.linalg.norm(r["out"][:, :3], axis=1)
    den = np.maximum(np.maximum(a, 1e-3 * np.median(a)), 0.1 * r["a_abs"])
    ea = np.linalg.norm(got[offs[k]:offs[k + 1], :3] - r["out"][:, :3], axis=1) / den
    assert ok.mean() > 0.9 and ea[ok].max() <= 1e-5
    ctx.close()


def test_graph_replay_equals_direct_call(bh):
    import torch
    sizes = workloads.batched_sizes(40, 1024, 65536, seed=3)
    pos, offs = _systems(sizes, seed=3)
    x = torch.from_numpy(pos).cuda()
    ctx = bh.Context(pos.shape[0], leaf_size=16, group_size=96, order=1, max_systems=40)
    assert bh.bh_batch_layout(ctx.h, offs) == 0
    a = torch.empty_like(x)
    assert bh.bh_force_batched(ctx.h, x, 0.5, 0.01, a) == 0
    b = torch.full_like(x, float("nan"))
    g = bh.BatchedGraph(ctx, x, 0.5, 0.01, b)
    for _ in range(2):
        b.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    assert ctx.status() == 0
    g.close()
    ctx.close()


def test_batched_layout_errors(bh):
    import torch
    ctx = bh.Context(200000, max_systems=4)
    assert bh.bh_batch_layout(ctx.h, np.array([0, 10, 70000])) == bh.BH_ERR_TOO_LARGE   # a system > 65536
    assert bh.bh_batch_layout(ctx.h, np.array([0, 10, 5])) == bh.BH_ERR_INVALID         # decreasing
    assert bh.bh_batch_layout(ctx.h, np.array([1, 10])) == bh.BH_ERR_INVALID             # not from 0
    assert bh.bh_batch_layout(ctx.h, np.arange(6) * 10) == bh.BH_ERR_TOO_LARGE           # 5 > max_systems
    x = torch.zeros((10, 4), device="cuda")
    assert bh.bh_force_batched(ctx.h, x, 0.5, 0.01, x) == bh.BH_ERR_STATE                # no layout yet
    assert bh.bh_batch_layout(ctx.h, np.array([0, 4, 10])) == 0
    assert bh.bh_force_batched(ctx.h, x, 0.0, 0.01, x) == bh.BH_ERR_INVALID
    ctx.close()
