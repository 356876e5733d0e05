"""GPU parity of the paper's per-particle walk (Sec. 4.4, Fig. 5, Appendix A).

The next links must equal the depth-first successor of every node (integer,
bit-exact).  Forces are compared with the oracle's per-particle walk on the
same particles at the bar of the group walk: 1e-5 relative per particle
(denominator floored at 1e-3 of the median |a| and at a tenth of the
particle's sum of term magnitudes), on every particle whose criterion
decisions all have a relative margin >= 1e-5; near-tie particles are only
checked to be valid tree results (within a few per cent).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5
MARGIN = 1e-5


@pytest.fixture(scope="module")
def bh():
    import torch
    assert torch.cuda.is_available()
    from paper_1112_4539_gb300 import _build
    _build.build()
    import paper_1112_4539_gb300 as m
    m.lib()
    return m


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _export(bh, ctx, what, dtype, count):
    import ctypes
    out = np.zeros(count, dtype=dtype)
    nb = ctypes.c_int64()
    rc = bh.lib().bh_export(ctx.h, bh.EXPORT[what], out.ctypes.data_as(ctypes.c_void_p), out.nbytes,
                            ctypes.byref(nb), None)
    assert rc == 0, rc
    return out[: nb.value // out.itemsize]


def _check(got, res, min_checked=0.85):
    ref, margin, a_abs = res["out"], res["margin"], res["a_abs"]
    a_ref = np.linalg.norm(ref[:, :3], axis=1)
    den = np.maximum(np.maximum(a_ref, 1e-3 * np.median(a_ref)), 0.1 * a_abs)
    ea = np.linalg.norm(got[:, :3] - ref[:, :3], axis=1) / den
    ep = np.abs(got[:, 3] - ref[:, 3]) / np.abs(ref[:, 3])
    ok = margin >= MARGIN
    assert ok.mean() >= min_checked, ok.mean()
    assert np.isfinite(got).all()
    assert ea[ok].max() <= TOL, ea[ok].max()
    assert ep[ok].max() <= TOL, ep[ok].max()
    if (~ok).any():
        assert ea[~ok].max() < 0.05 and ep[~ok].max() < 0.05
    return ok


@pytest.mark.parametrize("kind,n,seed,leaf", [("plummer", 4096, 0, 8), ("clumpy", 30011, 2, 16),
                                              ("uniform", 5000, 7, 1)])
def test_next_links_depth_first(bh, kind, n, seed, leaf):
    pos = workloads.make(kind, n, seed)
    ctx = bh.Context(n, leaf_size=leaf)
    x = _cuda(pos)
    out = ctx.evaluate(x, 0.5, 0.01, walk="particle")
    assert ctx.status() == 0 and np.isfinite(out.cpu().numpy()).all()
    nn = ctx.stats()["n_nodes"]
    child = _export(bh, ctx, "node_child", np.int32, nn)
    nch = _export(bh, ctx, "node_nchild", np.int32, nn)
    nxt = _export(bh, ctx, "next", np.int32, nn)
    # the depth-first order of the tree, restated: the successor of each
    # node's subtree is its next sibling, else its parent's successor
    want = np.full(nn, -2, np.int64)
    want[0] = -1
    stack = [0]
    while stack:
        v = stack.pop()
        for k in range(nch[v]):
            c = child[v] + k
            want[c] = c + 1 if k < nch[v] - 1 else want[v]
            stack.append(c)
    assert (want >= -1).all()
    np.testing.assert_array_equal(nxt, want)


@pytest.mark.parametrize("kind,n,seed,leaf,order,theta,eps", [
    ("plummer", 4096, 0, 8, 1, 0.5, 0.01),
    ("plummer", 4096, 0, 8, 2, 0.75, 0.01),
    ("clumpy", 30011, 2, 16, 2, 0.5, 1e-3),
    ("sphere", 20000, 5, 1, 1, 0.6, 0.01),
])
@pytest.mark.parametrize("unsoftened", [False, True])
def test_particle_walk_vs_oracle(bh, orc, kind, n, seed, leaf, order, theta, eps, unsoftened):
    pos = workloads.make(kind, n, seed)
    ctx = bh.Context(n, leaf_size=leaf, order=order)
    x = _cuda(pos)
    got = ctx.evaluate(x, theta, eps, walk="particle", unsoftened_cells=unsoftened).cpu().numpy()
    assert ctx.status() == 0
    st = ctx.stats()
    b = orc.Built(pos, leaf, 32, theta, order)
    res = orc.force_particles(b.spos, b.perm, b.tree, b.mom, eps, unsoftened_pc=unsoftened)
    ok = _check(got.astype(np.float64), res)
    # interaction counts: exact when no decision is a near tie
    want = int(res["n_pp"].sum() + res["n_pc"].sum())
    have = st["n_pp"] + st["n_pc"]
    if ok.all():
        assert (st["n_pp"], st["n_pc"]) == (int(res["n_pp"].sum()), int(res["n_pc"].sum()))
    else:
        assert abs(have - want) <= 1e-3 * want


def test_particle_walk_theta_to_zero_equals_direct(bh):
    import torch
    pos = workloads.make("plummer", 4096, 3)
    n, eps = pos.shape[0], 0.01
    ctx = bh.Context(n, leaf_size=8, order=2)
    x = _cuda(pos)
    got = ctx.evaluate(x, 1e-4, eps, walk="particle").cpu().numpy().astype(np.float64)
    st = ctx.stats()
    assert st["n_pc"] == 0 and st["n_pp"] == n * (n - 1)
    ref = torch.empty((n, 4), dtype=torch.float64, device="cuda:0")
    assert bh.direct_force(x, x, torch.arange(n, device="cuda:0"), eps, ref, 64) == 0
    ref = ref.cpu().numpy()
    a = np.linalg.norm(ref[:, :3], axis=1)
    ea = np.linalg.norm(got[:, :3] - ref[:, :3], axis=1) / np.maximum(a, 1e-3 * np.median(a))
    assert ea.max() < 1e-5
    assert (np.abs(got[:, 3] - ref[:, 3]) / np.abs(ref[:, 3])).max() < 1e-5


def test_particle_walk_small_and_errors(bh):
    import torch
    ctx = bh.Context(8, leaf_size=1)
    for n in (1, 2, 3):
        pos = workloads.make("plummer", 8, 1)[:n].copy()
        x = _cuda(pos)
        got = ctx.evaluate(x, 0.5, 0.0, walk="particle").cpu().numpy()
        assert ctx.status() == 0 and np.isfinite(got).all()
        if n == 1:
            assert (got == 0).all()
        if n == 2:
            d = pos[1, :3].astype(np.float64) - pos[0, :3]
            r = np.linalg.norm(d)
            np.testing.assert_allclose(got[0, :3], pos[1, 3] * d / r ** 3, rtol=1e-5)
            np.testing.assert_allclose(got[1, :3], -pos[0, 3] * d / r ** 3, rtol=1e-5)
    out = torch.empty((3, 4), device="cuda:0")
    assert bh.tree_force_particles(ctx.h, -1.0, out) == bh.BH_ERR_INVALID
    assert bh.lib().tree_force_particles(ctx.h, 0.01, 4, bh._dptr(out), None) == bh.BH_ERR_INVALID
    # individual softening without tree_softening after the build
    assert bh.lib().tree_force_particles(ctx.h, 0.01, 2, bh._dptr(out), None) == bh.BH_ERR_STATE
    fresh = bh.Context(8)
    assert bh.tree_force_particles(fresh.h, 0.01, out) == bh.BH_ERR_STATE
    fresh.close()
    ctx.close()
