"""GPU parity of the neighbour search and SPH density (general tree walk,
Sec. 4.3) against the oracle's all-pairs definition: neighbour counts are
integers decided by the same FP32 expression on both sides and must be
bit-exact; densities (FP32 sums of positive terms) within 1e-5 relative."""
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


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _radii(n, seed, lo=0.02, hi=0.1):
    return (lo + (hi - lo) * np.random.default_rng(seed).random(n)).astype(np.float32)


@pytest.mark.parametrize("kind,n,seed,leaf,G,curve", [
    ("clumpy", 20011, 3, 8, 64, 0),
    ("clumpy", 20011, 3, 16, 96, 1),
    ("plummer", 8192, 4, 1, 32, 0),
    ("uniform", 9001, 5, 8, 256, 0),
    ("sphere", 12000, 6, 16, 128, 1),
])
def test_counts_and_density_vs_oracle(bh, orc, kind, n, seed, leaf, G, curve):
    pos = workloads.make(kind, n, seed)
    h = _radii(n, seed)
    ctx = bh.Context(n, leaf_size=leaf, group_size=G, curve=curve)
    count, rho = ctx.neighbors(_cuda(pos), _cuda(h))
    assert ctx.status() == 0
    c_ref, r_ref = orc.sph_density(pos, h)
    np.testing.assert_array_equal(count.cpu().numpy(), c_ref)
    np.testing.assert_allclose(rho.cpu().numpy(), r_ref, rtol=1e-5)
    st = ctx.stats()
    assert st["n_pp"] >= int(c_ref.sum()) + n and st["n_pc"] == 0
    ctx.close()


def test_constant_radius_and_lattice(bh, orc):
    # cubic lattice with spacing 1/8 (exact coordinates), h = 4 spacings
    a, k = 0.125, 16
    g = np.arange(k, dtype=np.float32) * np.float32(a)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel(), np.full(X.size, 0.5, np.float32)], 1).astype(np.float32)
    ctx = bh.Context(pos.shape[0], leaf_size=8, group_size=64)
    count, rho = ctx.neighbors(_cuda(pos), 4 * a)
    c_ref, r_ref = orc.sph_density(pos, 4 * a)
    np.testing.assert_array_equal(count.cpu().numpy(), c_ref)
    np.testing.assert_allclose(rho.cpu().numpy(), r_ref, rtol=1e-5)
    ctx.close()


def test_degenerate_sets(bh, orc):
    ctx = bh.Context(1000, leaf_size=8, group_size=64)
    # one particle: no neighbour, density = m W(0)
    p1 = np.array([[0.3, 0.2, 0.1, 2.0]], np.float32)
    c, r = ctx.neighbors(_cuda(p1), 0.5)
    assert c.item() == 0 and r.item() == pytest.approx(2.0 * 8 / (np.pi * 0.125), rel=1e-6)
    # coincident particles: everyone neighbours everyone
    pc = np.tile(np.array([[0.5, 0.5, 0.5, 0.01]], np.float32), (777, 1))
    c, r = ctx.neighbors(_cuda(pc), 0.1)
    assert (c.cpu().numpy() == 776).all()
    np.testing.assert_allclose(r.cpu().numpy(), 777 * 0.01 * 8 / (np.pi * 1e-3), rtol=1e-5)
    # radius smaller than every separation: no neighbours
    pos = workloads.make("uniform", 999, 2)
    c, r = ctx.neighbors(_cuda(pos), 1e-6)
    c_ref, r_ref = orc.sph_density(pos, 1e-6)
    np.testing.assert_array_equal(c.cpu().numpy(), c_ref)
    ctx.close()


def test_errors(bh):
    import torch
    ctx = bh.Context(100)
    cnt = torch.empty(100, dtype=torch.int32, device="cuda:0")
    assert bh.tree_neighbors(ctx.h, 0.1, cnt) == bh.BH_ERR_STATE          # no tree yet
    x = _cuda(workloads.make("plummer", 100, 1))
    ctx.build(x)
    assert bh.tree_neighbors(ctx.h, 0.0, cnt) == bh.BH_ERR_INVALID
    assert bh.tree_neighbors(ctx.h, float("nan"), cnt) == bh.BH_ERR_INVALID
    h = torch.full((100,), 0.1, device="cuda:0")
    h[7] = float("nan")
    assert bh.tree_neighbors(ctx.h, h, cnt) == 0
    assert ctx.status() == bh.BH_ERR_NONFINITE
    ctx.close()
