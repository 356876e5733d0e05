"""Pins of the oracle's Peano-Hilbert ordering (the ordering Sec. 5 names as
better for locality than Morton's) against properties of the curve that its
code does not state: the first level visits the octants in reflected Gray-code
order, consecutive keys are face-adjacent cells at every depth, every octree
cell is one contiguous key range, and the octree read off Hilbert-sorted keys
is the Morton octree with its children reordered (same cells, same moments,
same per-particle forces)."""
import numpy as np
import pytest

import workloads

H, M = 1, 0


def test_first_level_is_gray_code(orc):
    for k in range(8):
        g = k ^ (k >> 1)  # reflected binary Gray code
        c = orc.cell_of_key(k << 27, H)
        assert tuple(v >> 9 for v in c) == ((g >> 2) & 1, (g >> 1) & 1, g & 1)
    assert orc.key_of_cell(0, 0, 0, H) == 0


def test_level3_curve_is_face_connected(orc):
    # the 512 level-3 cells, each through one of its level-10 cells
    cells = [(i, j, k) for i in range(8) for j in range(8) for k in range(8)]
    keys = np.array([orc.key_of_cell(i * 128 + 37, j * 128 + 5, k * 128 + 99, H) for i, j, k in cells])
    pref = keys >> 21
    assert sorted(pref.tolist()) == list(range(512))  # a bijection onto the level-3 prefixes
    order = np.argsort(pref)
    c = np.array(cells)[order]
    assert (np.abs(np.diff(c, axis=0)).sum(axis=1) == 1).all()


def test_deep_curve_face_connected_and_invertible(orc):
    rng = np.random.default_rng(11)
    for h in rng.integers(0, (1 << 30) - 1, 2000):
        a, b = np.array(orc.cell_of_key(h, H)), np.array(orc.cell_of_key(h + 1, H))
        assert np.abs(a - b).sum() == 1
        assert orc.key_of_cell(*a, H) == h
        assert (a < 1024).all()


@pytest.mark.parametrize("level", range(1, 10))
def test_cells_are_contiguous_key_ranges(orc, level):
    # two cells inside the same level-l cube share the top 3l key bits; two in
    # different cubes do not (so each cube is one contiguous range of keys)
    rng = np.random.default_rng(level)
    s = 10 - level
    for _ in range(300):
        base = rng.integers(0, 1 << level, 3)
        a = (base << s) + rng.integers(0, 1 << s, 3)
        b = (base << s) + rng.integers(0, 1 << s, 3)
        other = (rng.integers(0, 1 << level, 3) << s) + rng.integers(0, 1 << s, 3)
        ka, kb, ko = (orc.key_of_cell(*v, H) for v in (a, b, other))
        assert ka >> (3 * s) == kb >> (3 * s)
        assert (ko >> (3 * s) == ka >> (3 * s)) == bool((other >> s == base).all())


def _cells(b):
    """(level, cell coordinates at that level, count) of every node, from the
    Morton-ordered particles' integer cells computed with numpy."""
    box = b.box
    inv = np.float32(1024.0) / np.float32(box[3])
    q = (b.spos[:, :3].astype(np.float32) - box[:3].astype(np.float32)) * inv
    c = np.minimum(q.astype(np.int64), 1023)
    t = b.tree
    out = {}
    for v in range(t.n_nodes):
        l = int(t.level[v])
        key = (l,) + tuple(int(x) for x in c[t.first[v]] >> (10 - l))
        out[key] = v
    return out


@pytest.mark.parametrize("kind,n,seed,leaf", [("clumpy", 20000, 2, 8), ("plummer", 8192, 1, 1)])
def test_same_octree_for_both_orders(orc, kind, n, seed, leaf):
    pos = workloads.make(kind, n, seed)
    bm = orc.Built(pos, leaf, 32, 0.5, 2, curve=M)
    bh = orc.Built(pos, leaf, 32, 0.5, 2, curve=H)
    cm, ch = _cells(bm), _cells(bh)
    assert cm.keys() == ch.keys()
    vm = np.array([cm[k] for k in cm])
    vh = np.array([ch[k] for k in cm])
    np.testing.assert_array_equal(bm.tree.count[vm], bh.tree.count[vh])
    np.testing.assert_array_equal(bm.tree.nchild[vm], bh.tree.nchild[vh])
    np.testing.assert_allclose(bm.mom.com_m[vm], bh.mom.com_m[vh], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(bm.mom.s_eff[vm], bh.mom.s_eff[vh], rtol=1e-12)
    np.testing.assert_allclose(bm.mom.quad[vm], bh.mom.quad[vh], rtol=1e-9, atol=1e-16)
    # the Hilbert order keeps children face-adjacent: consecutive particles are closer
    step = lambda b: np.median(np.linalg.norm(np.diff(b.spos[:, :3].astype(np.float64), axis=0), axis=1))
    assert step(bh) <= step(bm) * 1.05


def test_particle_walk_forces_independent_of_order(orc):
    pos = workloads.make("plummer", 4096, 0)
    res = []
    for curve in (M, H):
        b = orc.Built(pos, 8, 32, 0.6, 2, curve=curve)
        res.append(orc.force_particles(b.spos, b.perm, b.tree, b.mom, 0.01))
    ok = (res[0]["margin"] > 1e-9) & (res[1]["margin"] > 1e-9)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(res[0]["out"][ok], res[1]["out"][ok], rtol=1e-11, atol=1e-13)
    np.testing.assert_array_equal(res[0]["n_pc"][ok], res[1]["n_pc"][ok])
