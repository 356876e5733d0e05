"""Pins of the FP64 CPU oracle against things other than itself.

Each test ties an oracle function to the paper, to mathematics or to an
independent routine: closed forms (two-body, truncated Plummer sphere),
conservation laws, hand-computed keys, library routines (numpy stable sort),
a brute-force restatement of the tree definition, identities the oracle does
not use (parallel-axis theorem), finite differences, the textbook traceless
quadrupole, convergence orders, and the paper's own error magnitudes
(Sec. 5, Table ERR_a) as an order-of-magnitude check.
"""
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Eq. (1)

def test_two_body_closed_form(orc):
    # Eq. (1) for two bodies: |a_1| = m2 d / (d^2 + eps^2)^1.5 toward body 2,
    # phi_1 = -m2 / sqrt(d^2 + eps^2).
    d, eps, m1, m2 = 0.75, 0.1, 0.25, 2.0
    p = np.array([[0, 0, 0, m1], [d, 0, 0, m2]], np.float32)
    out = orc.direct(p, eps=eps)
    h = (d * d + eps * eps) ** 0.5
    np.testing.assert_allclose(out[0], [m2 * d / h ** 3, 0, 0, -m2 / h], rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(out[1], [-m1 * d / h ** 3, 0, 0, -m1 / h], rtol=1e-14, atol=1e-300)


def test_direct_momentum_conservation(orc):
    p = workloads.plummer(2048, seed=5)
    out = orc.direct(p, eps=0.01)
    m = p[:, 3].astype(np.float64)
    tot = (m[:, None] * out[:, :3]).sum(axis=0)
    scale = (m * np.linalg.norm(out[:, :3], axis=1)).sum()
    assert np.linalg.norm(tot) <= 1e-12 * scale


def test_direct_gradient_of_potential(orc):
    # a = -grad(phi) at a field point (not one of the sources), central differences.
    p = workloads.plummer(64, seed=7)
    x0 = np.array([0.3, -0.2, 0.5], np.float64)
    h = 1.0 / 1024  # exactly representable, so x0 +- h e_k are exact float32 steps
    x0 = np.round(x0 * 1024) / 1024
    tgt = np.zeros((7, 4), np.float32)
    tgt[:, :3] = x0
    for k in range(3):
        tgt[1 + 2 * k, k] += h
        tgt[2 + 2 * k, k] -= h
    out = orc.direct(p, tgt, self_idx=np.full(7, -1, np.int64), eps=0.05)
    grad = np.array([(out[1 + 2 * k, 3] - out[2 + 2 * k, 3]) / (2 * h) for k in range(3)])
    np.testing.assert_allclose(-grad, out[0, :3], rtol=2e-5)


def _plummer_truncated(r, R=20.0):
    f = R ** 3 / (R * R + 1) ** 1.5
    phi_p = lambda x: -1.0 / np.sqrt(x * x + 1)
    phi = (phi_p(r) - phi_p(R)) / f - 1.0 / R
    amag = r / (f * (r * r + 1) ** 1.5)
    return phi, amag


def test_plummer_closed_form(orc):
    # Truncated, renormalised Plummer sphere: per radial bin, the mean inward
    # radial acceleration (unbiased by the random small-scale field, unlike |a|)
    # and the median potential against the closed form (statistical pin).
    n = 16384
    p = workloads.plummer(n, seed=11)
    out = orc.direct(p, eps=0.01)
    r = np.linalg.norm(p[:, :3].astype(np.float64), axis=1)
    ar = -(out[:, :3] * p[:, :3].astype(np.float64)).sum(1) / r
    # Tolerances follow the sampling noise of the enclosed mass (about 400
    # particles inside r = 0.3 at this N): 12% in the innermost bin, 5% beyond.
    edges = np.array([0.2, 0.4, 0.7, 1.0, 1.5, 2.0, 3.0])
    for lo, hi in zip(edges[:-1], edges[1:]):
        tol_a = 0.12 if lo < 0.3 else 0.05
        sel = (r >= lo) & (r < hi)
        assert sel.sum() > 200
        phi_t, a_t = _plummer_truncated(r[sel])
        ra = np.mean(ar[sel]) / np.mean(a_t)
        rp = np.median(out[sel, 3] / phi_t)
        assert abs(ra - 1) < tol_a, (lo, hi, ra)
        assert abs(rp - 1) < 0.02, (lo, hi, rp)


def test_direct_radial_attraction(orc):
    # Attractive sign: acceleration points toward the Plummer centre on average.
    p = workloads.plummer(4096, seed=12)
    out = orc.direct(p, eps=0.01)
    x = p[:, :3].astype(np.float64)
    cosang = -(out[:, :3] * x).sum(1) / (np.linalg.norm(out[:, :3], axis=1) * np.linalg.norm(x, axis=1))
    assert np.median(cosang) > 0.95
    assert (out[:, 3] < 0).all()


# ------------------------------------------------------ box, keys, sort

def test_bbox_matches_numpy(orc):
    p = workloads.clumpy(5000, seed=3)
    box = orc.bbox(p)
    lo = p[:, :3].min(0)
    ext = (p[:, :3].max(0) - lo).astype(np.float32)
    np.testing.assert_array_equal(box[:3], lo)
    assert box[3] == ext.max()


def test_bbox_degenerate(orc):
    p = np.tile(np.array([[0.5, -2.0, 3.0, 1.0]], np.float32), (10, 1))
    box = orc.bbox(p)
    np.testing.assert_array_equal(box, np.array([0.5, -2.0, 3.0, 1.0], np.float32))


def test_morton_golden(orc):
    rows = []
    with open(os.path.join(GOLDEN, "morton_keys.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    assert len(rows) >= 10
    for r in rows:
        x = np.array([[float(r[0]), float(r[1]), float(r[2]), 1.0]], np.float32)
        box = np.array([float(v) for v in r[3:7]], np.float32)
        k = orc.keys(x, box)
        assert int(k[0]) == int(r[7]), (r, int(k[0]))


def _interleave_py(cx, cy, cz):
    # bit string interleave, most significant triple first (independent formulation)
    bx, by, bz = format(cx, "010b"), format(cy, "010b"), format(cz, "010b")
    return int("".join(bx[i] + by[i] + bz[i] for i in range(10)), 2)


def test_morton_random_vs_independent(orc):
    rng = np.random.default_rng(0)
    p = np.zeros((3000, 4), np.float32)
    p[:, :3] = rng.uniform(-3, 5, (3000, 3)).astype(np.float32)
    box = orc.bbox(p)
    k = orc.keys(p, box)
    inv = np.float32(1024.0) / box[3]
    for i in range(0, 3000, 7):
        c = []
        for a in range(3):
            q = np.float32(np.float32(p[i, a] - box[a]) * inv)
            c.append(min(int(q), 1023))
        assert int(k[i]) == _interleave_py(*c)


def test_sort_matches_numpy_stable(orc):
    rng = np.random.default_rng(1)
    keys = rng.integers(0, 50, 20000).astype(np.uint32)  # many ties
    perm = orc.sort(keys)
    np.testing.assert_array_equal(perm, np.argsort(keys, kind="stable").astype(np.uint32))
    keys = rng.integers(0, 2 ** 30, 20001).astype(np.uint32)
    np.testing.assert_array_equal(orc.sort(keys), np.argsort(keys, kind="stable").astype(np.uint32))
    assert orc.sort(np.zeros(0, np.uint32)).shape == (0,)


# ------------------------------------------------------------- tree

def _tree_brute(skeys, n_leaf, max_level=10):
    """Definition restated: node = non-empty level-l cell whose parent cell has
    > n_leaf particles; sorted by (level, first)."""
    nodes = []
    n = skeys.shape[0]
    parent_count = None
    for l in range(max_level + 1):
        pref = (skeys.astype(np.uint64) >> np.uint64(3 * (max_level - l))).astype(np.int64)
        u, first, cnt = np.unique(pref, return_index=True, return_counts=True)
        counts = dict(zip(u.tolist(), cnt.tolist()))
        for pr, fi, c in zip(u.tolist(), first.tolist(), cnt.tolist()):
            if l == 0 or parent_count[pr >> 3] > n_leaf:
                nodes.append((l, fi, c, pr))
        parent_count = counts
    nodes.sort(key=lambda t: (t[0], t[1]))
    return nodes


@pytest.mark.parametrize("max_level", [10, 21])
@pytest.mark.parametrize("n_leaf", [1, 4, 8, 16])
def test_tree_matches_definition(orc, n_leaf, max_level):
    p = workloads.clumpy(3000, seed=4)
    box = orc.bbox(p)
    k = orc.keys(p, box, max_level=max_level)
    sk = k[orc.sort(k)]
    t = orc.tree_build(sk, n_leaf, max_level)
    ref = _tree_brute(sk, n_leaf, max_level)
    assert t.n_nodes == len(ref)
    np.testing.assert_array_equal(t.level, [r[0] for r in ref])
    np.testing.assert_array_equal(t.first, [r[1] for r in ref])
    np.testing.assert_array_equal(t.count, [r[2] for r in ref])
    pref = np.array([r[3] for r in ref], np.int64)
    for v in range(t.n_nodes):
        leaf = t.count[v] <= n_leaf or t.level[v] == max_level
        assert (t.nchild[v] == 0) == leaf
        if not leaf:
            ch = np.arange(t.child_first[v], t.child_first[v] + t.nchild[v])
            assert (t.level[ch] == t.level[v] + 1).all()
            assert ((pref[ch] >> 3) == pref[v]).all()
            assert t.count[ch].sum() == t.count[v]
            assert t.first[ch[0]] == t.first[v]
    # leaves partition the particles in order
    leaves = np.nonzero(t.nchild == 0)[0]
    lf = np.sort(t.first[leaves])
    order = np.argsort(t.first[leaves])
    ends = (t.first[leaves] + t.count[leaves])[order]
    assert lf[0] == 0 and ends[-1] == sk.shape[0]
    np.testing.assert_array_equal(lf[1:], ends[:-1])
    assert t.n_nodes <= orc.node_capacity(sk.shape[0], n_leaf, max_level)


def test_tree_coincident_particles(orc):
    p = np.tile(np.array([[1.0, 2.0, 3.0, 0.1]], np.float32), (20, 1))
    box = orc.bbox(p)
    k = orc.keys(p, box)
    assert (k == 0).all()
    t = orc.tree_build(k, 8)
    # a chain of single-child nodes down to one level-10 leaf holding all 20
    assert t.n_nodes == 11
    assert t.level[-1] == 10 and t.count[-1] == 20 and t.nchild[-1] == 0


def test_tree_empty_and_single(orc):
    t = orc.tree_build(np.zeros(0, np.uint32), 8)
    assert t.n_nodes == 0
    t = orc.tree_build(np.array([12345], np.uint32), 8)
    assert t.n_nodes == 1 and t.count[0] == 1 and t.nchild[0] == 0


# ---------------------------------------------------------- moments

def _built(orc, p, n_leaf=8, theta=0.5, order=2):
    box = orc.bbox(p)
    k = orc.keys(p, box)
    perm = orc.sort(k)
    sk, sp = k[perm], p[perm]
    t = orc.tree_build(sk, n_leaf)
    m = orc.moments(sp, sk, t, box, theta, order)
    return box, perm, sk, sp, t, m


def test_moments_root_and_parallel_axis(orc):
    p = workloads.plummer(4000, seed=8)
    box, perm, sk, sp, t, m = _built(orc, p)
    x = p[:, :3].astype(np.float64)
    w = p[:, 3].astype(np.float64)
    assert abs(m.com_m[0, 3] - w.sum()) < 1e-12
    np.testing.assert_allclose(m.com_m[0, :3], (w[:, None] * x).sum(0) / w.sum(), atol=1e-13)
    # parallel-axis theorem (not used by the oracle, which sums each node directly)
    for v in np.nonzero(t.nchild > 0)[0][:400]:
        ch = np.arange(t.child_first[v], t.child_first[v] + t.nchild[v])
        cp = m.com_m[v, :3]
        I = np.zeros(6)
        for c in ch:
            d = m.com_m[c, :3] - cp
            Mc = m.com_m[c, 3]
            I += m.quad[c] + Mc * np.array([d[0] * d[0], d[1] * d[1], d[2] * d[2],
                                            d[0] * d[1], d[0] * d[2], d[1] * d[2]])
        np.testing.assert_allclose(I, m.quad[v], rtol=1e-9, atol=1e-15 * m.com_m[v, 3])
        # mass is additive
        assert abs(m.com_m[ch, 3].sum() - m.com_m[v, 3]) <= 1e-14


def test_massless_node_takes_cell_centre(orc):
    # R14: a node of massless particles has the geometric centre of its cell as
    # centre of mass, so s = 0 and S_eff = (l / theta)^2.  Box: origin 0.1,
    # side 0.8; the massless pair sits in the level-1 cell with origin 0.1 and
    # side 0.4, centre 0.3 on each axis.
    p = np.array([[0.1, 0.1, 0.1, 0.0], [0.125, 0.1, 0.1, 0.0], [0.9, 0.9, 0.9, 1.0]], np.float32)
    box, perm, sk, sp, t, m = _built(orc, p, n_leaf=1, theta=0.5)
    v = [i for i in range(t.n_nodes) if t.level[i] == 1 and t.count[i] == 2][0]
    assert m.com_m[v, 3] == 0.0
    np.testing.assert_allclose(m.com_m[v, :3], [0.3, 0.3, 0.3], rtol=0, atol=1e-7)
    side = float(box[3]) / 2
    assert abs(m.s_eff[v] - (side / 0.5) ** 2) < 1e-12


def test_s_eff_hand_example(orc):
    # Eq. (2) for a hand-made case: box [0,4]^3 (origin 0, L = 4).  Particles at
    # (0.5,0.5,0.5) m=3 and (1.5,0.5,0.5) m=1.  With n_leaf = 1 the level-1
    # cell [0,2]^3 holds both: centre (1,1,1), COM (0.75,0.5,0.5),
    # s = sqrt(0.0625 + 0.25 + 0.25) = 0.75, l = 2, theta = 0.5:
    # S_eff = (2/0.5 + 0.75)^2 = 22.5625.  A far particle at (4,4,4) fixes L = 4.
    # The level-1 cell [2,4]x[0,2]x[0,2] (cell coordinates (1,0,0), centre
    # (3,1,1)) holds (2.5,0.5,0.5) and (3.5,1.5,0.5), m = 1: COM (3,1,0.5),
    # s = 0.5, S_eff = (4 + 0.5)^2 = 20.25; its centre tells the axes apart.
    p = np.array([[0.5, 0.5, 0.5, 3.0], [1.5, 0.5, 0.5, 1.0], [4.0, 4.0, 4.0, 1.0],
                  [2.5, 0.5, 0.5, 1.0], [3.5, 1.5, 0.5, 1.0]], np.float32)
    p0 = np.array([[0.0, 0.0, 0.0, 0.0]], np.float32)
    p = np.concatenate([p0, p])  # massless particle at the origin fixes xmin = 0
    box, perm, sk, sp, t, m = _built(orc, p, n_leaf=1, theta=0.5)
    assert tuple(box) == (0.0, 0.0, 0.0, 4.0)
    v = [i for i in range(t.n_nodes) if t.level[i] == 1 and t.count[i] == 3][0]
    np.testing.assert_allclose(m.com_m[v], [0.75, 0.5, 0.5, 4.0], rtol=1e-15)
    assert abs(m.side[v] - 2.0) < 1e-15
    assert abs(m.s_eff[v] - 22.5625) < 1e-12
    v2 = [i for i in range(t.n_nodes) if t.level[i] == 1 and t.count[i] == 2][0]
    np.testing.assert_allclose(m.com_m[v2], [3.0, 1.0, 0.5, 2.0], rtol=1e-15)
    assert abs(m.s_eff[v2] - 20.25) < 1e-12
    # root: l = 4, centre (2,2,2), COM = (1.5+1.5+4+2.5+3.5, 1.5+0.5+4+0.5+1.5, 1.5+0.5+4+0.5+0.5)/7
    com0 = np.array([13.0, 8.0, 7.0]) / 7.0
    s0 = np.linalg.norm(com0 - 2.0)
    assert abs(m.s_eff[0] - (4 / 0.5 + s0) ** 2) < 1e-12


# ------------------------------------------------------------- groups

@pytest.mark.parametrize("G", [8, 32, 64, 256])
def test_groups_partition(orc, G):
    p = workloads.clumpy(6000, seed=9)
    box, perm, sk, sp, t, m = _built(orc, p, n_leaf=8)
    gf, gc = orc.groups(t, G)
    assert gf[0] == 0 and (gf[:-1] + gc[:-1] == gf[1:]).all() and gf[-1] + gc[-1] == 6000
    assert (gc >= 1).all() and (gc <= G).all()
    # every group is a run of whole sibling nodes of one parent, or a chunk of one leaf
    node_at = {(int(t.first[v]), int(t.count[v])): v for v in range(t.n_nodes)}
    parent = np.full(t.n_nodes, -1)
    for v in range(t.n_nodes):
        for c in range(t.child_first[v], t.child_first[v] + t.nchild[v]):
            parent[c] = v
    for f, c in zip(gf.tolist(), gc.tolist()):
        if (f, c) in node_at:
            continue
        # find sibling nodes whose ranges tile [f, f+c)
        k, sib = f, []
        while k < f + c:
            cands = [v for v in range(t.n_nodes) if t.first[v] == k and t.count[v] <= G
                     and t.first[v] + t.count[v] <= f + c]
            if not cands:
                break
            v = min(cands, key=lambda u: t.level[u])
            sib.append(v)
            k += t.count[v]
        if k == f + c and len({parent[v] for v in sib}) == 1:
            continue
        # else: a chunk of an oversized leaf
        leaf = [v for v in range(t.n_nodes) if t.nchild[v] == 0 and t.first[v] <= f
                and f + c <= t.first[v] + t.count[v] and t.count[v] > G]
        assert leaf, (f, c)


@pytest.mark.parametrize("n_leaf,G", [(8, 32), (64, 32)])
def test_groups_cut_oversized_leaves_into_chunks_of_G(orc, n_leaf, G):
    # a leaf holding more than G particles (a level-10 cell of 200 coincident
    # particles, or any leaf when n_leaf > G) becomes the groups
    # [first + kG, first + min((k+1)G, count)), k = 0, 1, ...
    knot = np.concatenate([np.full((200, 3), 0.3), np.full((200, 1), 1e-4)], 1)
    p = np.concatenate([workloads.clumpy(3000, seed=20), knot]).astype(np.float32)
    box, perm, sk, sp, t, m = _built(orc, p, n_leaf=n_leaf)
    gf, gc = orc.groups(t, G)
    groups = set(zip(gf.tolist(), gc.tolist()))
    big = [v for v in range(t.n_nodes) if t.nchild[v] == 0 and t.count[v] > G]
    assert big
    for v in big:
        f, c = int(t.first[v]), int(t.count[v])
        for k in range(0, c, G):
            assert (f + k, min(G, c - k)) in groups, (v, k)


def test_groups_of_a_root_leaf(orc):
    # n <= n_leaf: the root is the only node, a leaf; with n > G it is cut into
    # chunks of G, the last one short
    p = workloads.plummer(50, seed=24)
    box, perm, sk, sp, t, m = _built(orc, p, n_leaf=64)
    assert t.n_nodes == 1 and t.nchild[0] == 0
    gf, gc = orc.groups(t, 32)
    assert list(zip(gf.tolist(), gc.tolist())) == [(0, 32), (32, 18)]
    gf, gc = orc.groups(t, 64)
    assert list(zip(gf.tolist(), gc.tolist())) == [(0, 50)]


def test_groups_greedy_maximal(orc):
    p = workloads.plummer(5000, seed=10)
    box, perm, sk, sp, t, m = _built(orc, p, n_leaf=8)
    G = 32
    gf, gc = orc.groups(t, G)
    starts = set(gf.tolist())
    # for each parent with count > G: a run break between two <=G siblings
    # happens only when the next sibling does not fit
    for v in range(t.n_nodes):
        if t.nchild[v] == 0 or t.count[v] <= G:
            continue
        run = 0
        for c in range(t.child_first[v], t.child_first[v] + t.nchild[v]):
            if t.count[c] > G:
                run = 0
                continue
            if int(t.first[c]) in starts and run > 0:
                assert run + t.count[c] > G
                run = t.count[c]
            else:
                run += t.count[c]


# ------------------------------------------------------- tree forces

@pytest.mark.parametrize("walk", ["group", "particle"])
def test_theta_to_zero_equals_direct(orc, walk):
    p = workloads.plummer(3000, seed=13)
    d = orc.direct(p, eps=0.01)
    res, b = orc.tree_force(p, theta=1e-4, eps=0.01, n_leaf=8, G=32, order=2, walk=walk)
    ea, ep = orc.rel_err(res["out"], d)
    assert ea.max() < 1e-12 and ep.max() < 1e-12
    assert (res["n_pc"] == 0).all()
    assert (res["n_pp"] == 2999).all()


def test_group_criterion_is_conservative(orc):
    p = workloads.clumpy(4000, seed=14)
    box, perm, sk, sp, t, m = _built(orc, p, n_leaf=8, theta=0.6)
    gf, gc = orc.groups(t, 32)
    for g in range(0, gf.shape[0], max(1, gf.shape[0] // 40)):
        pc, pp = orc.group_lists(sp, t, m, gf[g], gc[g])
        mem = sp[gf[g]:gf[g] + gc[g], :3].astype(np.float64)
        for v in pc:
            d2 = ((mem - m.com_m[v, :3]) ** 2).sum(1)
            assert (d2 > m.s_eff[v]).all()
        # opened leaves plus accepted nodes cover every particle exactly once
        cover = np.zeros(4000, np.int64)
        for v in list(pc) + list(pp):
            cover[t.first[v]:t.first[v] + t.count[v]] += 1
        assert (cover == 1).all()


def test_error_magnitude_and_ordering(orc):
    # Order-of-magnitude check against Table ERR_a (monopole, modified criterion,
    # theta = 0.5: mean a_error 1.4e-3 .. 2.0e-3 on the paper's disk galaxy),
    # and the expected orderings: error grows with theta, the quadrupole beats
    # the monopole, the conservative group criterion beats the per-particle one.
    n = 8192
    p = workloads.plummer(n, seed=15)
    d = orc.direct(p, eps=0.01)
    errs = {}
    for th in (0.3, 0.5, 0.75):
        for order in (1, 2):
            for walk in ("particle", "group"):
                res, _ = orc.tree_force(p, th, 0.01, order=order, walk=walk)
                ea, ep = orc.rel_err(res["out"], d)
                errs[th, order, walk] = (ea.mean(), ep.mean())
    a05 = errs[0.5, 1, "particle"][0]
    assert 3e-4 < a05 < 8e-3
    assert 3e-5 < errs[0.5, 1, "particle"][1] < 3e-3
    for order in (1, 2):
        for walk in ("particle", "group"):
            assert errs[0.3, order, walk][0] < errs[0.5, order, walk][0] < errs[0.75, order, walk][0]
    for th in (0.3, 0.5, 0.75):
        assert errs[th, 2, "particle"][0] < 0.5 * errs[th, 1, "particle"][0]
        assert errs[th, 1, "group"][0] < errs[th, 1, "particle"][0]


def test_tree_force_small_edge_cases(orc):
    # n = 1: no other particle, zero force
    p1 = np.array([[0.1, 0.2, 0.3, 1.0]], np.float32)
    res, b = orc.tree_force(p1, 0.5, 0.01)
    assert (res["out"] == 0).all()
    # n = 2: exact two-body
    p2 = np.array([[0, 0, 0, 1.0], [1, 0, 0, 2.0]], np.float32)
    res, b = orc.tree_force(p2, 0.5, 0.1)
    np.testing.assert_allclose(res["out"], orc.direct(p2, eps=0.1), rtol=1e-14)
    # all coincident: a = 0, phi = -(n-1) m / eps
    pc = np.tile(np.array([[1.0, 1.0, 1.0, 0.5]], np.float32), (12, 1))
    res, b = orc.tree_force(pc, 0.5, 0.1)
    np.testing.assert_allclose(res["out"][:, 3], -11 * 0.5 / 0.1, rtol=1e-14)
    assert (res["out"][:, :3] == 0).all()


# ---------------------------------------------------------- quadrupole

def _cluster(rng, k, a):
    y = rng.normal(size=(k, 3))
    y *= a * rng.uniform(0.2, 1.0, k)[:, None] / np.linalg.norm(y, axis=1)[:, None]
    m = rng.uniform(0.5, 1.5, k)
    y -= (m[:, None] * y).sum(0) / m.sum()  # centre of mass at the origin
    I = np.zeros(6)
    for w, v in zip(m, y):
        I += w * np.array([v[0] * v[0], v[1] * v[1], v[2] * v[2], v[0] * v[1], v[0] * v[2], v[1] * v[2]])
    return y, m, I


def test_quadrupole_gradient(orc):
    rng = np.random.default_rng(3)
    y, m, I = _cluster(rng, 10, 0.3)
    cm = np.array([0, 0, 0, m.sum()])
    x = np.array([2.0, -1.0, 1.5])
    for eps in (0.0, 0.2):
        f = orc.pc_eval(x, cm, I, eps)
        h = 1e-5
        g = np.zeros(3)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            g[k] = (orc.pc_eval(x + e, cm, I, eps)[3] - orc.pc_eval(x - e, cm, I, eps)[3]) / (2 * h)
        np.testing.assert_allclose(f[:3], -g, rtol=1e-7)


def test_quadrupole_textbook_at_zero_softening(orc):
    # Traceless form: phi = -M/r - r.Q.r / (2 r^5), Q = 3I - tr(I) 1,
    # a = -M r / r^3 + Q r / r^5 - 2.5 (r.Q.r) r / r^7.
    rng = np.random.default_rng(4)
    y, m, I6 = _cluster(rng, 7, 0.5)
    I = np.array([[I6[0], I6[3], I6[4]], [I6[3], I6[1], I6[5]], [I6[4], I6[5], I6[2]]])
    Q = 3 * I - np.trace(I) * np.eye(3)
    M = m.sum()
    for x in (np.array([3.0, 1.0, -2.0]), np.array([-0.5, 4.0, 0.3])):
        r = np.linalg.norm(x)
        phi = -M / r - x @ Q @ x / (2 * r ** 5)
        a = -M * x / r ** 3 + Q @ x / r ** 5 - 2.5 * (x @ Q @ x) * x / r ** 7
        f = orc.pc_eval(x, np.array([0, 0, 0, M]), I6, 0.0)
        np.testing.assert_allclose(f[:3], a, rtol=1e-12)
        assert abs(f[3] - phi) < 1e-12 * abs(phi)


def test_multipole_convergence_orders(orc):
    # Error of the monopole ~ (a/d)^2, of monopole+quadrupole ~ (a/d)^3
    # relative to the exact sum over the cluster's particles.
    rng = np.random.default_rng(5)
    y, m, I = _cluster(rng, 40, 1.0)
    src = np.zeros((40, 4), np.float32)
    src[:, :3] = y
    src[:, 3] = m
    # exact field from the float32-rounded cluster; recompute moments from it
    ys = src[:, :3].astype(np.float64)
    ms = src[:, 3].astype(np.float64)
    com = (ms[:, None] * ys).sum(0) / ms.sum()
    yy = ys - com
    I = np.array([(ms * yy[:, 0] ** 2).sum(), (ms * yy[:, 1] ** 2).sum(), (ms * yy[:, 2] ** 2).sum(),
                  (ms * yy[:, 0] * yy[:, 1]).sum(), (ms * yy[:, 0] * yy[:, 2]).sum(),
                  (ms * yy[:, 1] * yy[:, 2]).sum()])
    cm = np.array([com[0], com[1], com[2], ms.sum()])
    direction = np.array([0.6, -0.48, 0.64])
    e_mono, e_quad = [], []
    for d in (8.0, 16.0, 32.0, 64.0):
        x = com + d * direction
        tgt = np.zeros((1, 4), np.float32)
        tgt[0, :3] = x
        xe = tgt[0, :3].astype(np.float64)
        ex = orc.direct(src, tgt, self_idx=np.array([-1]), eps=0.0)[0]
        mono = orc.pc_eval(xe, cm, None, 0.0)
        quad = orc.pc_eval(xe, cm, I, 0.0)
        e_mono.append(np.linalg.norm(mono[:3] - ex[:3]) / np.linalg.norm(ex[:3]))
        e_quad.append(np.linalg.norm(quad[:3] - ex[:3]) / np.linalg.norm(ex[:3]))
    s_mono = np.log2(np.array(e_mono[:-1]) / np.array(e_mono[1:]))
    s_quad = np.log2(np.array(e_quad[:-1]) / np.array(e_quad[1:]))
    assert np.all(np.abs(s_mono - 2) < 0.35), s_mono
    assert np.all(np.abs(s_quad - 3) < 0.35), s_quad


def test_nodes_holding_members_are_opened(orc):
    # For theta above 1/sqrt(3) Eq. (2) alone could accept a cell that holds the
    # target; the walks open such cells, so a target never interacts with itself
    # through a multipole and its own particles all come from opened leaves.
    p = workloads.plummer(3000, seed=16)
    box, perm, sk, sp, t, m = _built(orc, p, n_leaf=8, theta=1.0)
    gf, gc = orc.groups(t, 32)
    for g in range(0, gf.shape[0], max(1, gf.shape[0] // 50)):
        pc, pp = orc.group_lists(sp, t, m, gf[g], gc[g])
        for v in pc:
            assert t.first[v] >= gf[g] + gc[g] or t.first[v] + t.count[v] <= gf[g]
    # with theta = 1 the per-particle walk stays finite and within a few percent
    # of the direct sum (Table ERR_a: about 1e-2 at theta = 1)
    d = orc.direct(p, eps=0.01)
    res, _ = orc.tree_force(p, 1.0, 0.01, walk="particle")
    ea, _ = orc.rel_err(res["out"], d)
    assert np.isfinite(ea).all() and ea.mean() < 0.05


@pytest.mark.parametrize("theta", [0.6, 1.0, 2.0])
def test_group_walk_follows_the_pinned_lists(orc, theta):
    # The force walk decides acceptance in its own loop; its per-target counts
    # must be those of the accepted-node and opened-leaf lists that the tests
    # above pin (conservative criterion, exact coverage, member-holding nodes
    # opened): n_pc = accepted nodes, n_pp = particles of opened leaves minus
    # the target itself.  Above theta = 1/sqrt(3) Eq. (2) alone can accept a
    # node holding members; at theta = 2 it does so for many groups.
    p = workloads.clumpy(4000, seed=14)
    res, b = orc.tree_force(p, theta, 0.01, n_leaf=8, G=32, order=2, walk="group")
    t = b.tree
    for g in range(b.g_first.shape[0]):
        gb, gc = int(b.g_first[g]), int(b.g_count[g])
        pc, pp = orc.group_lists(b.spos, t, b.mom, gb, gc)
        o = b.perm[gb:gb + gc]
        assert (res["n_pc"][o] == len(pc)).all()
        assert (res["n_pp"][o] == int(t.count[pp].sum()) - 1).all()


def test_particle_walk_single_particle_leaves_are_particles(orc):
    # A leaf holding one particle always gives a particle term (never a cell
    # term), whatever the criterion says: here the far particle C sits alone in
    # its level-1 cell, which Eq. (2) at theta = 1 would accept from A and B,
    # so A and B see only particle terms; C sees the cell {A, B}.
    p = np.array([[0.0, 0.0, 0.0, 1.0], [0.01, 0.0, 0.0, 1.0], [1.0, 1.0, 1.0, 1.0]], np.float32)
    res, b = orc.tree_force(p, 1.0, 0.01, n_leaf=1, walk="particle")
    assert list(res["n_pc"]) == [0, 0, 1] and list(res["n_pp"]) == [2, 2, 0]
    ea, ep = orc.rel_err(res["out"][:2], orc.direct(p, eps=0.01)[:2])
    assert ea.max() < 1e-12 and ep.max() < 1e-12


@pytest.mark.parametrize("theta", [0.5, 1.0, 4.0])
def test_particle_walk_equals_group_walk_of_single_particles(orc, theta):
    # With groups of one particle the group walk's box is the particle itself,
    # so its (pinned) criterion is the per-particle walk's: the same nodes are
    # accepted and the same leaves opened.  A one-particle node is a particle
    # term in one walk and an exact cell term (zero quadrupole) in the other,
    # so the forces agree to rounding; above theta = 1/sqrt(3) this also pins
    # that the per-particle walk never accepts a node holding its target.
    p = workloads.clumpy(3000, seed=25)
    rp, _ = orc.tree_force(p, theta, 0.01, n_leaf=8, G=1, order=2, walk="particle")
    rg, _ = orc.tree_force(p, theta, 0.01, n_leaf=8, G=1, order=2, walk="group")
    ea, ep = orc.rel_err(rp["out"], rg["out"])
    assert ea.max() < 1e-10 and ep.max() < 1e-10, (ea.max(), ep.max())
    assert (rp["n_pp"] + rp["n_pc"] == rg["n_pp"] + rg["n_pc"]).all()


def test_term_magnitude_sum(orc):
    # sum of |a_term| over a target's terms: equals |a| for a single other body,
    # bounds |a| from above (triangle inequality), and equals the direct sum of
    # magnitudes when every term is particle-particle (theta -> 0)
    p2 = np.array([[0, 0, 0, 1.0], [0.6, 0.8, 0, 2.0]], np.float32)
    res, b = orc.tree_force(p2, 0.5, 0.1)
    np.testing.assert_allclose(res["a_abs"], np.linalg.norm(res["out"][:, :3], axis=1), rtol=1e-14)
    p = workloads.plummer(800, seed=17)
    res, b = orc.tree_force(p, 1e-4, 0.01)
    x = p[:, :3].astype(np.float64)
    m = p[:, 3].astype(np.float64)
    d = x[None, :, :] - x[:, None, :]
    r2 = (d ** 2).sum(-1) + 1e-4
    mag = m[None, :] * np.sqrt((d ** 2).sum(-1)) / r2 ** 1.5
    np.fill_diagonal(mag, 0.0)
    np.testing.assert_allclose(res["a_abs"], mag.sum(1), rtol=1e-12)
    assert (res["a_abs"] >= np.linalg.norm(res["out"][:, :3], axis=1) * (1 - 1e-12)).all()


def test_particle_walk_unsoftened_cells(orc):
    # Appendix A's kernel applies cells without softening.  A light target at
    # the origin and a tight cluster near (1, 1, 1): with theta = 1 the cluster's
    # level-1 octant is accepted as one cell.  Unsoftened, the cell term must
    # match the exact eps = 0 sum over the cluster's particles to the
    # quadrupole truncation error ((a/D)^3 ~ 1e-9); softened, it must match the
    # eps = 0.1 sum instead (the two differ by ~1.5 eps^2 / D^2 = 5e-3).
    rng = np.random.default_rng(5)
    k = 50
    cl = np.concatenate([1.0 + 1e-3 * rng.random((k, 3)), np.full((k, 1), 1.0 / k)], axis=1)
    p = np.concatenate([np.array([[0.0, 0.0, 0.0, 1e-6]]), cl]).astype(np.float32)
    b = orc.Built(p, 8, 32, 1.0, 2)
    x = p[1:, :3].astype(np.float64) - p[0, :3].astype(np.float64)
    m = p[1:, 3].astype(np.float64)

    def exact(eps):
        r2 = (x * x).sum(1) + eps * eps
        return (m[:, None] * x / r2[:, None] ** 1.5).sum(0)

    eps = 0.1
    hard = orc.force_particles(b.spos, b.perm, b.tree, b.mom, eps, unsoftened_pc=True)
    soft = orc.force_particles(b.spos, b.perm, b.tree, b.mom, eps)
    assert hard["n_pc"][0] == 1 and hard["n_pp"][0] == 0
    e0, e1 = exact(0.0), exact(eps)
    rel = lambda a, r: np.linalg.norm(a - r) / np.linalg.norm(r)
    assert rel(hard["out"][0, :3], e0) < 1e-7
    assert rel(soft["out"][0, :3], e1) < 1e-7
    assert rel(e1, e0) > 1e-3
    # margins and term magnitudes (monopole parts) are reported per target
    assert np.isfinite(hard["margin"][0]) and hard["margin"][0] > 0
    assert abs(hard["a_abs"][0] / np.linalg.norm(e0) - 1) < 1e-5


# ------------------------------------------------------- 63-bit keys (21 levels)
@pytest.mark.parametrize("curve", [0, 1])
def test_deep_keys_extend_shallow_keys(orc, curve):
    # the 10-bit cell is the 21-bit cell shifted by 11 (the scale factor 2^11 is
    # exact in FP32), so a 63-bit key begins with the particle's 30-bit key
    for kind in ("clumpy", "plummer", "uniform"):
        p = workloads.make(kind, 20000, 8)
        box = orc.bbox(p)
        k30 = orc.keys(p, box, curve, 10).astype(np.uint64)
        k63 = orc.keys(p, box, curve, 21)
        assert k63.dtype == np.uint64 and (k63 < (np.uint64(1) << np.uint64(63))).all()
        np.testing.assert_array_equal(k63 >> np.uint64(33), k30)


def test_deep_keys_hand_corners(orc):
    # the box's low corner is key 0; the high corner is the last cell 2^21 - 1 on every axis
    p = np.array([[0.0, 0.0, 0.0, 1.0], [1.0, 1.0, 1.0, 1.0], [0.25, 0.5, 0.75, 1.0]], np.float32)
    box = orc.bbox(p)
    k = orc.keys(p, box, 0, 21)
    assert k[0] == 0 and k[1] == (1 << 63) - 1
    # (0.25, 0.5, 0.75) -> cells (2^19, 2^20, 3 * 2^19): bits 19/20 of each axis interleaved
    cx, cy, cz = 1 << 19, 1 << 20, 3 << 19
    want = 0
    for b in range(21):
        want |= (((cx >> b) & 1) << (3 * b + 2)) | (((cy >> b) & 1) << (3 * b + 1)) | (((cz >> b) & 1) << (3 * b))
    assert int(k[2]) == want


def test_deep_hilbert_face_connected(orc):
    rng = np.random.default_rng(21)
    for h in rng.integers(0, (1 << 63) - 1, 1500, dtype=np.int64):
        a, b = np.array(orc.cell_of_key(int(h), 1, 21)), np.array(orc.cell_of_key(int(h) + 1, 1, 21))
        assert np.abs(a - b).sum() == 1 and (a < (1 << 21)).all()
        assert orc.key_of_cell(*a, 1, 21) == int(h)


def test_deep_tree_removes_overflow_leaves(orc):
    # at 10 levels the clump cores overflow leaf 8; at 21 levels only particles
    # sharing one 2^-21 cell could, and the octree above the old leaves is unchanged
    rng = np.random.default_rng(3)
    knot = np.concatenate([0.2 + 1e-4 * rng.random((300, 3)), np.full((300, 1), 1e-4)], 1)
    p = np.concatenate([workloads.clumpy(60000, seed=2), knot]).astype(np.float32)
    b10 = orc.Built(p, 8, 64, 0.5, 1, max_level=10)
    b21 = orc.Built(p, 8, 64, 0.5, 1, max_level=21)
    l10 = b10.tree.nchild == 0
    assert b10.tree.count[l10].max() > 8
    l21 = b21.tree.nchild == 0
    big = l21 & (b21.tree.count > 8)
    for v in np.nonzero(big)[0]:
        ks = b21.skeys[b21.tree.first[v]:b21.tree.first[v] + b21.tree.count[v]]
        assert (ks == ks[0]).all()
    np.testing.assert_array_equal(b21.perm, b10.perm[np.argsort(b21.keys[b10.perm], kind="stable")])
    # nodes of levels <= 10 that are not max-depth leaves appear identically in both trees
    s10 = {(int(l), int(f), int(c)) for l, f, c, ch in zip(b10.tree.level, b10.tree.first, b10.tree.count,
                                                            b10.tree.nchild) if l < 10 or c <= 8}
    s21 = {(int(l), int(f), int(c)) for l, f, c in zip(b21.tree.level, b21.tree.first, b21.tree.count) if l <= 10}
    assert s10 <= s21


def test_deep_tree_theta_to_zero_equals_direct(orc):
    p = workloads.clumpy(3000, seed=5)
    res, _ = orc.tree_force(p, 1e-4, 0.01, n_leaf=4, G=32, order=2, max_level=21)
    ref = orc.direct(p, eps=0.01)
    np.testing.assert_allclose(res["out"], ref, rtol=1e-10, atol=1e-12)
