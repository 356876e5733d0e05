"""Pins of the oracle's individual, symmetrized softening (the symmetrized
Plummer potential that Sec. 7 names as an application, after Saitoh & Makino
2010): pair softening eps_ij^2 = (eps_i^2 + eps_j^2) / 2, a cell softened
with the mass-weighted mean of its particles' eps^2.  Fixed by closed forms,
symmetry, the common-softening special case, finite differences and the
theta -> 0 limit, not by the oracle itself."""
import numpy as np
import pytest

import oracle
import workloads


def _soft(n, seed, lo=0.002, hi=0.05):
    rng = np.random.default_rng(seed)
    return (10.0 ** rng.uniform(np.log10(lo), np.log10(hi), n)).astype(np.float32)


def test_two_bodies_closed_form_and_symmetry(orc):
    pos = np.array([[0.0, 0.0, 0.0, 0.25], [0.6, -0.3, 0.2, 0.75]], np.float32)
    eps = np.array([0.1, 0.4], np.float32)
    out = oracle.direct_sym(pos, eps)
    d = pos[1, :3].astype(np.float64) - pos[0, :3]
    h2 = d @ d + 0.5 * (float(eps[0]) ** 2 + float(eps[1]) ** 2)
    np.testing.assert_allclose(out[0, :3], 0.75 * d / h2 ** 1.5, rtol=1e-14)
    np.testing.assert_allclose(out[1, :3], -0.25 * d / h2 ** 1.5, rtol=1e-14)
    np.testing.assert_allclose(out[:, 3], [-0.75 / np.sqrt(h2), -0.25 / np.sqrt(h2)], rtol=1e-14)
    # the pair force is the same for both bodies
    np.testing.assert_allclose(0.25 * out[0, :3], -0.75 * out[1, :3], rtol=1e-14)


def test_momentum_is_conserved(orc):
    pos = workloads.plummer(500, seed=3)
    eps = _soft(500, 4)
    out = oracle.direct_sym(pos, eps)
    p = (pos[:, 3:4].astype(np.float64) * out[:, :3]).sum(axis=0)
    scale = (pos[:, 3:4] * np.abs(out[:, :3])).sum()
    assert np.abs(p).max() < 1e-13 * scale


def test_common_softening_is_the_plain_sum(orc):
    pos = workloads.clumpy(800, seed=5)
    eps = np.full(800, 0.01, np.float32)
    np.testing.assert_allclose(oracle.direct_sym(pos, eps), oracle.direct(pos, eps=float(eps[0])), rtol=1e-13,
                               atol=0)


def test_acceleration_is_minus_gradient_of_potential(orc):
    src = workloads.plummer(200, seed=6)
    eps_src = _soft(200, 7)
    x0 = np.array([[0.3125, -0.1875, 0.125, 0.0]], np.float64)  # exact in FP32
    e_t = np.array([0.03], np.float32)
    h = 2e-5

    def phi(x):
        # targets are FP32 on the way in: use an exactly representable point
        t = x.astype(np.float32)
        return oracle.direct_sym(src, eps_src, t, e_t, np.array([-1]))[0, 3], t

    a = oracle.direct_sym(src, eps_src, x0.astype(np.float32), e_t, np.array([-1]))[0, :3]
    for k in range(3):
        xp, xm = x0.copy(), x0.copy()
        xp[0, k] += h
        xm[0, k] -= h
        (pp, tp), (pm, tm) = phi(xp), phi(xm)
        grad = (pp - pm) / (float(tp[0, k]) - float(tm[0, k]))
        assert abs(-grad - a[k]) < 1e-7 * np.abs(a).max()


def test_cell_softening_is_the_mass_weighted_mean(orc):
    # one node holding two particles of unequal mass and softening
    pos = np.array([[0.1, 0.1, 0.1, 1.0], [0.1, 0.1, 0.1, 3.0]], np.float32)
    eps = np.array([0.2, 0.4], np.float32)
    tree = oracle.Tree(np.array([0], np.int32), np.array([0], np.int32), np.array([2], np.int32),
                       np.array([-1], np.int32), np.array([0], np.int32))
    e2 = oracle.cell_softening(pos, eps, tree)
    expect = (1.0 * float(eps[0]) ** 2 + 3.0 * float(eps[1]) ** 2) / 4.0
    assert abs(e2[0] - expect) < 1e-15
    # massless node: 0
    pos[:, 3] = 0.0
    assert oracle.cell_softening(pos, eps, tree)[0] == 0.0


def test_cell_softening_cancels_the_first_order_term(orc):
    # a coincident cluster of particles with spread softenings, seen from far:
    # with the mass-weighted mean the cell term's error falls as the square of
    # the spread; with the unweighted mean only linearly
    rng = np.random.default_rng(8)
    m = rng.uniform(0.5, 2.0, 16)
    base = rng.standard_normal(16)
    base -= (m * base).sum() / m.sum()       # mass-weighted zero mean
    x_i, e_i2 = np.array([0.05, 0.0, 0.0]), 0.01 ** 2

    def errs(scale):
        e2 = 0.02 ** 2 * (1.0 + scale * base)
        exact = -(m / np.sqrt(x_i @ x_i + 0.5 * (e_i2 + e2))).sum()
        weighted = -m.sum() / np.sqrt(x_i @ x_i + 0.5 * (e_i2 + (m * e2).sum() / m.sum()))
        plain = -m.sum() / np.sqrt(x_i @ x_i + 0.5 * (e_i2 + e2.mean()))
        return abs(weighted - exact), abs(plain - exact)

    w1, p1 = errs(0.2)
    w2, p2 = errs(0.1)
    assert 3.6 < w1 / w2 < 4.4      # second order
    assert 1.7 < p1 / p2 < 2.3      # first order
    # the oracle's cell softening is the weighted one
    pos = np.zeros((16, 4), np.float32)
    pos[:, 3] = m
    eps = np.sqrt(0.02 ** 2 * (1.0 + 0.2 * base)).astype(np.float32)
    tree = oracle.Tree(np.array([0], np.int32), np.array([0], np.int32), np.array([16], np.int32),
                       np.array([-1], np.int32), np.array([0], np.int32))
    e2o = oracle.cell_softening(pos, eps, tree)[0]
    e2f = eps.astype(np.float64) ** 2
    m32 = m.astype(np.float32).astype(np.float64)
    assert abs(e2o - (m32 * e2f).sum() / m32.sum()) < 1e-15


@pytest.mark.parametrize("order", [1, 2])
def test_particle_walk_at_theta_to_zero_is_the_direct_sum(orc, order):
    pos = workloads.clumpy(3000, seed=9)
    eps = _soft(3000, 10)
    res, _ = oracle.tree_force_sym(pos, eps, 1e-4, n_leaf=8, order=order)
    ref = oracle.direct_sym(pos, eps)
    np.testing.assert_allclose(res["out"], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_particle_walk_with_common_softening_is_the_plain_walk(orc):
    pos = workloads.plummer(4000, seed=11)
    eps = np.full(4000, 0.01, np.float32)
    a, _ = oracle.tree_force_sym(pos, eps, 0.6, n_leaf=8, order=2)
    b, _ = oracle.tree_force(pos, 0.6, float(eps[0]), n_leaf=8, order=2, walk="particle")
    np.testing.assert_allclose(a["out"], b["out"], rtol=1e-13, atol=0)
    assert (a["n_pp"] == b["n_pp"]).all() and (a["n_pc"] == b["n_pc"]).all()


def test_particle_walk_error_is_that_of_a_tree(orc):
    # at theta = 0.5 the symmetrized tree forces lie within tree accuracy of the direct sum
    pos = workloads.plummer(6000, seed=12)
    eps = _soft(6000, 13, 0.005, 0.05)
    res, _ = oracle.tree_force_sym(pos, eps, 0.5, n_leaf=8, order=2)
    ref = oracle.direct_sym(pos, eps)
    ea, _ = oracle.rel_err(res["out"], ref)
    assert np.percentile(ea, 99) < 1e-2 and np.median(ea) < 1e-3


def test_particle_walk_cell_term_uses_the_pair_mean(orc):
    # a far, tight cluster of 8 particles (one accepted cell for the lone
    # target): the cell term's softening is (eps_i^2 + mean eps_j^2) / 2, so
    # the tree force equals the symmetrized direct sum to the expansion's
    # accuracy ((cluster size / distance)^3 ~ 1e-9), while the target's own
    # eps^2 would be off by several per cent here
    rng = np.random.default_rng(14)
    cl = np.concatenate([1.0 + 1e-3 * rng.random((8, 1)), 1e-3 * rng.random((8, 2)),
                         rng.uniform(0.5, 1.5, (8, 1))], axis=1)
    pos = np.concatenate([[[0.0, 0.0, 0.0, 1.0]], cl]).astype(np.float32)
    eps = np.concatenate([[0.3], 0.001 + 0.002 * rng.random(8)]).astype(np.float32)
    res, b = oracle.tree_force_sym(pos, eps, 1.0, n_leaf=8, order=2)
    assert res["n_pc"][0] == 1 and res["n_pp"][0] == 0
    ref = oracle.direct_sym(pos, eps)
    np.testing.assert_allclose(res["out"][0], ref[0], rtol=1e-6)
