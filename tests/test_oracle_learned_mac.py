"""Pins of the oracle's learned opening criterion (network, training step,
features, labels, walk) against hand-computed values, finite differences,
closed forms of Adam and the limits where the walk reduces to known walks."""
import numpy as np
import pytest

import workloads

NP = 1313


def _path_net(w1=1.0, b1=0.0, w2=1.0, b2=0.0, w3=1.0, b3=0.0, k=0):
    """Network whose only path is feature k -> hidden 0 -> hidden 0 -> output."""
    P = np.zeros(NP)
    P[0 * 6 + k] = w1             # W1[0][k]
    P[192 + 0] = b1               # b1[0]
    P[224 + 0] = w2               # W2[0][0]
    P[224 + 1024 + 0] = b2        # b2[0]
    P[224 + 1024 + 32 + 0] = w3   # W3[0]
    P[-1] = b3
    return P


def test_forward_hand_networks(orc):
    assert orc.mlp_nparams() == NP
    X = np.zeros((4, 6))
    X[:, 2] = [-1.0, 0.25, 0.75, 3.0]
    # y = 2 * relu(0.5 * relu(x - 0.5) + 0) - 1 on feature 2
    P = _path_net(w1=1.0, b1=-0.5, w2=0.5, w3=2.0, b3=-1.0, k=2)
    y = orc.mlp_forward(P, X)
    np.testing.assert_allclose(y, [-1.0, -1.0, -0.75, 1.5], rtol=0, atol=1e-15)


def test_forward_bf16_emulation(orc):
    # bfloat16 keeps 8 significant bits (a unit in the last place of 1 is 2^-7) and
    # rounds to nearest, ties to even: 1 + 2^-9 -> 1, 1 + 5*2^-9 -> 1 + 2^-7,
    # 1 + 3*2^-9 -> 1 + 2^-7 (up: truncation would give 1), the ties 1 + 2^-8 -> 1
    # and 1 + 3*2^-8 -> 1 + 2^-6 (to the even neighbour), and the same for -x
    v = [1 + 2 ** -9, 1 + 5 * 2 ** -9, 1 + 3 * 2 ** -9, 1 + 2 ** -8, 1 + 3 * 2 ** -8]
    want = [1.0, 1 + 2 ** -7, 1 + 2 ** -7, 1.0, 1 + 2 ** -6]
    P = _path_net(k=0)
    X = np.zeros((len(v), 6))
    X[:, 0] = v
    np.testing.assert_allclose(orc.mlp_forward(P, X, bf16=False), X[:, 0], rtol=0, atol=0)
    np.testing.assert_allclose(orc.mlp_forward(P, X, bf16=True), want, rtol=0, atol=0)
    # negative inputs through a negated path: w1 = -1 makes the hidden unit -(-x) = x
    Pn = _path_net(w1=-1.0, k=0)
    np.testing.assert_allclose(orc.mlp_forward(Pn, -X, bf16=True), want, rtol=0, atol=0)


def test_loss_weights_and_gradient(orc):
    # constant network (all weights 0, b3 = c): loss = mean(w (c - y)^2), w = 4 below the label
    P = np.zeros(NP)
    P[-1] = 0.5
    X = np.zeros((3, 6))
    Y = np.array([1.0, 0.0, -2.0])
    loss, g = orc.mlp_loss_grad(P, X, Y, under_weight=4.0)
    assert abs(loss - (4 * 0.25 + 0.25 + 6.25) / 3) < 1e-15
    assert abs(g[-1] - (2 * 4 * -0.5 + 2 * 0.5 + 2 * 2.5) / 3) < 1e-15
    # central finite differences on a random network and batch
    rng = np.random.default_rng(0)
    P = rng.normal(0, 0.3, NP)
    X = rng.normal(0, 1, (64, 6))
    Y = rng.normal(-3, 1, 64)
    loss, g = orc.mlp_loss_grad(P, X, Y, under_weight=4.0)
    idx = rng.choice(NP, 60, replace=False)
    h = 1e-6
    for k in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (orc.mlp_loss_grad(Pp, X, Y)[0] - orc.mlp_loss_grad(Pm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_adam_closed_form(orc):
    # with zero moments, the bias-corrected first two steps under a constant
    # gradient g both move each parameter by -lr * g / (|g| + eps)
    P = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    lr, eps = 1e-2, 1e-8
    orc.adam_step(P, g, m, v, 1, lr=lr, eps=eps)
    np.testing.assert_allclose(P, [1.0 - lr * 0.3 / (0.3 + eps), -2.0 + lr * 4.0 / (4.0 + eps), 0.5], rtol=1e-14)
    orc.adam_step(P, g, m, v, 2, lr=lr, eps=eps)
    np.testing.assert_allclose(P, [1.0 - 2 * lr * 0.3 / (0.3 + eps), -2.0 + 2 * lr * 4.0 / (4.0 + eps), 0.5],
                               rtol=1e-12)


def test_features_hand_case(orc):
    lo, hi = [0, 0, 0], [1, 1, 1]
    cm = [3.5, 0.5, 0.5, 0.25]
    # second moments with trace 3, deviatoric part diag(2,-1,-1) and xy = 1: |.|_F = sqrt(4+1+1+2)
    quad = [3.0, 0.0, 0.0, 1.0, 0.0, 0.0]
    f = orc.mac_features_one(lo, hi, cm, quad, side=1.0, level=2, count=8, mtot=1.0)
    np.testing.assert_allclose(f, [1 / 3, np.log10(0.25), np.sqrt(8.0) / 0.25, np.sqrt(3) / 2 / 3, 0.2, 3 / 24],
                               rtol=1e-14)
    assert orc.mac_features_one(lo, hi, [0.5, 0.5, 0.5, 1.0], None, 1.0, 1, 2, 1.0) is None  # d = 0


def _built_with_atot(orc, pos, theta_guard, order, eps, G=64):
    b = orc.Built(pos, 8, G, theta_guard, order)
    d = orc.direct(pos, eps=eps)
    a_tot = np.linalg.norm(d[:, :3], axis=1)[b.perm]
    return b, a_tot


def test_labels_exact_cases(orc):
    pos = workloads.plummer(3000, seed=31)
    eps = 0.01
    b, a_tot = _built_with_atot(orc, pos, 1.0, 2, eps)
    X, Y, pg, pn = orc.mac_training_pairs(b, np.arange(0, b.g_first.size, 7), a_tot, eps, descend_above=1e-6)
    assert X.shape[0] > 100
    t = b.tree
    single = t.count[pn] == 1
    assert single.any()
    assert (Y[single] == -12).all()          # a one-particle cell is exact: floor value
    assert (Y <= 0.5).all() and (Y >= -12).all()
    # descending: a labelled internal node's guard-passing children are labelled
    # exactly when its label exceeds log10(descend_above) = -6
    groups = np.arange(0, b.g_first.size, 7)
    have = set(zip(pg.tolist(), pn.tolist()))
    for k in range(0, X.shape[0], 5):
        v = int(pn[k])
        if t.nchild[v] == 0:
            continue
        g = groups[pg[k]]
        gb, ge = int(b.g_first[g]), int(b.g_first[g] + b.g_count[g])
        mem = b.spos[gb:ge, :3].astype(np.float64)
        lo, hi = mem.min(0), mem.max(0)
        for c in range(t.child_first[v], t.child_first[v] + t.nchild[v]):
            com = b.mom.com_m[c, :3]
            d2 = float((np.maximum(np.maximum(lo - com, com - hi), 0.0) ** 2).sum())
            member = t.first[c] < ge and t.first[c] + t.count[c] > gb
            if d2 > b.mom.s_eff[c] and not member:
                assert ((int(pg[k]), c) in have) == bool(Y[k] > -6), (k, c)
    # independent recomputation of a few labels by brute force
    rng = np.random.default_rng(1)
    for k in rng.choice(np.nonzero(~single)[0], 10, replace=False):
        g = np.arange(0, b.g_first.size, 7)[pg[k]]
        gb, gc = b.g_first[g], b.g_count[g]
        v = pn[k]
        tgt = b.spos[gb:gb + gc]
        src = b.spos[t.first[v]:t.first[v] + t.count[v]]
        exact = orc.direct(src, tgt, self_idx=np.full(gc, -1), eps=eps)
        pc = np.array([orc.pc_eval(x.astype(np.float64), b.mom.com_m[v], b.mom.quad[v], eps) for x in tgt[:, :3]])
        err = np.linalg.norm(pc[:, :3] - exact[:, :3], axis=1) / a_tot[gb:gb + gc]
        assert abs(Y[k] - np.log10(max(err.max(), 1e-12))) < 1e-9


def test_learned_walk_limits(orc):
    pos = workloads.clumpy(4000, seed=32)
    eps, tg, tfb = 1e-3, 1.0, 0.5
    b = orc.Built(pos, 8, 64, tg, 2)
    fmin, fmax = np.full(6, -1e9), np.full(6, 1e9)
    always = np.zeros(NP)
    always[-1] = -100.0
    never = np.zeros(NP)
    never[-1] = 100.0
    # always-accept: the guard's plain group walk, also at a guard theta of 4,
    # where Eq. (2) alone would accept many nodes that hold group members
    for tgx in (tg, 4.0):
        bx = orc.Built(pos, 8, 64, tgx, 2)
        ref = orc.force_groups(bx.spos, bx.perm, bx.tree, bx.mom, bx.g_first, bx.g_count, eps)
        r = orc.force_groups_learned(bx, always, fmin, fmax, 1e-3, eps, tgx, tfb)
        np.testing.assert_allclose(r["out"], ref["out"], rtol=1e-13, atol=0)
        np.testing.assert_array_equal(r["n_pc"], ref["n_pc"])
    r = orc.force_groups_learned(b, never, fmin, fmax, 1e-3, eps, tg, tfb)
    d = orc.direct(pos, eps=eps)
    ea, ep = orc.rel_err(r["out"], d)
    assert ea.max() < 1e-12 and ep.max() < 1e-12 and (r["n_pc"] == 0).all()
    # every feature out of range (below, above, or both ends of an empty range):
    # the fallback is the plain criterion at theta_fb
    bf = orc.Built(pos, 8, 64, tfb, 2)
    ref = orc.force_groups(bf.spos, bf.perm, bf.tree, bf.mom, bf.g_first, bf.g_count, eps)
    for lo, hi in ((np.full(6, 1e9), np.full(6, -1e9)), (np.full(6, 1e9), np.full(6, 2e9)),
                   (np.full(6, -2e9), np.full(6, -1e9))):
        r = orc.force_groups_learned(b, always, lo, hi, 1e-3, eps, tg, tfb)
        ok = (ref["margin"] > 1e-9) & (r["margin_geo"] > 1e-9)
        np.testing.assert_allclose(r["out"][ok], ref["out"][ok], rtol=1e-12, atol=0)
        assert ok.mean() > 0.95
