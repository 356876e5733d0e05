"""Training and calibration of the learned opening criterion.

The criterion extends Eq. (2)'s geometric test: a 6 -> 32 -> 32 -> 1 ReLU
network predicts log10 of a node's relative force-error contribution to a
group of targets, and a node passing a permissive Eq. (2) guard is accepted
when the prediction is below log10(tau).  Everything here is a driver over
the C ABI: the labels come from the library's labelling kernel (errors the
method measures against direct sums over each node's particles), the fit
from its forward/backward/Adam kernels, the calibration from its walk.

    python -m paper_1112_4539_gb300.learned train --out weights.npz \
        --theta-guard 1.2 --groups 400 --epochs 60 --seeds 4

Random numbers (initial weights, group samples, batch order) are drawn here
with numpy's counter-based Philox generator from a recorded seed and passed
to the kernels as inputs.
"""
import argparse
import json
import math
import time

import numpy as np

from . import (MLP_ACT, MLP_NPARAM, BhError, Context, _check, bh_mac_label, bh_mac_set, bh_mlp_train,
               direct_force)

EPS = {"plummer": 0.01, "clumpy": 1e-3, "uniform": 0.01, "sphere": 0.01}

# training sets: seeded Plummer and Hernquist-clump systems, N = 2^18 .. 2^22
DEFAULT_SETS = [("plummer", 1 << 18, 10), ("clumpy", 1 << 18, 11), ("plummer", 1 << 19, 12),
                ("clumpy", 1 << 19, 13), ("plummer", 1 << 20, 14), ("clumpy", 1 << 20, 15),
                ("plummer", 1 << 21, 16), ("clumpy", 1 << 21, 17), ("plummer", 1 << 22, 18),
                ("clumpy", 1 << 22, 19)]


def _rng(seed):
    return np.random.Generator(np.random.Philox(key=int(seed)))


def init_params(seed=0):
    """He-uniform weights, zero biases; the output bias starts at -4 (log10 of a
    typical error contribution)."""
    rng = _rng(seed)
    P = np.zeros(MLP_NPARAM, np.float32)
    o = 0

    def take(n):
        nonlocal o
        s = slice(o, o + n)
        o += n
        return s

    w1, b1, w2, b2, w3, b3 = take(32 * 6), take(32), take(32 * 32), take(32), take(32), take(1)
    P[w1] = rng.uniform(-1, 1, 32 * 6) * math.sqrt(6.0 / 6)
    P[w2] = rng.uniform(-1, 1, 32 * 32) * math.sqrt(6.0 / 32)
    P[w3] = rng.uniform(-1, 1, 32) * math.sqrt(3.0 / 32)
    P[b3] = -4.0
    return P


def label_set(kind, n, seed, G, leaf, order, theta_guard, groups, log_floor=-6.0, ref_theta=0.3, group_seed=0):
    """Labelled (features, labels) of `groups` random groups of one seeded system,
    as device tensors."""
    import torch

    import workloads
    eps = EPS[kind]
    pos = workloads.make(kind, n, seed)
    x = torch.from_numpy(pos).cuda()
    ctx = Context(n, leaf_size=leaf, group_size=G, order=2)
    acc_ref = ctx.evaluate(x, ref_theta, eps)  # accurate quadrupole reference forces
    ctx.close()
    ctx = Context(n, leaf_size=leaf, group_size=G, order=order)
    ctx.build(x)
    ctx.moments(theta_guard)
    ng = ctx.stats()["n_groups"]
    sel = np.sort(_rng(1000 * seed + group_seed).choice(ng, min(groups, ng), replace=False)).astype(np.int32)
    g = torch.from_numpy(sel).cuda()
    cap = 4000 * sel.size
    for _ in range(3):
        X = torch.empty((cap, 6), dtype=torch.float32, device="cuda")
        Y = torch.empty(cap, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        _check(bh_mac_label(ctx.h, g, acc_ref, eps, log_floor, X, Y, cnt), "bh_mac_label")
        c = int(cnt.item())
        if c <= cap:
            break
        cap = c
    rc = ctx.status()
    ctx.close()
    if rc != 0:
        raise BhError(rc, "labelling")
    return X[:c].clone(), Y[:c].clone()


def training_set(sets=DEFAULT_SETS, G=96, leaf=16, order=2, theta_guard=1.0, groups=200, log_floor=-6.0):
    import torch
    Xs, Ys = [], []
    for kind, n, seed in sets:
        X, Y = label_set(kind, n, seed, G, leaf, order, theta_guard, groups, log_floor)
        Xs.append(X)
        Ys.append(Y)
    return torch.cat(Xs), torch.cat(Ys)


def feature_range(X, margin=0.02):
    """Per-feature [min, max] of the training set, widened by `margin` of the span."""
    lo = X.min(dim=0).values.cpu().numpy().astype(np.float64)
    hi = X.max(dim=0).values.cpu().numpy().astype(np.float64)
    span = np.maximum(hi - lo, 1e-6)
    return (lo - margin * span).astype(np.float32), (hi + margin * span).astype(np.float32)


def train(X, Y, epochs=20, batch=8192, lr=1e-3, under_weight=4.0, seed=0, params=None):
    """Fit the network on the GPU; returns (params float32[1313], mean loss per epoch)."""
    import torch
    n = int(Y.numel())
    rng = _rng(seed)
    P = torch.from_numpy(init_params(seed) if params is None else np.asarray(params, np.float32)).cuda()
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    work = torch.empty(batch * MLP_ACT + MLP_NPARAM + 64, dtype=torch.float32, device="cuda")
    steps = max(1, (n + batch - 1) // batch)
    hist = []
    t = 0
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
        loss = torch.zeros(steps, dtype=torch.float32, device="cuda")
        _check(bh_mlp_train(X, Y, order, P, m, v, work, steps, batch, lr, under_weight, loss, 0 if ep == 0 else t),
               "bh_mlp_train")
        t += steps
        hist.append(float(loss.mean().item()))
    return P.cpu().numpy(), hist


def p99_error(acc, idx_t, ref):
    import torch
    g = acc[idx_t].double()
    da = torch.linalg.norm(g[:, :3] - ref[:, :3], dim=1) / torch.linalg.norm(ref[:, :3], dim=1)
    return float(torch.quantile(da, 0.99))


def fp64_judge(x, eps, n_sample=4096, seed=101):
    """FP64 direct accelerations of seeded sample targets (the error judge)."""
    import torch

    import workloads
    idx = workloads.sample_targets(x.shape[0], n_sample, seed=seed)
    idx_t = torch.from_numpy(idx).to(x.device)
    ref = torch.empty((idx.size, 4), dtype=torch.float64, device=x.device)
    _check(direct_force(x, x[idx_t].contiguous(), idx_t, eps, ref, 64), "direct_force")
    return idx_t, ref


def evaluate_learned(ctx, x, theta_guard, eps, params, fmin, fmax, tau, theta_fb, acc):
    _check(bh_mac_set(ctx.h, params, fmin, fmax, tau, theta_fb), "bh_mac_set")
    return ctx.evaluate(x, theta_guard, eps, acc)


def calibrate_tau(ctx, x, idx_t, ref, eps, params, fmin, fmax, theta_guard=1.0, theta_fb=0.5, target=1e-3,
                  lo=-7.0, hi=-0.5, iters=12):
    """Largest tau (bisection on log10 tau) whose p99 error is <= target."""
    import torch
    acc = torch.empty_like(x)
    if p99_error(evaluate_learned(ctx, x, theta_guard, eps, params, fmin, fmax, 10 ** lo, theta_fb, acc), idx_t,
                 ref) > target:
        return None
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        e = p99_error(evaluate_learned(ctx, x, theta_guard, eps, params, fmin, fmax, 10 ** mid, theta_fb, acc),
                      idx_t, ref)
        if e <= target:
            lo = mid
        else:
            hi = mid
    return 10 ** lo


def calibrate_theta(ctx, x, idx_t, ref, eps, target=1e-3, lo=0.2, hi=1.0, iters=10):
    import torch
    acc = torch.empty_like(x)
    bh_mac_set(ctx.h, None)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if p99_error(ctx.evaluate(x, mid, eps, acc), idx_t, ref) <= target:
            lo = mid
        else:
            hi = mid
    return lo


def save(path, params, fmin, fmax, meta):
    np.savez(path, params=np.asarray(params, np.float32), fmin=np.asarray(fmin, np.float32),
             fmax=np.asarray(fmax, np.float32), meta=json.dumps(meta))


def load(path):
    d = np.load(path)
    return d["params"], d["fmin"], d["fmax"], json.loads(str(d["meta"]))


# validation sets of the seed selection (not used for training or testing)
VALIDATION_SETS = [("clumpy", 1 << 22, 5), ("plummer", 1 << 22, 5)]


def matched_speedup(ctx, x, idx_t, ref, eps, params, fmin, fmax, theta_guard, theta_fb=0.5, reps=3):
    """Time of the plain criterion over that of the learned one, each at its own
    p99 = 1e-3 operating point (theta and tau bisected), and the interaction ratio."""
    import torch
    acc = torch.empty_like(x)

    def timed(theta):
        ctx.evaluate(x, theta, eps, acc)
        torch.cuda.synchronize()
        s0 = ctx.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ctx.evaluate(x, theta, eps, acc)
        e1.record()
        torch.cuda.synchronize()
        s1 = ctx.stats()
        return (e0.elapsed_time(e1) / reps,
                (s1["n_pp_total"] - s0["n_pp_total"] + s1["n_pc_total"] - s0["n_pc_total"]) / reps)

    theta = calibrate_theta(ctx, x, idx_t, ref, eps)
    bh_mac_set(ctx.h, None)
    t_plain, i_plain = timed(theta)
    tau = calibrate_tau(ctx, x, idx_t, ref, eps, params, fmin, fmax, theta_guard=theta_guard, theta_fb=theta_fb)
    if tau is None:
        bh_mac_set(ctx.h, None)
        return None
    _check(bh_mac_set(ctx.h, params, fmin, fmax, tau, theta_fb), "bh_mac_set")
    t_learned, i_learned = timed(theta_guard)
    bh_mac_set(ctx.h, None)
    return dict(theta=theta, tau=tau, speedup=t_plain / t_learned, interaction_ratio=i_learned / i_plain)


def main():
    import torch

    import workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train"])
    ap.add_argument("--out", required=True)
    ap.add_argument("--G", type=int, default=96)
    ap.add_argument("--leaf", type=int, default=16)
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--theta-guard", type=float, default=1.0)
    ap.add_argument("--groups", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--seeds", type=int, default=1,
                    help="train seeds seed..seed+K-1 and keep the one with the best geometric-mean matched-p99 "
                         "speedup on the validation sets")
    a = ap.parse_args()
    t0 = time.time()
    X, Y = training_set(G=a.G, leaf=a.leaf, order=a.order, theta_guard=a.theta_guard, groups=a.groups)
    t1 = time.time()
    fmin, fmax = feature_range(X)
    val = []
    if a.seeds > 1:
        for kind, n, seed in VALIDATION_SETS:
            x = torch.from_numpy(workloads.make(kind, n, seed)).cuda()
            idx_t, ref = fp64_judge(x, EPS[kind])
            val.append((kind, x, idx_t, ref, EPS[kind], Context(n, leaf_size=a.leaf, group_size=a.G, order=a.order)))
    best = None
    for seed in range(a.seed, a.seed + a.seeds):
        params, hist = train(X, Y, epochs=a.epochs, seed=seed)
        score, rows = 0.0, {}
        for kind, x, idx_t, ref, eps, ctx in val:
            r = matched_speedup(ctx, x, idx_t, ref, eps, params, fmin, fmax, a.theta_guard)
            rows[kind] = r
            score += math.log(r["speedup"]) if r else -1e9
        if best is None or score > best[0]:
            best = (score, seed, params, hist, rows)
    score, seed, params, hist, rows = best
    for *_, ctx in val:
        ctx.close()
    meta = dict(G=a.G, leaf=a.leaf, order=a.order, theta_guard=a.theta_guard, groups=a.groups,
                epochs=a.epochs, seed=seed, samples=int(Y.numel()), sets=DEFAULT_SETS, loss=hist,
                label_s=t1 - t0, train_s=time.time() - t1)
    if a.seeds > 1:
        meta["selection"] = ("best of seeds %d-%d by geometric-mean matched-p99 speedup on %s"
                             % (a.seed, a.seed + a.seeds - 1, VALIDATION_SETS))
        meta["validation"] = rows
    save(a.out, params, fmin, fmax, meta)
    print(json.dumps({k: v for k, v in meta.items() if k != "loss"}))


if __name__ == "__main__":
    main()
