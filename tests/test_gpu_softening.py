"""GPU parity of individual, symmetrized softening (the symmetrized Plummer
potential that Sec. 7 names as an application, after Saitoh & Makino 2010)
in the paper's per-particle walk: tree_softening + tree_force_particles with
BH_PWALK_INDIVIDUAL_SOFTENING against the oracle's per-particle walk with the
same softening rule (pair: (eps_i^2 + eps_j^2)/2, cell: eps_i^2/2 plus half
the mass-weighted mean eps^2), at the 1e-5 bar of the other force tests."""
import numpy as np
import pytest

import workloads
from test_gpu_parity import MARGIN, _check_force, _cuda

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


def _soft(n, seed, lo=0.002, hi=0.05):
    rng = np.random.default_rng(seed)
    return (10.0 ** rng.uniform(np.log10(lo), np.log10(hi), n)).astype(np.float32)


@pytest.mark.parametrize("kind,n,seed,theta,leaf,order,unsoft,max_level", [
    ("plummer", 4096, 0, 0.5, 8, 1, False, 10),
    ("plummer", 20011, 1, 0.6, 16, 2, False, 10),
    ("clumpy", 30011, 2, 0.5, 8, 2, False, 10),
    ("clumpy", 30011, 2, 0.4, 8, 2, True, 10),
    ("sphere", 10000, 4, 0.8, 1, 1, False, 10),
    ("clumpy", 20000, 3, 0.5, 8, 2, False, 21),
])
def test_symmetrized_softening_matches_oracle(bh, orc, kind, n, seed, theta, leaf, order, unsoft, max_level):
    pos = workloads.make(kind, n, seed)
    eps = _soft(n, seed + 100)
    ctx = bh.Context(n, leaf_size=leaf, group_size=64, order=order, max_level=max_level)
    got = ctx.evaluate_symmetrized(_cuda(pos), _cuda(eps), theta, unsoftened_cells=unsoft).cpu().numpy()
    assert ctx.status() == 0
    st = ctx.stats()
    ref, _ = orc.tree_force_sym(pos, eps, theta, n_leaf=leaf, order=order, max_level=max_level,
                                unsoftened_pc=unsoft)
    _check_force(got.astype(np.float64), ref["out"], ref["margin"], a_abs=ref["a_abs"],
                 case="%s %d symmetrized softening" % (kind, n))
    if (ref["margin"] >= MARGIN).all():
        assert st["n_pp"] == int(ref["n_pp"].sum()) and st["n_pc"] == int(ref["n_pc"].sum())
    ctx.close()


def test_theta_to_zero_is_the_symmetrized_direct_sum(bh, orc):
    pos = workloads.clumpy(5000, seed=7)
    eps = _soft(5000, 8)
    ctx = bh.Context(5000, leaf_size=8, order=2)
    got = ctx.evaluate_symmetrized(_cuda(pos), _cuda(eps), 1e-4).cpu().numpy().astype(np.float64)
    assert ctx.status() == 0
    ref = orc.direct_sym(pos, eps)
    a = np.linalg.norm(ref[:, :3], axis=1)
    ea = np.linalg.norm(got[:, :3] - ref[:, :3], axis=1) / np.maximum(a, 1e-3 * np.median(a))
    assert ea.max() < 1e-5 and (np.abs(got[:, 3] - ref[:, 3]) / np.abs(ref[:, 3])).max() < 1e-5
    ctx.close()


def test_common_softening_gives_the_plain_walk_bits(bh):
    # h_i + h_j = eps^2 exactly when every length is eps, and a cell's mean is eps^2 / 2
    import torch
    pos = workloads.plummer(30000, seed=9)
    eps = np.full(30000, 0.01, np.float32)
    x = _cuda(pos)
    ctx = bh.Context(30000, leaf_size=8, order=2)
    plain = torch.empty_like(x)
    ctx.build(x)
    ctx.moments(0.6)
    ctx.force_particles(float(eps[0]), plain)
    sym = ctx.evaluate_symmetrized(x, _cuda(eps), 0.6)
    assert ctx.status() == 0
    assert torch.equal(plain, sym)
    ctx.close()


def test_softening_state_and_errors(bh):
    import torch
    pos = _cuda(workloads.plummer(1000, seed=1))
    eps = _cuda(_soft(1000, 2))
    out = torch.empty_like(pos)
    ctx = bh.Context(1000)
    assert bh.tree_softening(ctx.h, eps) == bh.BH_ERR_STATE          # no tree yet
    ctx.build(pos)
    ctx.moments(0.5)
    assert bh.tree_force_particles(ctx.h, 0.0, out, individual_softening=True) == bh.BH_ERR_STATE
    ctx.softening(eps)
    assert bh.tree_force_particles(ctx.h, 0.0, out, individual_softening=True) == bh.BH_OK
    ctx.build(pos)                                                     # a new tree clears it
    ctx.moments(0.5)
    assert bh.tree_force_particles(ctx.h, 0.0, out, individual_softening=True) == bh.BH_ERR_STATE
    import ctypes
    assert bh.lib().tree_softening(ctx.h, ctypes.c_void_p(eps.data_ptr() + 2), None) == bh.BH_ERR_INVALID
    bad = eps.clone()
    bad[5] = -1.0
    ctx.softening(bad)
    assert ctx.status() == bh.BH_ERR_NONFINITE
    bad[5] = float("nan")
    ctx.softening(bad)
    assert ctx.status() == bh.BH_ERR_NONFINITE
    ctx.softening(eps)
    assert ctx.status() == bh.BH_OK
    ctx.close()


def test_symmetrized_direct_sum(bh, orc):
    import torch
    pos = workloads.plummer(20000, seed=15)
    eps = _soft(20000, 16)
    x, e = _cuda(pos), _cuda(eps)
    ref = orc.direct_sym(pos, eps)
    idx = np.arange(20000, dtype=np.int64)
    for prec, tol in ((64, 1e-12), (32, 1e-5)):
        out = torch.empty((20000, 4), dtype=torch.float64 if prec == 64 else torch.float32, device="cuda:0")
        assert bh.direct_force_sym(x, e, x, e, _cuda(idx), out, prec) == 0
        got = out.cpu().numpy().astype(np.float64)
        a = np.linalg.norm(ref[:, :3], axis=1)
        ea = np.linalg.norm(got[:, :3] - ref[:, :3], axis=1) / np.maximum(a, 1e-3 * np.median(a))
        assert (np.percentile(ea, 99) if prec == 32 else ea.max()) < tol
    # sampled targets (the error judge's use), and targets that are not sources
    sub = workloads.sample_targets(20000, 300, seed=101)
    out = torch.empty((300, 4), dtype=torch.float64, device="cuda:0")
    assert bh.direct_force_sym(x, e, x[_cuda(sub)].contiguous(), e[_cuda(sub)].contiguous(), _cuda(sub), out, 64) == 0
    np.testing.assert_allclose(out.cpu().numpy(), ref[sub], rtol=1e-12)
    # symmetric pair forces: total momentum vanishes
    out = torch.empty((20000, 4), dtype=torch.float64, device="cuda:0")
    assert bh.direct_force_sym(x, e, x, e, _cuda(idx), out, 64) == 0
    p = (pos[:, 3:4].astype(np.float64) * out.cpu().numpy()[:, :3]).sum(axis=0)
    assert np.abs(p).max() < 1e-12 * (pos[:, 3:4] * np.abs(ref[:, :3])).sum()
