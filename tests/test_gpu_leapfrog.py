"""GPU parity of the leapfrog update (Sec. 1's orbit loop: compute the
forces, integrate, repeat) through the C ABI.

bh_kick_drift computes v' = fma(a, dt_kick, v) and x' = fma(v', dt_drift, x)
in FP32: each component is one correctly rounded FMA of FP32 inputs, so it
differs from the oracle's FP64 update by at most half an FP32 unit in the
last place of v', and x' by half a unit of x' plus dt_drift times the
rounding of v'.  The bar below allows one unit of each (2^-23 relative).
Component 3 of positions (mass) and velocities is never touched.
"""
import numpy as np
import pytest

import workloads
from test_gpu_parity import _check_force, _cuda

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -23


@pytest.fixture(scope="module")
def bh():
    import torch
    assert torch.cuda.is_available()
    from paper_1112_4539_gb300 import _build
    _build.build()
    import paper_1112_4539_gb300 as m
    m.lib()
    return m


def _check_update(x0, v0, a, dtk, dtd, x1, v1, orc):
    # the library receives the time steps as FP32 values
    dtk, dtd = float(np.float32(dtk)), float(np.float32(dtd))
    px, pv = orc.kick_drift(x0.astype(np.float64), v0.astype(np.float64), a.astype(np.float64), dtk, dtd)
    gx, gv = x1.astype(np.float64), v1.astype(np.float64)
    tol_v = ULP * np.abs(pv[:, :3]) + 1e-37
    tol_x = ULP * np.abs(px[:, :3]) + abs(dtd) * ULP * np.abs(pv[:, :3]) + 1e-37
    assert (np.abs(gv[:, :3] - pv[:, :3]) <= tol_v).all(), np.abs(gv[:, :3] - pv[:, :3]).max()
    assert (np.abs(gx[:, :3] - px[:, :3]) <= tol_x).all(), np.abs(gx[:, :3] - px[:, :3]).max()
    np.testing.assert_array_equal(x1[:, 3], x0[:, 3])
    np.testing.assert_array_equal(v1[:, 3], v0[:, 3])


@pytest.mark.parametrize("n", [1, 7, 100003])
@pytest.mark.parametrize("dtk,dtd", [(5e-5, 1e-4), (1e-4, 1e-4), (0.3, -0.7)])
def test_kick_drift_matches_oracle(bh, orc, n, dtk, dtd):
    rng = np.random.default_rng(n)
    x = rng.uniform(-2.0, 2.0, (n, 4)).astype(np.float32)
    v = rng.standard_normal((n, 4)).astype(np.float32)
    a = (rng.standard_normal((n, 4)) * 10.0 ** rng.uniform(-3, 3, (n, 1))).astype(np.float32)
    ctx = bh.Context(max(n, 1), device=0)
    gx, gv, ga = _cuda(x), _cuda(v), _cuda(a)
    ctx.kick_drift(gx, gv, ga, dtk, dtd)
    _check_update(x, v, a, dtk, dtd, gx.cpu().numpy(), gv.cpu().numpy(), orc)
    ctx.close()


def test_kick_drift_empty_and_errors(bh):
    import torch
    ctx = bh.Context(16, device=0)
    e = torch.empty((0, 4), dtype=torch.float32, device="cuda:0")
    ctx.kick_drift(e, e.clone(), e.clone(), 1e-4, 1e-4)
    x = torch.zeros((4, 4), dtype=torch.float32, device="cuda:0")
    import ctypes
    lib = bh.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.bh_kick_drift(ctx.h, ctypes.c_void_p(x.data_ptr() + 4), ctypes.c_void_p(x.data_ptr()),
                             ctypes.c_void_p(x.data_ptr()), 3, ctypes.c_float(1.0), ctypes.c_float(1.0),
                             s) == bh.BH_ERR_INVALID
    assert lib.bh_kick_drift(ctx.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                             ctypes.c_void_p(x.data_ptr()), -1, ctypes.c_float(1.0), ctypes.c_float(1.0),
                             s) == bh.BH_ERR_INVALID
    ctx.close()


def test_ten_kick_drift_kick_steps_clumpy(bh, orc):
    """The clumpy workload's orbit loop at reduced N: ten kick-drift-kick
    steps of dt = 1e-4 from rest (the two half kicks between forces merged),
    the tree rebuilt every step, in the benchmark's kernel configuration.  At
    every step the GPU's forces are checked against the oracle's group walk
    on the GPU's current positions, and the GPU's update against the
    oracle's update of the same inputs."""
    import torch
    n, eps, theta, dt = 30011, 1e-3, 0.525, 1e-4
    pos = workloads.clumpy(n, seed=2)
    ctx = bh.Context(n, device=0, leaf_size=16, group_size=96, order=2)
    x = _cuda(pos)
    v = torch.zeros_like(x)
    acc = torch.empty_like(x)
    for step in range(10):
        ctx.evaluate(x, theta, eps, acc)
        assert ctx.status() == 0
        xs, vs, a = x.cpu().numpy(), v.cpu().numpy(), acc.cpu().numpy()
        ref, _ = orc.tree_force(xs, theta, eps, n_leaf=16, G=96, order=2, walk="group")
        _check_force(a.astype(np.float64), ref["out"], ref["margin"], a_abs=ref["a_abs"],
                     case="clumpy %d leapfrog step %d" % (n, step))
        dtk = dt / 2 if step == 0 else dt
        ctx.kick_drift(x, v, acc, dtk, dt)
        _check_update(xs, vs, a, dtk, dt, x.cpu().numpy(), v.cpu().numpy(), orc)
    assert np.abs(x.cpu().numpy()[:, :3] - pos[:, :3]).max() > 0  # the particles moved
    ctx.close()


def test_checkpoint_and_resume_give_the_same_bits(bh, tmp_path):
    """Six leapfrog steps straight through, against three steps, a
    checkpoint, a resume into a new driver and three more steps."""
    import torch
    from paper_1112_4539_gb300 import leapfrog
    pos = workloads.clumpy(40000, seed=5)
    cfg = dict(leaf_size=16, group_size=96, order=2)
    a = leapfrog.Leapfrog(_cuda(pos), dt=1e-4, theta=0.525, eps=1e-3, **cfg)
    a.step(6)
    assert a.status() == 0
    b = leapfrog.Leapfrog(_cuda(pos), dt=1e-4, theta=0.525, eps=1e-3, **cfg)
    b.step(3)
    p = str(tmp_path / "ck.npz")
    b.checkpoint(p)
    b.close()
    c = leapfrog.Leapfrog.resume(p)
    assert c.step_count == 3 and abs(c.time - 3e-4) < 1e-15 and c.cfg == cfg
    c.step(3)
    assert c.status() == 0
    assert torch.equal(a.pos, c.pos) and torch.equal(a.vel, c.vel)
    # the closing half kick synchronises the velocities without touching the state
    v = c.synchronised_velocities()
    assert torch.equal(c.vel, a.vel) and not torch.equal(v, c.vel)
    a.close()
    c.close()
