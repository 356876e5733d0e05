"""Bounded device waits end, are reported, and leave the context usable.

The library's kernels wait in three places: the paired walk's tile ring
(mbarriers), the sort's decoupled look-back and the TMA-staged walk's
mbarriers for its bulk copies.  bh_selftest_wait launches
one such wait that nothing will satisfy, through the same device functions;
the test checks that it gives up on its own, that bh_status reports
BH_ERR_DEVICE_TIMEOUT once (then clears it), and that the next force
evaluation on the same context gives the same bits as before.  Nothing here
faults or traps the GPU: the wait ends by its own limit.
"""
import time

import numpy as np
import pytest

import workloads
from test_gpu_parity import _cuda

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


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_wait_times_out_and_context_recovers(bh, which):
    pos = workloads.plummer(4096, seed=0)
    x = _cuda(pos)
    for variant in (bh.WALK_ONE_WARP, bh.WALK_PAIRED, bh.WALK_TMA):
        ctx = bh.Context(4096, leaf_size=8, group_size=64, order=2, walk_variant=variant)
        ref = ctx.evaluate(x, 0.5, 0.01).cpu().numpy()
        assert ctx.status() == bh.BH_OK
        t0 = time.perf_counter()
        assert bh.bh_selftest_wait(ctx.h, which) == bh.BH_OK
        assert ctx.status() == bh.BH_ERR_DEVICE_TIMEOUT
        assert time.perf_counter() - t0 < 30.0
        assert ctx.status() == bh.BH_OK  # reported once, then cleared
        got = ctx.evaluate(x, 0.5, 0.01).cpu().numpy()
        assert ctx.status() == bh.BH_OK
        np.testing.assert_array_equal(got, ref)
        ctx.close()


def test_selftest_rejects_unknown_wait(bh):
    ctx = bh.Context(16)
    assert bh.bh_selftest_wait(ctx.h, 7) == bh.BH_ERR_INVALID
    ctx.close()
