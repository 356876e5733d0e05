"""The allocation-free entry point against the regular one.

bh_tree_force_static serves callers that cannot call cudaMalloc (code running
during CUDA graph capture, plugins whose host owns all device memory,
real-time loops that must not allocate).  It keeps its work arrays in a fixed
device array instead of a context's slab, so its results must match the
context path's.  This file is collected last on purpose: a failure here comes
after every other test has run.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _rel(got, ref):
    a_ref = np.linalg.norm(ref[:, :3], axis=1)
    den = np.maximum(a_ref, 1e-3 * np.median(a_ref))
    ea = np.linalg.norm(got[:, :3] - ref[:, :3], axis=1) / den
    ep = np.abs(got[:, 3] - ref[:, 3]) / np.abs(ref[:, 3])
    return ea.max(), ep.max()


def test_static_entry_matches_context_path_twice():
    import torch
    from paper_1112_4539_gb300 import _build
    _build.build()
    import paper_1112_4539_gb300 as bh

    theta, eps = 0.5, 0.01
    cfg = dict(leaf_size=8, group_size=64, order=2)
    # two calls in a row, the second with a different and larger system
    for kind, n, seed in (("plummer", 20000, 21), ("clumpy", bh.STATIC_MAX_N, 22)):
        pos = workloads.make(kind, n, seed)
        x = torch.from_numpy(pos).to("cuda:0")
        ctx = bh.Context(n, device=0, **cfg)
        ref = ctx.evaluate(x, theta, eps).cpu().numpy().astype(np.float64)
        assert ctx.status() == 0
        ctx.close()
        out = torch.full_like(x, float("nan"))
        rc, st = bh.bh_tree_force_static(x, theta, eps, out, bh.config(**cfg))
        assert rc == bh.BH_OK and st == bh.BH_OK
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        ea, ep = _rel(got, ref)
        assert ea <= 1e-5 and ep <= 1e-5, (kind, ea, ep)
    # beyond the stated maximum: a clear error, nothing launched
    big = torch.zeros((bh.STATIC_MAX_N + 1, 4), dtype=torch.float32, device="cuda:0")
    rc, _ = bh.bh_tree_force_static(big, theta, eps, torch.empty_like(big))
    assert rc == bh.BH_ERR_TOO_LARGE


def test_static_entry_replays_from_a_cuda_graph():
    # The reason for the entry point: captured once into a CUDA graph (after a
    # first, synchronous call on the device), the graph replays the whole
    # evaluation on whatever particles the input buffer holds, with the bits of
    # a direct call.
    import torch
    from paper_1112_4539_gb300 import _build
    _build.build()
    import paper_1112_4539_gb300 as bh

    n, theta, eps = 20000, 0.5, 0.01
    cfg = bh.config(leaf_size=8, group_size=64, order=2)
    x = torch.from_numpy(workloads.plummer(n, seed=30)).to("cuda:0")
    out = torch.empty_like(x)
    rc, st = bh.bh_tree_force_static(x, theta, eps, out, cfg)
    assert rc == bh.BH_OK and st == bh.BH_OK
    ref1 = out.clone()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        rc, st = bh.bh_tree_force_static(x, theta, eps, out, cfg, status=False)
    assert rc == bh.BH_OK and st is None
    out.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref1)
    # new particles in the same buffer, alternating with the first set: every
    # replay's sort takes fresh look-back epochs from the device's build
    # counter, so no replay can read a word an earlier replay left behind
    sets = [torch.from_numpy(workloads.plummer(n, seed=30)).to("cuda:0"),
            torch.from_numpy(workloads.clumpy(n, seed=31)).to("cuda:0")]
    refs = []
    for s in sets:
        r = torch.empty_like(x)
        rc, st = bh.bh_tree_force_static(s, theta, eps, r, cfg)
        assert rc == bh.BH_OK and st == bh.BH_OK
        refs.append(r)
    for k in range(6):
        x.copy_(sets[(k + 1) % 2])
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, refs[(k + 1) % 2]), k
    del g
