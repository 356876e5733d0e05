"""Checkpoint files of the leapfrog driver (host side, no GPU): the state
round-trips exactly, the write is atomic, and malformed files are refused."""
import json
import os

import numpy as np
import pytest

from paper_1112_4539_gb300 import leapfrog


def _state(n=1000, seed=0):
    rng = np.random.default_rng(seed)
    pos = rng.standard_normal((n, 4)).astype(np.float32)
    vel = rng.standard_normal((n, 4)).astype(np.float32)
    meta = dict(format=leapfrog.FORMAT, step=7, time=7e-4, dt=1e-4, theta=0.525, eps=1e-3, n=n,
                cfg=dict(leaf_size=16, group_size=96, order=2))
    return pos, vel, meta


def test_round_trip_is_exact(tmp_path):
    pos, vel, meta = _state()
    p = str(tmp_path / "ck.npz")
    leapfrog.save(p, pos, vel, meta)
    pos2, vel2, meta2 = leapfrog.load(p)
    np.testing.assert_array_equal(pos2, pos)
    np.testing.assert_array_equal(vel2, vel)
    assert meta2 == meta
    assert os.listdir(tmp_path) == ["ck.npz"]  # no temporary left behind


def test_overwrite_replaces_the_previous_checkpoint(tmp_path):
    p = str(tmp_path / "ck.npz")
    for seed in (1, 2):
        pos, vel, meta = _state(seed=seed)
        meta["step"] = seed
        leapfrog.save(p, pos, vel, meta)
    pos2, _, meta2 = leapfrog.load(p)
    assert meta2["step"] == 2 and np.array_equal(pos2, _state(seed=2)[0])


def test_malformed_files_are_refused(tmp_path):
    pos, vel, meta = _state()
    with pytest.raises(ValueError):
        leapfrog.save(str(tmp_path / "a.npz"), pos[:, :3], vel[:, :3], meta)
    p = str(tmp_path / "b.npz")
    bad = dict(meta, format=99)
    np.savez(p, pos=pos, vel=vel, meta=np.frombuffer(json.dumps(bad).encode(), np.uint8))
    with pytest.raises(ValueError):
        leapfrog.load(p)
    bad = dict(meta, n=meta["n"] + 1)
    np.savez(p, pos=pos, vel=vel, meta=np.frombuffer(json.dumps(bad).encode(), np.uint8))
    with pytest.raises(ValueError):
        leapfrog.load(p)
