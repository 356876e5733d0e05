"""The orbit loop of Sec. 1 (compute the forces, integrate the orbits,
repeat) as a kick-drift-kick leapfrog around the library's force evaluation,
with checkpoint and resume.

Each step rebuilds the tree from the current positions, evaluates the
forces and applies one leapfrog update on the device (bh_kick_drift): the
first step kicks by dt/2 from the forces at the start, every later step by
dt (the two half kicks between consecutive forces merged), then drifts by dt.
Velocities therefore live at half steps; `synchronised_velocities` adds the
closing half kick without changing the state.

A checkpoint holds the particles (x, y, z, m), the half-step velocities, the
step count, the time, and the settings that define the trajectory; resuming
from it and taking k more steps gives the same bits as not stopping (the
evaluation is deterministic).  Files are written to a temporary name and
renamed, so a crash leaves the previous checkpoint intact.
"""
import json
import os

import numpy as np

from . import Context, _check

FORMAT = 1


class Leapfrog:
    """Kick-drift-kick leapfrog of one particle set on one device.

    pos: (n, 4) float32 tensor (x, y, z, m) on the device, updated in place;
    vel: (n, 4) float32 tensor or None (zero); dt, theta, eps: the step, the
    opening angle and the softening; cfg: Context settings (leaf_size,
    group_size, order, ...)."""

    def __init__(self, pos, vel=None, dt=1e-4, theta=0.5, eps=0.01, step=0, time=0.0, device=0, **cfg):
        import torch
        self.pos = pos
        self.vel = torch.zeros_like(pos) if vel is None else vel
        self.acc = torch.empty_like(pos)
        self.dt, self.theta, self.eps = float(dt), float(theta), float(eps)
        self.step_count, self.time = int(step), float(time)
        self.cfg = dict(cfg)
        self.device = device
        self.ctx = Context(pos.shape[0], device=device, **cfg)

    def close(self):
        self.ctx.close()

    def step(self, nsteps=1, stream=None):
        """Advance nsteps leapfrog steps (stream-ordered, asynchronous)."""
        for _ in range(nsteps):
            self.ctx.evaluate(self.pos, self.theta, self.eps, self.acc, stream=stream)
            kick = 0.5 * self.dt if self.step_count == 0 else self.dt
            self.ctx.kick_drift(self.pos, self.vel, self.acc, kick, self.dt, stream=stream)
            self.step_count += 1
            self.time += self.dt

    def synchronised_velocities(self):
        """Velocities at the current time: the half-step velocities plus the
        closing half kick from the forces at the current positions."""
        import torch
        if self.step_count == 0:
            return self.vel.clone()
        acc = torch.empty_like(self.pos)
        self.ctx.evaluate(self.pos, self.theta, self.eps, acc)
        v = self.vel.clone()
        v[:, :3] += 0.5 * self.dt * acc[:, :3]
        return v

    def status(self):
        return self.ctx.status()

    # ------------------------------------------------------------ checkpoints
    def state(self):
        """Host copy of everything a checkpoint holds."""
        meta = dict(format=FORMAT, step=self.step_count, time=self.time, dt=self.dt, theta=self.theta,
                    eps=self.eps, n=int(self.pos.shape[0]), cfg=self.cfg)
        return self.pos.cpu().numpy(), self.vel.cpu().numpy(), meta

    def checkpoint(self, path):
        """Write the state to `path` (.npz), atomically."""
        _check(self.status(), "device status before checkpoint")
        pos, vel, meta = self.state()
        save(path, pos, vel, meta)

    @classmethod
    def resume(cls, path, device=0):
        """A Leapfrog continuing from the checkpoint at `path`."""
        import torch
        pos, vel, meta = load(path)
        dev = torch.device("cuda", device)
        return cls(torch.from_numpy(pos).to(dev), torch.from_numpy(vel).to(dev), dt=meta["dt"],
                   theta=meta["theta"], eps=meta["eps"], step=meta["step"], time=meta["time"], device=device,
                   **meta["cfg"])


def save(path, pos, vel, meta):
    """Checkpoint file: pos and vel (float32, n x 4) and a JSON record of the
    step, time and settings; written under a temporary name, then renamed."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    vel = np.ascontiguousarray(vel, dtype=np.float32)
    if pos.ndim != 2 or pos.shape[1] != 4 or vel.shape != pos.shape:
        raise ValueError("pos and vel must be (n, 4) arrays of the same shape")
    tmp = "%s.tmp.%d" % (path, os.getpid())
    with open(tmp, "wb") as f:
        np.savez(f, pos=pos, vel=vel, meta=np.frombuffer(json.dumps(meta, sort_keys=True).encode(), np.uint8))
    os.replace(tmp, path)


def load(path):
    """(pos, vel, meta) of a checkpoint written by save."""
    with np.load(path) as z:
        pos, vel = z["pos"].copy(), z["vel"].copy()
        meta = json.loads(z["meta"].tobytes().decode())
    if meta.get("format") != FORMAT:
        raise ValueError("unknown checkpoint format %r" % meta.get("format"))
    if pos.shape != (meta["n"], 4) or vel.shape != pos.shape:
        raise ValueError("checkpoint arrays do not match its record")
    return pos, vel, meta
