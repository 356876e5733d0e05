"""Pins of the oracle's leapfrog update (Sec. 1: compute the forces,
integrate the orbits, repeat), fixed by what the mathematics gives, not by
the oracle itself:

* one update worked by hand;
* the kick-drift-kick leapfrog on a harmonic oscillator, whose positions at
  the whole steps are exactly x_n = x_0 cos(n theta) with
  cos(theta) = 1 - (omega h)^2 / 2 (the Stormer-Verlet recurrence
  x_{n+1} - 2 x_n + x_{n-1} = -(omega h)^2 x_n);
* the two-body circular orbit (masses 1/2 at separation 1, G = 1): radius 1,
  energy -1/8 and period 2 pi are known exactly; a second-order symplectic
  step keeps the radius and the energy and returns to the start after one
  period, up to O(h^2);
* time reversibility of the kick-drift-kick step.
"""
import numpy as np
import pytest

import oracle


def test_one_update_by_hand(orc):
    pos = np.array([[1.0, -2.0, 0.5, 7.0]])
    vel = np.array([[2.0, 1.0, -1.0, 3.0]])
    acc = np.array([[3.0, -4.0, 8.0, -9.0]])
    p, v = oracle.kick_drift(pos, vel, acc, 0.5, 0.25)
    # v' = v + a dt_kick = (3.5, -1, 3); x' = x + v' dt_drift (the new velocity)
    np.testing.assert_array_equal(v, [[3.5, -1.0, 3.0, 3.0]])
    np.testing.assert_array_equal(p, [[1.875, -2.25, 1.25, 7.0]])
    # the inputs are not modified
    assert pos[0, 0] == 1.0 and vel[0, 0] == 2.0


def _harmonic(omega, h, nsteps, merged):
    x = np.array([[1.0, 0.5, -2.0, 7.0]])
    v = np.zeros((1, 4))

    def acc(x):
        a = np.zeros_like(x)
        a[:, :3] = -omega * omega * x[:, :3]
        return a

    a = acc(x)
    xs = []
    for n in range(1, nsteps + 1):
        if merged:  # the two half kicks around each force merged into one kick by h
            x, v = oracle.kick_drift(x, v, a, h / 2 if n == 1 else h, h)
            a = acc(x)
        else:
            x, v = oracle.kick_drift(x, v, a, h / 2, h)
            a = acc(x)
            x, v = oracle.kick_drift(x, v, a, h / 2, 0.0)  # the closing half kick
        xs.append(x[0].copy())
    return np.array(xs)


@pytest.mark.parametrize("merged", [False, True])
def test_harmonic_oscillator_closed_form(orc, merged):
    omega, h = 1.3, 0.05
    xs = _harmonic(omega, h, 200, merged)
    theta = np.arccos(1.0 - (omega * h) ** 2 / 2.0)
    n = np.arange(1, 201)[:, None]
    expect = np.array([1.0, 0.5, -2.0])[None, :] * np.cos(n * theta)
    np.testing.assert_allclose(xs[:, :3], expect, rtol=0, atol=1e-11)
    assert (xs[:, 3] == 7.0).all()


def _two_body_acc(p):
    a = np.zeros_like(p)
    d = p[1, :3] - p[0, :3]
    r = np.linalg.norm(d)
    a[0, :3] = p[1, 3] * d / r ** 3
    a[1, :3] = -p[0, 3] * d / r ** 3
    a[0, 3] = -p[1, 3] / r
    a[1, 3] = -p[0, 3] / r
    return a


def _energy(p, v):
    kin = 0.5 * (p[:, 3] * (v[:, :3] ** 2).sum(axis=1)).sum()
    return kin - p[0, 3] * p[1, 3] / np.linalg.norm(p[1, :3] - p[0, :3])


def test_two_body_circular_orbit(orc):
    p = np.array([[-0.5, 0.0, 0.0, 0.5], [0.5, 0.0, 0.0, 0.5]])
    v = np.array([[0.0, -0.5, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0]])
    assert _energy(p, v) == -0.125
    nstep = 1000
    h = 2.0 * np.pi / nstep  # the period is 2 pi
    p0 = p.copy()
    a = _two_body_acc(p)
    dr, de, back = 0.0, [], []
    for period in range(10):
        for _ in range(nstep):
            p, v = oracle.kick_drift(p, v, a, h / 2, h)
            a = _two_body_acc(p)
            p, v = oracle.kick_drift(p, v, a, h / 2, 0.0)
            dr = max(dr, abs(np.linalg.norm(p[1, :3] - p[0, :3]) - 1.0))
        de.append(abs(_energy(p, v) / -0.125 - 1.0))
        back.append(np.abs(p[:, :3] - p0[:, :3]).max())
    assert dr < 1e-4                     # the circle is kept to O(h^2)
    assert max(de) < 1e-8                # energy: no secular drift
    assert back[0] < 1e-4                # back at the start after one period
    # the phase error grows linearly in time (second order per step)
    assert back[9] < 12 * back[0]
    # total momentum stays zero
    assert np.abs((p[:, 3:4] * v[:, :3]).sum(axis=0)).max() < 1e-14


def test_kick_drift_kick_is_time_reversible(orc):
    rng = np.random.default_rng(7)
    p = np.concatenate([rng.standard_normal((5, 3)), rng.uniform(0.1, 1.0, (5, 1))], axis=1)
    v = np.concatenate([0.3 * rng.standard_normal((5, 3)), np.zeros((5, 1))], axis=1)

    def acc(p):  # softened direct sum (Eq. 1), written out for the five bodies
        a = np.zeros_like(p)
        for i in range(5):
            for j in range(5):
                if i != j:
                    d = p[j, :3] - p[i, :3]
                    a[i, :3] += p[j, 3] * d / (d @ d + 0.01) ** 1.5
        return a

    p0, v0 = p.copy(), v.copy()
    h = 1e-2
    for sweep in range(2):
        for _ in range(50):
            p, v = oracle.kick_drift(p, v, acc(p), h / 2, h)
            p, v = oracle.kick_drift(p, v, acc(p), h / 2, 0.0)
        if sweep == 0:
            v[:, :3] = -v[:, :3]
    np.testing.assert_allclose(p, p0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(-v[:, :3], v0[:, :3], rtol=0, atol=1e-12)
