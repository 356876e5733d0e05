"""Seeded synthetic particle sets for the force evaluation (inputs only).

This module holds none of the method's arithmetic: it only draws particle
positions and masses.  Both the CUDA path's tests and benchmark and the CPU
oracle's tests consume its arrays.  All draws use numpy's counter-based
Philox generator keyed by the seed, so a (kind, n, seed) triple always gives
the same float32 (n, 4) array of (x, y, z, m).

The paper measures on randomly filled spheres and a GalactICS disk galaxy
(Sec. 5); neither data set exists here, so these generators stand in for them:
  plummer    Plummer sphere, unit mass and scale radius, truncated at r = 20;
  clumpy     64 Hernquist spheres (a = 0.05, truncated at 20 a) with masses
             log-uniform over one decade and centres uniform in the unit cube,
             holding 80% of the particles, plus 20% uniform background in the
             unit cube; equal-mass particles, total mass 1;
  uniform    uniform cube [0, 1]^3 (the paper's Sec. 6.3 comparison set);
  sphere     uniform ball of radius 1 (the paper's Sec. 5 random sphere);
  batched    many Plummer spheres with N drawn log-uniformly in [nmin, nmax].
"""
import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _isotropic(rng, n):
    """Unit vectors uniform on the sphere."""
    z = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1)


def plummer_radii(rng, n, rmax=20.0):
    """Radii of a unit Plummer sphere by inverse CDF, M(<r) = r^3 / (1 + r^2)^1.5,
    redrawing any radius beyond rmax."""
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x = rng.uniform(0.0, 1.0, todo.size)
        x = np.maximum(x, 1e-300)
        rr = 1.0 / np.sqrt(np.maximum(x ** (-2.0 / 3.0) - 1.0, 1e-300))
        ok = rr <= rmax
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    return r


def plummer(n, seed=0, rmax=20.0, mass=1.0):
    """Plummer sphere of total mass `mass` and unit scale radius, truncated at rmax."""
    rng = _rng(seed)
    r = plummer_radii(rng, n, rmax)
    x = r[:, None] * _isotropic(rng, n)
    out = np.empty((n, 4), dtype=np.float32)
    out[:, :3] = x
    out[:, 3] = np.float32(mass / max(n, 1))
    return out


def hernquist_radii(rng, n, a, cut=20.0):
    """Hernquist radii by inverse CDF, M(<r) = r^2 / (r + a)^2, truncated at cut * a."""
    xmax = (cut / (cut + 1.0)) ** 2
    x = rng.uniform(0.0, xmax, n)
    s = np.sqrt(x)
    return a * s / (1.0 - s)


def clumpy(n, seed=2, n_clumps=64, a=0.05, background=0.2):
    """64 Hernquist clumps + uniform background (equal-mass particles, total mass 1)."""
    rng = _rng(seed)
    n_bg = int(round(background * n))
    n_cl = n - n_bg
    w = 10.0 ** rng.uniform(0.0, 1.0, n_clumps)
    w = w / w.sum()
    # particles per clump proportional to clump mass (largest remainder)
    exact = w * n_cl
    cnt = np.floor(exact).astype(np.int64)
    rem = n_cl - int(cnt.sum())
    if rem > 0:
        cnt[np.argsort(-(exact - cnt), kind="stable")[:rem]] += 1
    centres = rng.uniform(0.0, 1.0, (n_clumps, 3))
    parts = []
    for c in range(n_clumps):
        k = int(cnt[c])
        if k == 0:
            continue
        r = hernquist_radii(rng, k, a)
        parts.append(centres[c] + r[:, None] * _isotropic(rng, k))
    parts.append(rng.uniform(0.0, 1.0, (n_bg, 3)))
    x = np.concatenate(parts, axis=0)
    # shuffle so the caller's order carries no spatial structure
    x = x[rng.permutation(n)]
    out = np.empty((n, 4), dtype=np.float32)
    out[:, :3] = x
    out[:, 3] = np.float32(1.0 / max(n, 1))
    return out


def uniform_cube(n, seed=0):
    rng = _rng(seed)
    out = np.empty((n, 4), dtype=np.float32)
    out[:, :3] = rng.uniform(0.0, 1.0, (n, 3))
    out[:, 3] = np.float32(1.0 / max(n, 1))
    return out


def uniform_sphere(n, seed=0):
    rng = _rng(seed)
    r = rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    out = np.empty((n, 4), dtype=np.float32)
    out[:, :3] = r[:, None] * _isotropic(rng, n)
    out[:, 3] = np.float32(1.0 / max(n, 1))
    return out


def batched_sizes(n_sys, nmin=1024, nmax=65536, seed=3):
    """System sizes N_k = round(2^U(log2 nmin, log2 nmax))."""
    rng = _rng(seed)
    e = rng.uniform(np.log2(nmin), np.log2(nmax), n_sys)
    return np.rint(2.0 ** e).astype(np.int64)


def batched_plummer(n_sys=512, nmin=1024, nmax=65536, seed=3):
    """Concatenated independent Plummer spheres; returns (pos (sum N, 4), offsets (n_sys+1,))."""
    sizes = batched_sizes(n_sys, nmin, nmax, seed)
    offs = np.zeros(n_sys + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    pos = np.empty((int(offs[-1]), 4), dtype=np.float32)
    for k in range(n_sys):
        pos[offs[k]:offs[k + 1]] = plummer(int(sizes[k]), seed=1000 * int(seed) + k)
    return pos, offs


def plummer_search_radii(pos, n_ngb=64):
    """Search radii for a unit Plummer sphere (unit mass) that enclose about
    n_ngb neighbours: (4/3) pi h^3 rho(r) N = n_ngb with the analytic density
    rho(r) = 3 / (4 pi) (1 + r^2)^(-5/2)."""
    n = pos.shape[0]
    r2 = (pos[:, :3].astype(np.float64) ** 2).sum(1)
    rho = 3.0 / (4.0 * np.pi) * (1.0 + r2) ** -2.5
    return ((3.0 * n_ngb) / (4.0 * np.pi * rho * n)) ** (1.0 / 3.0)


def softening_lengths(n, eps, seed=17, spread=4.0):
    """Individual softening lengths, log-uniform in [eps/spread, eps*spread]
    (float32, seeded): a stand-in for per-particle softening of mixed mass
    resolution."""
    rng = _rng(seed)
    return (eps * np.exp(rng.uniform(-np.log(spread), np.log(spread), n))).astype(np.float32)


def sample_targets(n, n_sample=4096, seed=101):
    """Seeded, sorted, distinct sample of target indices for the FP64 error check."""
    rng = _rng(seed)
    k = min(n, n_sample)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def make(kind, n, seed):
    if kind == "plummer":
        return plummer(n, seed)
    if kind == "clumpy":
        return clumpy(n, seed)
    if kind == "uniform":
        return uniform_cube(n, seed)
    if kind == "sphere":
        return uniform_sphere(n, seed)
    raise ValueError(kind)
