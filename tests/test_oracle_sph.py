"""Pins of the oracle's neighbour search and SPH density (the short-range use
of the general tree walk, Sec. 4.3) against things other than itself: the
kernel's normalisation and shape, exact lattice sums, and scipy's k-d tree."""
import numpy as np
import pytest

import workloads


def test_kernel_normalised_and_continuous(orc):
    from scipy.integrate import quad
    for h in (0.3, 1.0, 2.5):
        integral, _ = quad(lambda r: 4.0 * np.pi * r * r * orc.sph_kernel(r, h), 0.0, h, points=[0.5 * h],
                           epsabs=1e-13, epsrel=1e-12)
        assert abs(integral - 1.0) < 1e-10
        c = 8.0 / (np.pi * h ** 3)
        assert orc.sph_kernel(0.0, h) == pytest.approx(c, rel=1e-15)
        assert orc.sph_kernel(0.5 * h, h) == pytest.approx(0.25 * c, rel=1e-14)        # both pieces meet
        assert orc.sph_kernel(0.5 * h * (1 + 1e-9), h) == pytest.approx(0.25 * c, rel=1e-7)
        assert orc.sph_kernel(h, h) == 0.0 and orc.sph_kernel(1.5 * h, h) == 0.0


def test_lattice_counts_and_density(orc):
    # cubic lattice, spacing a = 1/8 (coordinates exact in FP32), h = 4a:
    # interior neighbours are the integer vectors with 0 < |v|^2 < 16, and the
    # SPH density of a uniform lattice is m / a^3 up to the kernel's lattice
    # discretisation error
    a, k = 0.125, 14
    g = np.arange(k, dtype=np.float32) * np.float32(a)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel(), np.full(X.size, 1.0, np.float32)], 1).astype(np.float32)
    h = 4 * a
    count, rho = orc.sph_density(pos, h)
    v = np.arange(-4, 5)
    V = np.array(np.meshgrid(v, v, v, indexing="ij")).reshape(3, -1).T
    r2 = (V * V).sum(1)
    want = int(((r2 > 0) & (r2 < 16)).sum())
    interior = np.all((pos[:, :3] >= 4 * a) & (pos[:, :3] <= (k - 5) * a), axis=1)
    assert interior.sum() > 100
    assert (count[interior] == want).all()
    # exact lattice sum of the kernel for the interior particles
    lat = sum(orc.sph_kernel(np.sqrt(q) * a, h) for q in r2[r2 < 16])
    np.testing.assert_allclose(rho[interior], lat, rtol=1e-12)
    assert abs(lat * a ** 3 - 1.0) < 2e-3  # rho ~ m / a^3


@pytest.mark.parametrize("kind,n,seed", [("clumpy", 6000, 3), ("plummer", 5000, 4)])
def test_counts_match_kdtree(orc, kind, n, seed):
    from scipy.spatial import cKDTree
    pos = workloads.make(kind, n, seed)
    rng = np.random.default_rng(seed)
    x = pos[:, :3].astype(np.float64)
    h = (0.02 + 0.08 * rng.random(n)).astype(np.float32)
    count, rho = orc.sph_density(pos, h)
    t = cKDTree(x)
    lo = np.array([len(t.query_ball_point(x[i], float(h[i]) * (1 - 1e-5))) - 1 for i in range(n)])
    hi = np.array([len(t.query_ball_point(x[i], float(h[i]) * (1 + 1e-5))) - 1 for i in range(n)])
    assert (lo <= count).all() and (count <= hi).all()
    assert (lo == hi).mean() > 0.99 and (count[lo == hi] == lo[lo == hi]).all()
    # density from the k-d tree's neighbour lists (FP64 distances) agrees to FP32 rounding of r
    for i in rng.choice(n, 200, replace=False):
        js = [j for j in t.query_ball_point(x[i], float(h[i]) * (1 - 1e-5)) if j != i]
        if lo[i] != hi[i]:
            continue
        want = pos[i, 3] * orc.sph_kernel(0.0, h[i]) + sum(
            pos[j, 3] * orc.sph_kernel(np.linalg.norm(x[j] - x[i]), h[i]) for j in js)
        assert rho[i] == pytest.approx(want, rel=1e-5)


def test_coincident_particles_are_neighbours(orc):
    # R19: distinct particles at the same position are neighbours (their
    # distance 0 is below any radius); only the particle itself is excluded
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(9)
    knot = np.tile(np.array([[0.5, 0.5, 0.5, 1.0]], np.float32), (40, 1))
    rest = np.concatenate([rng.random((500, 3)), np.ones((500, 1))], 1).astype(np.float32)
    pos = np.concatenate([knot, rest])
    h = np.full(pos.shape[0], 0.1, np.float32)
    count, rho = orc.sph_density(pos, h)
    t = cKDTree(pos[:, :3].astype(np.float64))
    want = np.array([len(t.query_ball_point(pos[i, :3], 0.1 * (1 - 1e-6))) - 1 for i in range(40)])
    assert (count[:40] == want).all() and (want >= 39).all()
