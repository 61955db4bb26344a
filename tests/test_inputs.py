"""The seeded input generators keep their contracts: float32-exact values,
coordinates inside the box with images that rebuild the unwrapped chains,
the stated densities, bond lengths and lattice geometry, Maxwell velocities at
the target temperature with no net momentum, reproducible streams.  CPU only."""
import numpy as np
import pytest

from paper_2608_14911_gb300 import inputs as I


def _f32_exact(a):
    a = np.asarray(a, dtype=np.float64)
    return np.array_equal(a, a.astype(np.float32).astype(np.float64))


def _inside(c):
    return bool(np.all(c.x >= 0.0) and np.all(c.x < c.box))


@pytest.mark.parametrize("gen", ["walk", "lattice"])
def test_kg_starts(gen):
    nch, nb, rho = 30, 40, 0.85
    c = (I.kg_random_walk(nch, nb, density=rho, seed=5) if gen == "walk"
         else I.kg_lattice(nch, nb, density=rho, seed=5, jitter=0.05))
    n = nch * nb
    assert c.n == n and _f32_exact(c.x) and _f32_exact(c.box) and _inside(c)
    assert abs(n / np.prod(c.box) - rho) < 1e-5 * rho
    # chains of consecutive ids
    assert c.bonds.shape == (nch * (nb - 1), 2)
    assert np.all(c.bonds[:, 1] == c.bonds[:, 0] + 1)
    assert not np.any((c.bonds[:, 0] + 1) % nb == 0)
    # unwrapped bond vectors: x + img L along each chain
    u = c.x + c.img * c.box
    b = np.linalg.norm(u[c.bonds[:, 1]] - u[c.bonds[:, 0]], axis=1)
    if gen == "walk":
        assert np.abs(b - 0.97).max() < 1e-5
    else:
        a = c.meta["spacing"]
        assert np.abs(b - a).max() <= 2 * np.sqrt(3) * 0.05 + 1e-5
        # overlap-free: no two beads closer than the spacing minus the jitter
        d = c.x[:, None, :] - c.x[None, :, :]
        d -= c.box * np.round(d / c.box)
        r = np.sqrt((d ** 2).sum(axis=2)) + np.eye(n) * 1e9
        assert r.min() > a - 2 * np.sqrt(3) * 0.05 - 1e-6
    # the same seed gives the same system, another seed another one
    again = (I.kg_random_walk(nch, nb, density=rho, seed=5) if gen == "walk"
             else I.kg_lattice(nch, nb, density=rho, seed=5, jitter=0.05))
    assert np.array_equal(again.x, c.x) and np.array_equal(again.img, c.img)
    other = (I.kg_random_walk(nch, nb, density=rho, seed=6) if gen == "walk"
             else I.kg_lattice(nch, nb, density=rho, seed=6, jitter=0.05))
    assert not np.array_equal(other.x, c.x)


def test_snake_sites_are_face_neighbours():
    for m in (2, 3, 5):
        s = I.snake_sites(m)
        assert len({tuple(p) for p in s}) == m ** 3
        assert np.all(np.abs(np.diff(s, axis=0)).sum(axis=1) == 1)


def test_lj_fcc_lattice():
    c = I.lj_fcc(4, 5, 6, density=0.8442)
    assert c.n == 4 * 4 * 5 * 6 and _inside(c) and _f32_exact(c.x)
    assert abs(c.n / np.prod(c.box) - 0.8442) < 1e-5
    a = (4.0 / 0.8442) ** (1.0 / 3.0)
    d = c.x[:, None, :] - c.x[None, :, :]
    d -= c.box * np.round(d / c.box)
    r = np.sqrt((d ** 2).sum(axis=2)) + np.eye(c.n) * 1e9
    # every site has its 12 nearest neighbours at a / sqrt(2)
    nn = (np.abs(r - a / np.sqrt(2)) < 1e-5).sum(axis=1)
    assert np.all(nn == 12) and abs(r.min() - a / np.sqrt(2)) < 1e-5


def test_random_positions_fill_the_box():
    box = np.array([7.0, 9.0, 11.0])
    c = I.random_positions(20000, box, seed=3)
    assert _inside(c) and _f32_exact(c.x)
    # uniform: each half of each edge holds about half the particles
    for k in range(3):
        frac = (c.x[:, k] < box[k] / 2).mean()
        assert abs(frac - 0.5) < 5 * np.sqrt(0.25 / c.n)


@pytest.mark.parametrize("kT,mass", [(1.0, 1.0), (0.72, 1.0), (2.0, 3.0)])
def test_maxwell_velocities(kT, mass):
    n = 5000
    v = I.maxwell_velocities(n, kT, seed=9, mass=mass)
    assert v.shape == (n, 3) and _f32_exact(v)
    assert np.abs(v.mean(axis=0)).max() < 1e-6
    assert abs(mass * (v * v).sum() / (3 * n) - kT) < 1e-5 * kT
    # Gaussian: the fourth moment of a component is 3 sigma^4
    s2 = kT / mass
    k4 = (v ** 4).mean() / s2 ** 2
    assert abs(k4 - 3.0) < 0.25


def test_replica_sizes():
    sizes = I.replica_sizes(512, seed=42)
    nc = np.array([a for a, _ in sizes])
    nb = np.array([b for _, b in sizes])
    assert len(sizes) == 512
    assert nc.min() >= 10 and nc.max() <= 400 and nb.min() >= 20 and nb.max() <= 200
    # uniform on the closed ranges: the means sit near the middles
    assert abs(nc.mean() - 205) < 5 * 113 / np.sqrt(512)
    assert abs(nb.mean() - 110) < 5 * 52 / np.sqrt(512)
    assert I.replica_sizes(512, seed=42) == sizes
