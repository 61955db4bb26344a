"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only (positions, velocities, topologies,
replica sizes); none of the method's arithmetic.  Both the CUDA library and the
oracle consume what it produces.  Every coordinate, velocity and box edge it
returns is a float64 that is exactly representable in float32, so a float32
store of the state loses nothing and both sides see identical inputs.

Random numbers come from numpy's Philox bit generator keyed by (seed, tag), so
each kind of draw has its own stream.
"""
from dataclasses import dataclass, field

import numpy as np

TAG_VELOCITIES = 1
TAG_CHAINS = 2
TAG_REPLICAS = 3
TAG_POSITIONS = 5


def rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(tag)]))


def f32(a):
    """Round to the nearest float32 value, returned as float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@dataclass
class Config:
    """One synthetic system in id order."""
    box: np.ndarray                      # (3,) float64, float32-exact
    x: np.ndarray                        # (n,3) in [0, box), float32-exact
    img: np.ndarray                      # (n,3) int32 image counters
    types: np.ndarray                    # (n,) int32
    bonds: np.ndarray                    # (nb,2) int64 particle ids
    v: np.ndarray = None                 # (n,3) or None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _wrap_unwrapped(u: np.ndarray, box: np.ndarray):
    """Split unwrapped float64 coordinates into float32-exact x in [0, L) and
    integer images, so that x + img * L reproduces u up to float32 rounding."""
    img = np.floor(u / box).astype(np.int64)
    x = f32(u - img * box)
    over = x >= box
    x[over] -= box[np.nonzero(over)[1]]
    img[over] += 1
    neg = x < 0
    x[neg] = 0.0
    return x, img.astype(np.int32)


def cubic_box(n: int, density: float) -> np.ndarray:
    return f32(np.full(3, (n / density) ** (1.0 / 3.0)))


def chain_bonds(nchains: int, nbeads: int) -> np.ndarray:
    """Linear chains of consecutive ids: chain c holds ids c*nbeads .. +nbeads-1."""
    base = (np.arange(nchains, dtype=np.int64) * nbeads)[:, None]
    k = np.arange(nbeads - 1, dtype=np.int64)[None, :]
    a = (base + k).reshape(-1)
    return np.stack([a, a + 1], axis=1)


def kg_random_walk(nchains: int, nbeads: int, density: float = 0.85, seed: int = 42,
                   bond: float = 0.97) -> Config:
    """Kremer-Grest melt start: chain starts uniform in a cubic box, each next
    bead a step of length `bond` in a uniformly random direction (no
    self-avoidance).  Overlaps are expected; a soft push-off removes them."""
    n = nchains * nbeads
    box = cubic_box(n, density)
    g = rng(seed, TAG_CHAINS)
    start = g.random((nchains, 1, 3)) * box
    d = g.normal(size=(nchains, nbeads - 1, 3))
    d *= bond / np.linalg.norm(d, axis=2, keepdims=True)
    u = np.concatenate([start, start + np.cumsum(d, axis=1)], axis=1).reshape(-1, 3)
    x, img = _wrap_unwrapped(u, box)
    return Config(box, x, img, np.zeros(n, np.int32), chain_bonds(nchains, nbeads),
                  meta=dict(kind="kg_random_walk", nchains=nchains, nbeads=nbeads,
                            density=density, seed=seed))


def snake_sites(m: int) -> np.ndarray:
    """Sites of an m^3 simple cubic grid in boustrophedon order: consecutive
    sites are always face neighbours."""
    z = np.repeat(np.arange(m), m * m)
    yi = np.tile(np.repeat(np.arange(m), m), m)          # row index inside a plane
    y = np.where(z % 2 == 0, yi, m - 1 - yi)
    row = z * m + yi                                      # global row counter
    xi = np.tile(np.arange(m), m * m)
    x = np.where(row % 2 == 0, xi, m - 1 - xi)
    return np.stack([x, y, z], axis=1).astype(np.int64)


def kg_lattice(nchains: int, nbeads: int, density: float = 0.85, seed: int = 42,
               jitter: float = 0.05) -> Config:
    """Overlap-free Kremer-Grest start: beads on a simple cubic grid of
    ceil(n^(1/3))^3 sites filling the cubic box, taken in boustrophedon order
    and cut into chains, then jittered uniformly by +-jitter.  Bonded beads are
    one grid spacing apart (1.0557 sigma at density 0.85 when n is a cube)."""
    n = nchains * nbeads
    box = cubic_box(n, density)
    m = int(np.ceil(n ** (1.0 / 3.0) - 1e-9))
    a = box[0] / m
    sites = snake_sites(m)[:n]
    g = rng(seed, TAG_CHAINS)
    u = (sites + 0.5) * a + g.uniform(-jitter, jitter, size=(n, 3))
    x, img = _wrap_unwrapped(u, box)
    return Config(box, x, img, np.zeros(n, np.int32), chain_bonds(nchains, nbeads),
                  meta=dict(kind="kg_lattice", nchains=nchains, nbeads=nbeads,
                            density=density, seed=seed, spacing=float(a)))


def lj_fcc(nx: int, ny: int, nz: int, density: float = 0.8442) -> Config:
    """Face-centred cubic lattice of nx*ny*nz unit cells (4 atoms each) at the
    given number density; orthorhombic box nx*a x ny*a x nz*a."""
    a = (4.0 / density) ** (1.0 / 3.0)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) + 0.25
    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1).astype(np.float64)
    u = ((cells[:, None, :] + basis[None, :, :]) * a).reshape(-1, 3)
    box = f32(np.array([nx * a, ny * a, nz * a]))
    x, img = _wrap_unwrapped(u, box)
    n = x.shape[0]
    return Config(box, x, img, np.zeros(n, np.int32), np.zeros((0, 2), np.int64),
                  meta=dict(kind="lj_fcc", cells=(nx, ny, nz), density=density))


def random_positions(n: int, box, seed: int = 42) -> Config:
    """Uniformly random positions (the example script's getRandomPos start)."""
    box = f32(np.asarray(box, dtype=np.float64))
    g = rng(seed, TAG_POSITIONS)
    x, img = _wrap_unwrapped(g.random((n, 3)) * box, box)
    return Config(box, x, img, np.zeros(n, np.int32), np.zeros((0, 2), np.int64),
                  meta=dict(kind="random", seed=seed))


def maxwell_velocities(n: int, kT: float, seed: int = 42, mass: float = 1.0) -> np.ndarray:
    """Gaussian velocities with the centre-of-mass velocity removed and the
    kinetic temperature sum(m v^2)/(3n) rescaled to kT exactly (before the
    float32 rounding)."""
    g = rng(seed, TAG_VELOCITIES)
    v = g.normal(size=(n, 3)) * np.sqrt(kT / mass)
    v -= v.mean(axis=0, keepdims=True)
    t = mass * (v * v).sum() / (3.0 * n)
    if t > 0:
        v *= np.sqrt(kT / t)
    return f32(v)


def replica_sizes(R: int, seed: int = 42, chains=(10, 400), length=(20, 200)):
    """(nchains, nbeads) per replica: both uniform integers on the closed ranges."""
    g = rng(seed, TAG_REPLICAS)
    nc = g.integers(chains[0], chains[1] + 1, size=R)
    nb = g.integers(length[0], length[1] + 1, size=R)
    return [(int(a), int(b)) for a, b in zip(nc, nb)]
