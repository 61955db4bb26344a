"""Shared test fixtures: the same seeded systems handed to the CUDA library and
to the oracle, with their interaction sets stated once for both sides."""
import numpy as np

import oracle as O
from paper_2608_14911_gb300 import espp, inputs as I

WCA_RC = 2.0 ** (1.0 / 6.0)


class Case:
    def __init__(self, name, cfg, pair, bond, rc_list, skin, v=None):
        self.name = name
        self.cfg = cfg
        self.pair = pair          # {(a, b): spec} as the oracle takes it
        self.bond = bond
        self.rc_list = rc_list
        self.skin = skin
        self.v = v
        ntypes = int(cfg.types.max()) + 1 if cfg.n else 1
        self.model = O.Model(ntypes, pair, bond)

    def system(self, precision, seed=42, build=True):
        c = self.cfg
        s = espp.System(c.box, c.n, c.types, c.bonds, precision=precision, seed=seed)
        for (a, b), spec in self.pair.items():
            if spec[0] == "wca":
                s.set_wca(spec[1], spec[2], a, b)
            elif spec[0] == "lj":
                s.set_lj(spec[1], spec[2], spec[3], spec[4], a, b)
            elif spec[0] == "lj_capped":
                s.set_lj_capped(spec[1], spec[2], spec[3], spec[5], spec[4], a, b)
        if self.bond is not None:
            s.set_fene(self.bond[1], self.bond[2])
        s.set_state(c.x, self.v, c.img)
        if build:
            s.build_neighbors(self.rc_list, self.skin)
        return s

    def oracle_state(self):
        c = self.cfg
        return O.State(c.box, c.x, self.v, c.img, c.types, c.bonds)


KG_PAIR = {(0, 0): ("wca", 1.0, 1.0)}
KG_BOND = ("fene", 30.0, 1.5)
LJ_PAIR = {(0, 0): ("lj", 1.0, 1.0, 2.5, True)}


def kg_case(nchains=20, nbeads=50, seed=42, jitter=0.05, kT=1.0):
    c = I.kg_lattice(nchains, nbeads, density=0.85, seed=seed, jitter=jitter)
    v = I.maxwell_velocities(c.n, kT, seed=seed)
    return Case("kg%d" % c.n, c, KG_PAIR, KG_BOND, WCA_RC, 0.4, v)


def lj_case(cells=(6, 6, 6), seed=1, kT=0.72, noise=0.08):
    c = I.lj_fcc(*cells, density=0.8442)
    g = np.random.default_rng(seed)
    c.x = I.f32(np.mod(c.x + g.normal(0, noise, c.x.shape), c.box))
    c.x[c.x >= c.box] = 0.0
    v = I.maxwell_velocities(c.n, kT, seed=seed)
    return Case("lj%d" % c.n, c, LJ_PAIR, None, 2.5, 0.3, v)


def two_type_case(seed=3):
    c = I.lj_fcc(6, 6, 7, density=0.7)
    g = np.random.default_rng(seed)
    c.x = I.f32(np.mod(c.x + g.uniform(-0.25, 0.25, c.x.shape), c.box))
    c.x[c.x >= c.box] = 0.0
    c.types = (g.random(c.n) < 0.4).astype(np.int32)
    pair = {(0, 0): ("lj", 1.0, 1.0, 2.5, True), (0, 1): ("lj", 1.5, 0.9, 2.2, True),
            (1, 1): ("wca", 0.7, 1.1)}
    v = I.maxwell_velocities(c.n, 1.0, seed=seed)
    return Case("two%d" % c.n, c, pair, None, 2.5, 0.3, v)


def capped_case(n=1500, L=12.0, seed=9):
    c = I.random_positions(n, (L, L, L), seed=seed)
    pair = {(0, 0): ("lj_capped", 1.0, 1.0, WCA_RC, True, 0.8)}
    return Case("capped%d" % n, c, pair, None, WCA_RC, 0.3, np.zeros((n, 3)))


def rel_rms(a, b):
    den = np.sqrt((b ** 2).sum())
    return np.sqrt(((a - b) ** 2).sum()) / (den if den > 0 else 1.0)
