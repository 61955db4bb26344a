"""Pins for the oracle: checks against what the mathematics and the literature
fix, independent of the oracle's own code (closed forms, known-answer vectors,
brute force, invariants, limits).  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2608_14911_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_values():
    vals = {}
    with open(os.path.join(GOLDEN, "literature_values.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, value, tol = line.split()[:3]
            vals[name] = (float(value), float(tol))
    return vals


LIT = golden_values()
KG = O.Model(1, {(0, 0): ("wca", 1.0, 1.0)}, ("fene", 30.0, 1.5))


# --------------------------------------------------------------------------
# Philox and the noise map
# --------------------------------------------------------------------------
def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = O.philox(r[0:4], r[4:6])
        assert [int(v) for v in out] == r[6:10]


def test_uniform_map_is_the_odd_grid():
    # every top-24-bit pattern must land on a distinct odd multiple of 2^-25
    k = np.arange(2 ** 24, dtype=np.uint64)
    words = ((k << np.uint64(8)) | np.uint64(0xA5)).astype(np.uint32)
    r = O.uniform_centered(words)
    j = np.round(r * 2.0 ** 25).astype(np.int64)
    assert np.all(j.astype(np.float64) * 2.0 ** -25 == r)
    expect = np.arange(-(2 ** 24 - 1), 2 ** 24, 2, dtype=np.int64)
    assert np.array_equal(np.sort(j), expect)
    assert r.max() < 0.5 and r.min() > -0.5
    # low 8 bits are ignored
    assert O.uniform_centered(np.array([0x12345600], np.uint32))[0] == \
        O.uniform_centered(np.array([0x123456ff], np.uint32))[0]


def test_langevin_noise_keying():
    a = O.langevin_noise(42, 7, 5)
    b = O.langevin_noise(42, 7, 5)
    c = O.langevin_noise(42, 8, 5)
    d = O.langevin_noise(43, 7, 5)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c) and not np.array_equal(a, d)
    # particle i at step s uses counter (i, s_lo, s_hi, 0) under key (seed_lo, seed_hi)
    out = O.philox([3, 7, 0, 0], [42, 0])
    assert np.array_equal(a[3], O.uniform_centered(out[:3]))
    big = (1 << 33) + 5
    out = O.philox([1, big & 0xffffffff, big >> 32, 0], [(9 << 32 | 11) & 0xffffffff, 9])
    assert np.array_equal(O.langevin_noise((9 << 32) | 11, big, 2)[1],
                          O.uniform_centered(out[:3]))


# --------------------------------------------------------------------------
# Potentials
# --------------------------------------------------------------------------
def test_lj_closed_forms():
    m = O.Model(1, {(0, 0): ("lj", 1.0, 1.0, 3.0, False)})
    rmin, tol = LIT["lj_min_r"]
    u, fr = O.pair_eval(m, 0, 0, rmin ** 2)
    assert abs(u - LIT["lj_min_u"][0]) < 1e-12
    assert abs(fr) < 1e-12
    u, fr = O.pair_eval(m, 0, 0, 1.0)
    assert abs(u) < 1e-15 and fr > 0  # U(sigma) = 0, repulsive inside the well
    u, fr = O.pair_eval(m, 0, 0, 2.5 ** 2)
    assert abs(u - LIT["lj_u_rc25"][0]) < LIT["lj_u_rc25"][1]
    # epsilon and sigma both enter: the minimum scales with sigma, depth with eps
    m2 = O.Model(1, {(0, 0): ("lj", 2.0, 1.5, 5.0, False)})
    u, fr = O.pair_eval(m2, 0, 0, (rmin * 1.5) ** 2)
    assert abs(u + 2.0) < 1e-12 and abs(fr) < 1e-12
    # beyond the cutoff nothing
    assert O.pair_eval(m, 0, 0, 3.0 ** 2) == (0.0, 0.0)


def test_shifted_lj_and_wca_vanish_at_cutoff():
    m = O.Model(1, {(0, 0): ("lj", 1.0, 1.0, 2.5, True)})
    u, fr = O.pair_eval(m, 0, 0, (2.5 - 1e-9) ** 2)
    assert abs(u) < 1e-9
    u0, _ = O.pair_eval(m, 0, 0, 1.0)
    assert abs(u0 - (-LIT["lj_u_rc25"][0])) < 1e-11  # U(sigma) = -U_raw(rc)
    w = O.Model(1, {(0, 0): ("wca", 1.0, 1.0)})
    rc = 2.0 ** (1.0 / 6.0)
    u, fr = O.pair_eval(w, 0, 0, (rc * (1 - 1e-9)) ** 2)
    assert abs(u) < 1e-12 and abs(fr) < 1e-6
    u, fr = O.pair_eval(w, 0, 0, 1.0)
    assert abs(u - 1.0) < 1e-14  # WCA U(sigma) = eps
    assert O.pair_eval(w, 0, 0, rc * rc) == (0.0, 0.0)  # strict r < rc


def test_capped_lj_holds_force_magnitude():
    cap = 0.8
    capped = O.Model(1, {(0, 0): ("lj_capped", 1.0, 1.0, 2.0 ** (1 / 6), True, cap)})
    plain = O.Model(1, {(0, 0): ("wca", 1.0, 1.0)})
    u_c, fr_c = O.pair_eval(plain, 0, 0, cap * cap)
    fmag = fr_c * cap
    for r in (0.05, 0.3, 0.79):
        u, fr = O.pair_eval(capped, 0, 0, r * r)
        assert abs(fr * r - fmag) < 1e-10 * fmag
        assert abs(u - (u_c + fmag * (cap - r))) < 1e-9 * fmag
    for r in (0.81, 1.0, 1.1):
        assert O.pair_eval(capped, 0, 0, r * r) == O.pair_eval(plain, 0, 0, r * r)


def test_fene_limits_and_kg_bond_minimum():
    # harmonic limit at small r: fr -> -K
    _, fr, _ = O.bond_eval(KG, 1e-8)
    assert abs(fr + 30.0) < 1e-6
    # energy diverges towards R0 and the bond breaks at r >= R0
    u1, _, _ = O.bond_eval(KG, 1.49 ** 2)
    u2, _, _ = O.bond_eval(KG, 1.4999 ** 2)
    assert u2 > u1 > 0
    assert O.bond_eval(KG, 1.5 ** 2)[2] == 1
    # the total bonded force (FENE + WCA) changes sign at the KG bond minimum
    def total(r):
        _, frb, _ = O.bond_eval(KG, r * r)
        _, frp = O.pair_eval(KG, 0, 0, r * r)
        return frb + frp
    lo, hi = 0.9, 1.05
    assert total(lo) > 0 > total(hi)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if total(mid) > 0:
            lo = mid
        else:
            hi = mid
    val, tol = LIT["kg_bond_min"]
    assert abs(lo - val) < tol


# --------------------------------------------------------------------------
# Forces: finite differences, Newton's third law, invariances
# --------------------------------------------------------------------------
def _total_energy(model, box, x, types, bonds):
    _, en = O.forces(model, box, x, types, bonds)
    return en[0] + en[1]


def _small_systems():
    out = []
    c = I.kg_lattice(4, 16, density=0.85, seed=3, jitter=0.15)
    out.append(("kg", KG, c))
    c = I.lj_fcc(2, 2, 2, density=0.8442)
    g = np.random.default_rng(5)
    c.x = np.mod(c.x + g.uniform(-0.2, 0.2, c.x.shape), c.box)
    out.append(("lj", O.Model(1, {(0, 0): ("lj", 1.0, 1.0, 2.5, True)}), c))
    c = I.lj_fcc(2, 2, 2, density=0.6)
    c.types = (np.arange(c.n) % 2).astype(np.int32)
    c.x = np.mod(c.x + g.uniform(-0.3, 0.3, c.x.shape), c.box)
    two = O.Model(2, {(0, 0): ("lj", 1.0, 1.0, 2.5, True), (0, 1): ("lj", 1.5, 0.9, 2.2, True),
                      (1, 1): ("wca", 0.7, 1.1)})
    out.append(("two-type", two, c))
    c = I.random_positions(40, (5.0, 5.0, 5.0), seed=9)
    out.append(("capped", O.Model(1, {(0, 0): ("lj_capped", 1.0, 1.0, 1.12246, True, 0.8)}), c))
    return out


@pytest.mark.parametrize("name,model,cfg", _small_systems(), ids=lambda v: v if isinstance(v, str) else "")
def test_forces_are_minus_energy_gradient(name, model, cfg):
    f, _ = O.forces(model, cfg.box, cfg.x, cfg.types, cfg.bonds)
    h = 1e-6
    rng = np.random.default_rng(1)
    idx = rng.choice(cfg.n, size=min(cfg.n, 12), replace=False)
    scale = np.abs(f).max()
    for i in idx:
        for c in range(3):
            xp = cfg.x.copy()
            xm = cfg.x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd = -(_total_energy(model, cfg.box, xp, cfg.types, cfg.bonds)
                   - _total_energy(model, cfg.box, xm, cfg.types, cfg.bonds)) / (2 * h)
            assert abs(fd - f[i, c]) < 2e-6 * max(1.0, scale), (name, i, c, fd, f[i, c])


@pytest.mark.parametrize("name,model,cfg", _small_systems(), ids=lambda v: v if isinstance(v, str) else "")
def test_newton_third_law(name, model, cfg):
    f, _ = O.forces(model, cfg.box, cfg.x, cfg.types, cfg.bonds)
    assert np.all(np.abs(f.sum(axis=0)) <= 1e-12 * np.abs(f).sum())


@pytest.mark.parametrize("name,model,cfg", _small_systems(), ids=lambda v: v if isinstance(v, str) else "")
def test_sampled_forces_equal_the_full_evaluation(name, model, cfg):
    # the full-size parity tests compare sampled particles with forces_subset:
    # it must give exactly the rows of the (pinned) full evaluation, also with
    # bonded exclusions and under a sheared boundary
    sel = np.random.default_rng(4).permutation(cfg.n)[: max(1, cfg.n // 3)]
    for excl, shear in ((False, 0.0), (True, 0.0), (False, 0.3)):
        O.set_exclude_bonded(excl)
        O.set_lees_edwards(shear != 0.0, shear)
        try:
            f, _ = O.forces(model, cfg.box, cfg.x, cfg.types, cfg.bonds, time=2.1)
            fs = O.forces_subset(model, cfg.box, cfg.x, cfg.types, cfg.bonds, sel, time=2.1)
        finally:
            O.set_exclude_bonded(False)
            O.set_lees_edwards(False)
        assert np.array_equal(fs, f[sel]), (name, excl, shear)


def test_translation_and_permutation_invariance():
    c = I.kg_lattice(10, 20, seed=4, jitter=0.1)
    f0, e0 = O.forces(KG, c.box, c.x, c.types, c.bonds)
    shift = np.array([3.3, -1.7, 0.45])
    xs = np.mod(c.x + shift, c.box)
    f1, e1 = O.forces(KG, c.box, xs, c.types, c.bonds)
    rel = np.sqrt(((f1 - f0) ** 2).sum() / (f0 ** 2).sum())
    assert rel < 1e-12
    assert np.allclose(e1, e0, rtol=1e-12)
    perm = np.random.default_rng(2).permutation(c.n)
    inv = np.argsort(perm)
    bonds = inv[c.bonds]
    f2, e2 = O.forces(KG, c.box, c.x[perm], c.types[perm], bonds)
    rel = np.sqrt(((f2[inv] - f0) ** 2).sum() / (f0 ** 2).sum())
    assert rel < 1e-14
    assert np.allclose(e2, e0, rtol=1e-13)


def test_two_particle_forces_by_hand():
    # two beads along x across the periodic boundary: distance 1.0 via the image
    box = np.array([10.0, 10.0, 10.0])
    x = np.array([[0.25, 5.0, 5.0], [9.25, 5.0, 5.0]])
    m = O.Model(1, {(0, 0): ("lj", 1.0, 1.0, 2.5, False)})
    f, en = O.forces(m, box, x, np.zeros(2, np.int32), np.zeros((0, 2), np.int64))
    # at r = sigma: U = 0, |F| = 24 eps / sigma, pushing particle 0 towards +x
    assert abs(en[0]) < 1e-14
    assert abs(f[0, 0] - 24.0) < 1e-12 and abs(f[1, 0] + 24.0) < 1e-12
    assert abs(en[2] - 24.0) < 1e-12  # virial r.F = 1 * 24


# --------------------------------------------------------------------------
# Neighbour sets
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["random", "lj", "kg", "dense"])
def test_cell_neighbours_equal_brute_force(kind):
    if kind == "random":
        c = I.random_positions(500, (9.0, 7.5, 11.0), seed=1)
        rcut = 2.3
    elif kind == "lj":
        c = I.lj_fcc(4, 4, 3)
        c.x = np.mod(c.x + np.random.default_rng(0).normal(0, 0.1, c.x.shape), c.box)
        rcut = 2.8
    elif kind == "kg":
        c = I.kg_lattice(20, 50, seed=2, jitter=0.2)
        rcut = 2.0 ** (1 / 6) + 0.4
    else:
        c = I.random_positions(1200, (8.0, 8.0, 8.0), seed=3)
        rcut = 1.5
    rb, cb = O.neighbors(c.box, c.x, rcut, method="brute")
    rc_, cc = O.neighbors(c.box, c.x, rcut, method="cells")
    assert np.array_equal(rb, rc_) and np.array_equal(cb, cc)
    assert cb.size > 0


def test_neighbour_count_matches_ideal_gas_estimate():
    # uniform random points: mean neighbour count -> rho * 4/3 pi r^3
    c = I.random_positions(4000, (15.0, 15.0, 15.0), seed=11)
    row, cols = O.neighbors(c.box, c.x, 1.5)
    rho = c.n / np.prod(c.box)
    expect = rho * 4.0 / 3.0 * math.pi * 1.5 ** 3
    assert abs(cols.size / c.n - expect) < 0.05 * expect


# --------------------------------------------------------------------------
# Integrator
# --------------------------------------------------------------------------
FREE = O.Model(1, {})


def _free_variance_closed_form(nsteps, dt, gamma, kT, m=1.0):
    """Exact variance of one full-step velocity component of a free particle
    under the scheme (friction on the velocity present at the force step,
    noise variance 2 gamma m kT / dt), starting from v = 0."""
    S = 2.0 * gamma * m * kT / dt            # noise force variance
    vh = (dt / (2 * m)) ** 2 * S             # var v(1/2)
    var_full = []
    for s in range(1, nsteps + 1):
        var_full.append((1 - gamma * dt / 2) ** 2 * vh + (dt / (2 * m)) ** 2 * S)
        vh = (1 - gamma * dt) ** 2 * vh + (dt / m) ** 2 * S
    return np.array(var_full)


@pytest.mark.parametrize("gamma,dt,m", [(10.0, 0.05, 1.0), (1.0, 0.005, 1.0), (10.0, 0.05, 2.5)])
def test_free_particle_langevin_closed_form(gamma, dt, m):
    n = 200000
    kT = 1.7
    nsteps = 12 if gamma * dt > 0.1 else 3
    st = O.State(np.array([50.0, 50.0, 50.0]), np.full((n, 3), 25.0))
    model = O.Model(1, {}, masses=[m])
    expect = _free_variance_closed_form(nsteps, dt, gamma, kT, m)
    got = []
    for s in range(nsteps):
        O.integrate(model, st, 1, dt, gamma, kT, seed=123)
        got.append((st.v ** 2).mean())
    got = np.array(got)
    # sample variance of 3n draws; the uniform noise has kurtosis < 3 so the
    # Gaussian error bar sqrt(2/3n) is conservative
    err = expect * np.sqrt(2.0 / (3 * n))
    assert np.all(np.abs(got - expect) < 5 * err), (got, expect)
    if gamma * dt > 0.1:
        # equilibrium: full-step velocities carry exactly kT/m
        assert abs(expect[-1] - kT / m) < 1e-6 * kT / m
    assert abs(st.v.mean()) < 5 * np.sqrt(expect[-1] / (3 * n))


def test_reversibility_without_thermostat():
    c = I.kg_lattice(5, 20, seed=8, jitter=0.05)
    st = O.State(c.box, c.x, I.maxwell_velocities(c.n, 1.0, seed=3), c.img, c.types, c.bonds)
    x0 = st.x + st.img * st.box
    O.integrate(KG, st, 200, 0.005, 0.0, 0.0, seed=1)
    st.v = -st.v
    st.f_valid = False
    O.integrate(KG, st, 200, 0.005, 0.0, 0.0, seed=1)
    x1 = st.x + st.img * st.box
    assert np.abs(x1 - x0).max() < 1e-8


def _kg_equilibrated(nsteps=2000, seed=42):
    c = I.kg_lattice(20, 50, seed=seed, jitter=0.05)
    st = O.State(c.box, c.x, I.maxwell_velocities(c.n, 1.0, seed=seed), c.img, c.types, c.bonds)
    O.integrate(KG, st, nsteps, 0.005, 1.0, 1.0, seed=seed)
    return st


def test_nve_energy_drift():
    st = _kg_equilibrated(1000)
    st.f_valid = False
    O.integrate(KG, st, 0, 0.005, 0.0, 0.0, seed=0)
    es = []
    for _ in range(40):
        o = O.observables(KG, st)
        es.append(o["ke"] + o["pe_pair"] + o["pe_bond"])
        O.integrate(KG, st, 100, 0.005, 0.0, 0.0, seed=0)
    es = np.array(es) / st.n
    assert np.abs(es - es[0]).max() < 1e-3
    # no secular trend beyond the fluctuation level
    slope = np.polyfit(np.arange(es.size), es, 1)[0] * es.size
    assert abs(slope) < 1e-3


@pytest.mark.slow
def test_equipartition_and_kg_bond_length():
    st = _kg_equilibrated(2000)
    temps, bonds = [], []
    for _ in range(50):
        O.integrate(KG, st, 40, 0.005, 1.0, 1.0, seed=42)
        o = O.observables(KG, st)
        temps.append(o["temperature"])
        bonds.append(o["mean_bond"])
    temps = np.array(temps)
    # 50 samples of T with per-sample std ~ sqrt(2/(3N)) = 0.026
    assert abs(temps.mean() - 1.0) < 0.02
    val, tol = LIT["kg_mean_bond"]
    assert abs(np.mean(bonds) - val) < tol


# --------------------------------------------------------------------------
# Observables
# --------------------------------------------------------------------------
def test_observables_closed_forms():
    # a straight rod of 8 beads, spacing 1.0, wrapped across the boundary:
    # Rg^2 = b^2 (n^2 - 1) / 12
    box = np.array([6.0, 6.0, 6.0])
    u = np.stack([np.arange(8) * 1.0 + 2.5, np.full(8, 3.0), np.full(8, 3.0)], axis=1)
    img = np.floor(u / box).astype(np.int32)
    x = u - img * box
    bonds = np.stack([np.arange(7), np.arange(1, 8)], axis=1)
    v = np.zeros((8, 3))
    v[:, 0] = 2.0
    st = O.State(box, x, v, img, None, bonds)
    o = O.observables(O.Model(1, {}, ("fene", 30.0, 1.5)), st)
    assert abs(o["rg2"] - (64 - 1) / 12.0) < 1e-12
    assert abs(o["mean_bond"] - 1.0) < 1e-12
    assert abs(o["ke"] - 8 * 0.5 * 4.0) < 1e-12
    assert abs(o["px"] - 16.0) < 1e-12 and o["nmol"] == 1.0
    # ideal gas pressure P = N kT / V with T from the kinetic energy
    c = I.random_positions(1000, (10.0, 10.0, 10.0), seed=1)
    vel = I.maxwell_velocities(1000, 1.3, seed=2)
    o = O.observables(FREE, O.State(c.box, c.x, vel))
    assert abs(o["pressure"] - 1000 * o["temperature"] / 1000.0) < 1e-12
    assert abs(o["temperature"] - 1.3) < 1e-6


def test_rdf_counts_small():
    box = np.array([10.0, 10.0, 10.0])
    x = np.array([[1.0, 1.0, 1.0], [1.5, 1.0, 1.0], [1.0, 2.2, 1.0], [9.7, 1.0, 1.0]])
    c = O.rdf_counts(box, x, 2.0, 20)
    # unique distances: 0.5, 1.2, 1.3 (via image), 1.3 (0-3 is 1.3), ...
    d = []
    for i in range(4):
        for j in range(i + 1, 4):
            dd = x[i] - x[j]
            dd -= box * np.round(dd / box)
            d.append(np.linalg.norm(dd))
    expect = np.histogram([r for r in d if r < 2.0], bins=20, range=(0, 2.0))[0]
    assert np.array_equal(c, expect)


# --------------------------------------------------------------------------
# Tabulated potentials
# --------------------------------------------------------------------------
def test_linear_table_is_interpolated_exactly():
    # u and F linear in r: linear interpolation reproduces them everywhere
    rc, n = 3.0, 31
    r = np.linspace(0.0, rc, n)
    O.set_table(0, rc, 2.0 - 0.5 * r, 3.0 + 0.25 * r)
    m = O.Model(1, {(0, 0): ("table", 0, rc)})
    for rr in (0.013, 0.77, 1.2345, 2.999):
        u, fr = O.pair_eval(m, 0, 0, rr * rr)
        assert abs(u - (2.0 - 0.5 * rr)) < 1e-13
        assert abs(fr * rr - (3.0 + 0.25 * rr)) < 1e-12
    assert O.pair_eval(m, 0, 0, rc * rc) == (0.0, 0.0)


def test_lj_table_within_interpolation_bound():
    # a table sampled from 12-6 LJ: |F_table - F| <= h^2/8 max|F''| between nodes
    rc, n = 2.5, 4096
    r = np.linspace(0.0, rc, n)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.where(r > 0.5, 4 * (r ** -12 - r ** -6), 0.0)
        f = np.where(r > 0.5, 24 * (2 * r ** -13 - r ** -7), 0.0)
    O.set_table(1, rc, u, f)
    tab = O.Model(1, {(0, 0): ("table", 1, rc)})
    lj = O.Model(1, {(0, 0): ("lj", 1.0, 1.0, rc, False)})
    h = rc / (n - 1)
    for rr in np.linspace(0.9, 2.49, 37):
        _, fr_t = O.pair_eval(tab, 0, 0, rr * rr)
        _, fr_a = O.pair_eval(lj, 0, 0, rr * rr)
        # F'' of LJ is bounded by 24*(2*13*14 r^-15) near r = 0.9
        bound = h * h / 8 * 24 * 2 * 13 * 14 * 0.9 ** -15
        assert abs(fr_t * rr - fr_a * rr) <= bound


def test_table_bond_breaks_beyond_range():
    rmax, n = 1.5, 301
    r = np.linspace(0.0, rmax, n)
    O.set_table(2, rmax, 15.0 * r * r, -30.0 * r)
    m = O.Model(1, {}, ("table", 2))
    u, fr, st = O.bond_eval(m, 0.49)
    assert st == 0 and abs(fr + 30.0) < 1e-12 and abs(u - 15.0 * 0.49) < 1e-3
    assert O.bond_eval(m, 1.5 ** 2)[2] == 1


# --------------------------------------------------------------------------
# Learned MLP pair potential
# --------------------------------------------------------------------------
def _mlp_params(seed=0, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, O.MLP_NPARAMS)


def test_mlp_force_is_minus_energy_derivative():
    O.set_mlp(_mlp_params(1), 3.5)
    h = 1e-6
    for r in (0.4, 0.97, 1.5, 2.2, 3.1, 3.45):
        u, du = O.mlp_pair(r)
        fd = (O.mlp_pair(r + h)[0] - O.mlp_pair(r - h)[0]) / (2 * h)
        assert abs(du - fd) < 1e-7 * max(1.0, abs(du))


def test_mlp_parameter_gradients_by_finite_differences():
    p = _mlp_params(2)
    O.set_mlp(p, 3.5)
    r = 1.37
    _, _, g_du, g_u = O.mlp_pair(r, want_grad=True)
    rng = np.random.default_rng(3)
    # W1, b1, W2, b2, w3 and b3 blocks
    blocks = [(0, 2048), (2048, 2112), (2112, 6208), (6208, 6272), (6272, 6336), (6336, 6337)]
    h = 1e-6
    for lo, hi in blocks:
        for k in rng.choice(np.arange(lo, hi), size=min(6, hi - lo), replace=False):
            q = p.copy()
            q[k] += h
            O.set_mlp(q, 3.5)
            up, dp = O.mlp_pair(r)
            q[k] -= 2 * h
            O.set_mlp(q, 3.5)
            um, dm = O.mlp_pair(r)
            assert abs(g_du[k] - (dp - dm) / (2 * h)) < 1e-6 * max(1.0, abs(g_du[k])), k
            assert abs(g_u[k] - (up - um) / (2 * h)) < 1e-6 * max(1.0, abs(g_u[k])), k
    O.set_mlp(p, 3.5)


def test_mlp_envelope_vanishes_at_cutoff():
    p = _mlp_params(4)
    O.set_mlp(p, 3.5)
    # phi and dphi/dr vanish at rc, so u tends to the zero-input value and du/dr to 0
    u_rc, du_rc = O.mlp_pair(3.5 - 1e-7)
    assert abs(du_rc) < 1e-6
    W1 = p[:2048].reshape(64, 32)
    b1, W2 = p[2048:2112], p[2112:6208].reshape(64, 64)
    b2, w3, b3 = p[6208:6272], p[6272:6336], p[6336]
    silu = lambda z: z / (1 + np.exp(-z))
    u0 = w3 @ silu(W2 @ silu(b1) + b2) + b3
    assert abs(u_rc - u0) < 1e-9
    # zero hidden weights: u is the constant w3 . silu(b2) + b3
    q = p.copy()
    q[2112:6208] = 0.0
    O.set_mlp(q, 3.5)
    u, du = O.mlp_pair(1.0)
    assert abs(u - (w3 @ silu(b2) + b3)) < 1e-12 and abs(du) < 1e-15
    O.set_mlp(p, 3.5)


def test_mlp_radial_basis_centres_and_width():
    # du/dW1[a, k] = (adjoint of unit a) * phi_k(r), so the ratio of two
    # neighbouring entries is phi_{k+1}(r) / phi_k(r): the envelope cancels,
    # and for Gaussians of width w centred a spacing D apart its logarithm is
    # the straight line (2 r - (2k + 1) D) D / (2 w^2).  The reading's 32
    # bases on [0, rc] put D = w = rc / 31: slope 1/w, zero midway between
    # the centres.
    rc = 3.5
    O.set_mlp(_mlp_params(6), rc)
    D = w = rc / 31
    for r in np.linspace(0.05, rc - 0.05, 29):
        g_u = O.mlp_pair(r, want_grad=True)[3]
        row = g_u[:2048].reshape(64, 32)
        a = int(np.argmax(np.abs(row).max(axis=1)))
        for k in range(max(0, int(r / D) - 2), min(31, int(r / D) + 3)):
            got = np.log(row[a, k + 1] / row[a, k])
            want = (2 * r - (2 * k + 1) * D) * D / (2 * w * w)
            assert abs(got - want) < 1e-9, (r, k, got, want)


def test_bonded_exclusion_removes_exactly_the_bonded_pairs():
    c = I.kg_lattice(5, 20, seed=6, jitter=0.1)
    m = O.Model(1, {(0, 0): ("lj", 1.0, 1.0, 2.5, True)})
    f_all, _ = O.forces(m, c.box, c.x, c.types, np.zeros((0, 2), np.int64))
    O.set_exclude_bonded(True)
    try:
        f_ex, _ = O.forces(O.Model(1, {(0, 0): ("lj", 1.0, 1.0, 2.5, True)}, None), c.box, c.x, c.types, c.bonds)
    finally:
        O.set_exclude_bonded(False)
    # add back the bonded pair forces by hand: F_i += fr d over bonded partners
    f_back = f_ex.copy()
    for a, b in c.bonds:
        d = c.x[a] - c.x[b]
        d -= c.box * np.round(d / c.box)
        _, fr = O.pair_eval(m, 0, 0, float(d @ d))
        f_back[a] += fr * d
        f_back[b] -= fr * d
    assert np.abs(f_back - f_all).max() < 1e-10 * np.abs(f_all).max()


def test_force_matching_gradient_by_finite_differences():
    # the loss gradient equals central differences of the loss itself
    c = I.kg_lattice(4, 25, density=0.2125, seed=12, jitter=0.3)
    g = np.random.default_rng(13)
    X = np.stack([np.mod(c.x + g.normal(0, 0.2, c.x.shape), c.box) for _ in range(2)])
    Y = g.normal(0, 1.0, X.shape)
    p = _mlp_params(7, 0.2)
    O.set_mlp(p, 3.5)
    rb = np.linspace(0.0, 4.0, 401)
    O.set_table(9, 4.0, 5.0 * (rb - 2.0) ** 2, -10.0 * (rb - 2.0))
    model = O.Model(1, {}, ("table", 9))
    O.set_exclude_bonded(True)
    try:
        loss, grad = O.mlp_loss_grad(model, c.box, X, Y, c.types, c.bonds)
        h = 1e-6
        for k in (5, 2050, 3000, 6210, 6300):
            q = p.copy()
            q[k] += h
            O.set_mlp(q, 3.5)
            lp, _ = O.mlp_loss_grad(model, c.box, X, Y, c.types, c.bonds)
            q[k] -= 2 * h
            O.set_mlp(q, 3.5)
            lm, _ = O.mlp_loss_grad(model, c.box, X, Y, c.types, c.bonds)
            fd = (lp - lm) / (2 * h)
            assert abs(grad[k] - fd) < 1e-6 * max(1.0, abs(fd)), (k, grad[k], fd)
    finally:
        O.set_exclude_bonded(False)
        O.set_mlp(p, 3.5)


def test_wrap_just_below_zero_keeps_the_unwrapped_position():
    # a free particle drifting from x = 1e-20 to x = -2e-18: x + L rounds to L
    # in double, so the wrap must leave it at 0 in its own image (the
    # unwrapped coordinate x + img L stays -2e-18, not -L); the same at the
    # upper face for comparison
    free = O.Model(1, {})
    L = 10.0
    for x0, v0 in ((1e-20, -4e-16), (L - 1e-6, 4e-4)):
        st = O.State([L, L, L], [[x0, 5.0, 5.0]], [[v0, 0.0, 0.0]])
        O.integrate(free, st, 1, 0.005, 0.0, 0.0, seed=1)
        unwrapped = st.x[0, 0] + st.img[0, 0] * L
        assert 0.0 <= st.x[0, 0] < L
        assert abs(unwrapped - (x0 + 0.005 * v0)) < 1e-12, (st.x[0, 0], st.img[0, 0])


def _loss_by_hand(X, Y, box, bonds, rc, rb_max, ub, fb, variant="right"):
    """Force-matching loss recomputed outside the oracle's loss routine: pair
    forces F_i = sum_j -u'(r_ij) (x_i - x_j)/r_ij over unordered pairs
    (bonded 1-2 pairs excluded) from the per-pair derivative alone, bond
    forces from a linear interpolation of the bond table, then
    loss = sum_f sum_i |F_i - Y_fi|^2 / (frames x sites).  `variant` plants
    one of three plausible mistakes, to show that the pin would see it."""
    nf, n, _ = X.shape
    bset = {(min(a, b), max(a, b)) for a, b in bonds}
    total = 0.0
    for f in range(nf):
        x = X[f]
        F = np.zeros((n, 3))
        for i in range(n):
            d = x[i] - x[i + 1:]
            d -= box * np.round(d / box)
            r = np.sqrt((d * d).sum(axis=1))
            for k in np.nonzero(r < rc)[0]:
                j = i + 1 + k
                if (i, j) in bset:
                    continue
                _, du = O.mlp_pair(float(r[k]))
                fij = -du * d[k] / r[k]
                F[i] += fij
                F[j] -= fij
                if variant == "pairs_twice":
                    F[i] += fij
                    F[j] -= fij
        Fb = np.zeros((n, 3))
        for a, b in bonds:
            d = x[a] - x[b]
            d -= box * np.round(d / box)
            r = float(np.sqrt(d @ d))
            fr = np.interp(r, np.linspace(0.0, rb_max, fb.size), fb)
            Fb[a] += fr * d / r
            Fb[b] -= fr * d / r
        e = (F - Fb if variant == "bond_sign" else F + Fb) - Y[f]
        total += (e * e).sum()
    return total / (nf if variant == "frames_only" else nf * n)


def test_force_matching_loss_value_recomputed_by_hand():
    # the loss value itself (not only its gradient) against an independent
    # evaluation from per-pair derivatives and the bond table
    c = I.kg_lattice(4, 25, density=0.2125, seed=12, jitter=0.3)
    g = np.random.default_rng(14)
    X = np.stack([np.mod(c.x + g.normal(0, 0.2, c.x.shape), c.box) for _ in range(2)])
    Y = g.normal(0, 1.0, X.shape)
    p = _mlp_params(8, 0.2)
    O.set_mlp(p, 3.5)
    rb = np.linspace(0.0, 4.0, 401)
    ub, fb = 5.0 * (rb - 2.0) ** 2, -10.0 * (rb - 2.0)
    O.set_table(9, 4.0, ub, fb)
    model = O.Model(1, {}, ("table", 9))
    O.set_exclude_bonded(True)
    try:
        loss, _ = O.mlp_loss_grad(model, c.box, X, Y, c.types, c.bonds)
    finally:
        O.set_exclude_bonded(False)
    want = _loss_by_hand(X, Y, c.box, c.bonds, 3.5, 4.0, ub, fb)
    assert abs(loss - want) < 1e-10 * abs(want), (loss, want)
    # each planted mistake moves the value far outside that tolerance
    for variant in ("frames_only", "bond_sign", "pairs_twice"):
        wrong = _loss_by_hand(X, Y, c.box, c.bonds, 3.5, 4.0, ub, fb, variant)
        assert abs(wrong - want) > 1e-3 * abs(want), variant


# --------------------------------------------------------------------------
# DPD thermostat (paper "Functionality": dissipative particle dynamics)
# --------------------------------------------------------------------------
@pytest.fixture
def dpd_on():
    def on(rc):
        O.set_dpd(True, rc)
    yield on
    O.set_dpd(False)


LJ_FLUID = O.Model(1, {(0, 0): ("lj", 1.0, 1.0, 2.5, True)})


def _unwrapped(st):
    return st.x + st.img * st.box


def _ideal_dpd_gas(n, density, seed):
    side = (n / density) ** (1.0 / 3.0)
    c = I.random_positions(n, np.array([side] * 3), seed=seed)
    v = I.maxwell_velocities(n, 1.0, seed=seed)
    v -= v.mean(axis=0)
    return O.State(c.box, c.x, v)


def test_dpd_theta_keying_and_moments():
    # symmetric in the pair, keyed by step and seed, word 0 of the Philox
    # block with counter (min id, max id | 2^31, step lo, step hi)
    assert O.dpd_theta(7, 3, 11, 5) == O.dpd_theta(7, 11, 3, 5)
    assert O.dpd_theta(7, 3, 11, 5) != O.dpd_theta(7, 3, 11, 6)
    assert O.dpd_theta(7, 3, 11, 5) != O.dpd_theta(8, 3, 11, 5)
    step = (1 << 33) + 9
    out = O.philox([3, 11 | 0x80000000, step & 0xffffffff, step >> 32], [7, 0])
    assert O.dpd_theta(7, 11, 3, step) == math.sqrt(12.0) * O.uniform_centered(out[:1])[0]
    # the pair counter never meets the per-particle one (bit 31 of word 1)
    assert (11 | 0x80000000) != 11
    g = I.rng(3, 0)
    a = g.integers(0, 1 << 20, 20000)
    b = g.integers(0, 1 << 20, 20000)
    th = np.array([O.dpd_theta(99, int(x), int(y), 17) for x, y in zip(a, b)])
    # zero mean, unit variance (uniform: 4th moment 9/5)
    assert abs(th.mean()) < 5 / math.sqrt(th.size)
    assert abs(th.var() - 1.0) < 5 * math.sqrt(0.8 / th.size)
    assert np.abs(th).max() < math.sqrt(3.0)


def test_dpd_two_particles_closed_form(dpd_on):
    # kT = 0, no conservative force: the relative velocity along the pair axis
    # decays as exp(-2 gamma w^2 t) (reduced mass 1/2), the perpendicular
    # component is untouched, the centre of mass moves uniformly
    dpd_on(1.0)
    gamma, r0, dt, nsteps = 4.5, 0.5, 1e-3, 100
    x = np.array([[5.0, 5.0, 5.0], [5.0 + r0, 5.0, 5.0]])
    # equal perpendicular velocities keep the pair axis along x
    v = np.array([[0.3 + 5e-4, 0.2, -0.1], [0.3 - 5e-4, 0.2, -0.1]])
    st = O.State(np.array([10.0, 10.0, 10.0]), x, v)
    O.integrate(FREE, st, nsteps, dt, gamma, 0.0, seed=1)
    w = 1.0 - r0 / 1.0
    u = st.v[0, 0] - st.v[1, 0]
    assert abs(u / 1e-3 - math.exp(-2 * gamma * w * w * nsteps * dt)) < 2e-3
    assert np.array_equal(st.v[:, 1:], v[:, 1:])
    assert abs(st.v[:, 0].sum() - v[:, 0].sum()) < 1e-15
    # beyond the cutoff nothing acts
    v = np.array([[0.3, 0.2, -0.1], [-0.3, -0.4, 0.7]])
    st = O.State(np.array([10.0, 10.0, 10.0]), np.array([[5.0, 5.0, 5.0], [7.2, 5.0, 5.0]]), v)
    O.integrate(FREE, st, 20, dt, gamma, 1.0, seed=1)
    assert np.array_equal(st.v, v)


def test_dpd_conserves_momentum(dpd_on):
    dpd_on(1.0)
    c = I.lj_fcc(5, 5, 5, density=0.8442)
    v = I.maxwell_velocities(c.n, 1.5, seed=4) + np.array([0.02, -0.01, 0.005])
    st = O.State(c.box, c.x, v)
    p0 = st.v.sum(axis=0)
    assert np.abs(p0).max() > 1.0  # a non-trivial total momentum to keep
    O.integrate(LJ_FLUID, st, 200, 0.005, 4.5, 1.0, seed=4)
    assert np.abs(st.v.sum(axis=0) - p0).max() < 1e-10
    # with Langevin the same run loses it to the solvent
    O.set_dpd(False)
    st = O.State(c.box, c.x, v)
    O.integrate(LJ_FLUID, st, 200, 0.005, 4.5, 1.0, seed=4)
    assert np.abs(st.v.sum(axis=0) - p0).max() > 1.0


def test_dpd_galilean_invariance(dpd_on):
    # only relative velocities enter: a uniform boost u is carried along exactly
    dpd_on(1.0)
    c = I.lj_fcc(4, 4, 4, density=0.8442)
    v = I.maxwell_velocities(c.n, 1.0, seed=6)
    u = np.array([0.7, -1.3, 0.25])
    a = O.State(c.box, c.x, v)
    b = O.State(c.box, c.x, v + u)
    nsteps, dt = 100, 0.005
    O.integrate(LJ_FLUID, a, nsteps, dt, 4.5, 1.0, seed=9)
    O.integrate(LJ_FLUID, b, nsteps, dt, 4.5, 1.0, seed=9)
    assert np.abs(b.v - a.v - u).max() < 1e-9
    assert np.abs(_unwrapped(b) - _unwrapped(a) - u * nsteps * dt).max() < 1e-9


def test_dpd_dissipates_without_noise(dpd_on):
    dpd_on(1.0)
    st = _ideal_dpd_gas(400, 3.0, seed=2)
    ke = [0.5 * (st.v ** 2).sum()]
    for _ in range(30):
        O.integrate(FREE, st, 1, 0.01, 4.5, 0.0, seed=2)
        ke.append(0.5 * (st.v ** 2).sum())
    ke = np.array(ke)
    assert np.all(np.diff(ke) < 0)
    assert ke[-1] < 0.5 * ke[0]
    assert np.abs(st.v.sum(axis=0)).max() < 1e-10


def test_dpd_equipartition(dpd_on):
    # fluctuation-dissipation: an ideal DPD gas (density 3, rc 1, gamma 4.5)
    # settles at the bath temperature
    dpd_on(1.0)
    kT = 1.0
    st = _ideal_dpd_gas(648, 3.0, seed=11)
    st.v *= math.sqrt(0.3)  # start cold
    O.integrate(FREE, st, 300, 0.01, 4.5, kT, seed=11)
    t = []
    for _ in range(60):
        O.integrate(FREE, st, 10, 0.01, 4.5, kT, seed=11)
        t.append((st.v ** 2).sum() / (3 * (st.n - 1)))
    assert abs(np.mean(t) - kT) < 0.03 * kT, np.mean(t)


# --------------------------------------------------------------------------
# Lees-Edwards boundary conditions (paper "State of the field" and "New
# features"): flow along x, gradient along z, offset delta = gdot Lz t
# --------------------------------------------------------------------------
@pytest.fixture
def le_on():
    def on(shear):
        O.set_lees_edwards(True, shear)
    yield on
    O.set_lees_edwards(False)
    O.set_dpd(False)


def _le_images(box, delta, xi, xj, na=3):
    """Displacements x_i - image(x_j) over the explicit sheared images."""
    delta = delta % box[0]  # the same set of images, a few boxes to enumerate
    out = []
    for b in (-1, 0, 1):
        for a in range(-na, na + 1):
            for c in (-1, 0, 1):
                img = np.array([a * box[0] + b * delta, c * box[1], b * box[2]])
                out.append(xi - (xj + img))
    return np.array(out)


def test_le_neighbours_match_image_enumeration(le_on):
    box = np.array([8.0, 9.0, 10.0])
    shear, t = 0.37, 5.3
    delta = shear * box[2] * t  # several box lengths along x
    le_on(shear)
    c = I.random_positions(500, box, seed=12)
    rcut = 1.5
    row, cols = O.neighbors(box, c.x, rcut, time=t)
    got = set()
    for i in range(c.n):
        for j in cols[row[i]:row[i + 1]]:
            got.add((i, int(j)))
    want = set()
    for i in range(c.n):
        d = c.x[i] - c.x  # (n, 3) plain differences
        best = np.full(c.n, np.inf)
        for b in (-1, 0, 1):
            for a in range(-4, 5):
                for cc in (-1, 0, 1):
                    img = np.array([a * box[0] + b * delta, cc * box[1], b * box[2]])
                    best = np.minimum(best, ((d - img) ** 2).sum(axis=1))
        for j in np.nonzero(best < rcut * rcut)[0]:
            if j != i:
                want.add((i, int(j)))
    assert got == want and len(want) > 500
    # with the shear off the same positions give the plain periodic sets
    O.set_lees_edwards(False)
    row0, cols0 = O.neighbors(box, c.x, rcut)
    assert {(i, int(j)) for i in range(c.n) for j in cols0[row0[i]:row0[i + 1]]} != want


def test_le_ballistic_motion(le_on):
    # no forces, no thermostat: seen from the image frame a particle came
    # from, its velocity never changes (each crossing of a sheared face takes
    # gdot Lz off v_x per box), and the unwrapped position
    # x + img_x Lx + img_z delta(t) moves on a straight line
    shear, dt, nsteps = 0.5, 0.01, 1500
    le_on(shear)
    box = np.array([6.0, 6.0, 6.0])
    c = I.random_positions(300, box, seed=3)
    v = I.maxwell_velocities(300, 1.0, seed=3)
    st = O.State(box, c.x, v)

    def frame_velocity(s):
        p = s.v.copy()
        p[:, 0] += s.img[:, 2] * shear * box[2]
        return p

    def unwrapped(s):
        u = s.x + s.img * box
        u[:, 0] += s.img[:, 2] * shear * box[2] * s.time
        return u

    u0 = unwrapped(st)
    O.integrate(FREE, st, nsteps, dt, 0.0, 0.0, seed=1)
    assert abs(st.time - nsteps * dt) < 1e-12
    assert np.abs(st.img[:, 2]).max() >= 2  # particles crossed the sheared faces
    assert np.abs(frame_velocity(st) - v).max() < 1e-11
    assert np.array_equal(st.v[:, 1:], v[:, 1:])
    # each particle moves with its initial velocity seen from its own image frame
    assert np.abs(unwrapped(st) - (u0 + v * nsteps * dt)).max() < 1e-9


def _dpd_shear_run(shear, nsteps, seed=5, box=(5.0, 5.0, 6.0), gamma=4.5):
    box = np.array(box)
    n = int(3.0 * box.prod())
    c = I.random_positions(n, box, seed=seed)
    v = I.maxwell_velocities(n, 1.0, seed=seed)
    v[:, 0] += shear * (c.x[:, 2] - box[2] / 2)  # start on the linear profile
    st = O.State(box, c.x, v)
    O.set_dpd(True, 1.0)
    prof, pxz, temp = [], [], []
    for _ in range(nsteps // 20):
        O.integrate(FREE, st, 20, 0.01, gamma, 1.0, seed=seed)
        o = O.observables(FREE, st)
        pxz.append(o["pxz"])
        temp.append(o["temperature"])
        prof.append(np.polyfit(st.x[:, 2] - box[2] / 2, st.v[:, 0], 1)[0])
    return np.array(prof), np.array(pxz), np.array(temp)


def test_le_dpd_keeps_the_linear_profile(le_on):
    # a DPD fluid sheared through the boundaries keeps the imposed linear
    # velocity profile, stays at the bath temperature (relative to the
    # profile) and carries a negative xz pressure (momentum flows down the
    # gradient)
    shear = 0.5
    le_on(shear)
    prof, pxz, temp = _dpd_shear_run(shear, 2000)
    assert abs(prof[len(prof) // 2:].mean() - shear) < 0.1 * shear, prof
    assert abs(temp[len(temp) // 2:].mean() - 1.0) < 0.05, temp.mean()
    assert pxz.mean() < -3 * pxz.std() / math.sqrt(pxz.size), (pxz.mean(), pxz.std())
    # without the sheared boundary the same start relaxes the profile away
    O.set_lees_edwards(False)
    prof0, _, _ = _dpd_shear_run(shear, 2000)
    assert prof0[-10:].mean() < 0.5 * shear


def test_le_langevin_relative_to_profile(le_on):
    # an ideal gas under the profile-biased Langevin thermostat follows the
    # streaming profile, with the bath temperature relative to it
    shear = 0.5
    le_on(shear)
    box = np.array([6.0, 6.0, 6.0])
    c = I.random_positions(2000, box, seed=8)
    st = O.State(box, c.x, I.maxwell_velocities(2000, 1.0, seed=8))
    O.integrate(FREE, st, 600, 0.01, 2.0, 1.0, seed=8)
    slopes, temps = [], []
    for _ in range(20):
        O.integrate(FREE, st, 10, 0.01, 2.0, 1.0, seed=8)
        slopes.append(np.polyfit(st.x[:, 2] - box[2] / 2, st.v[:, 0], 1)[0])
        temps.append(O.observables(FREE, st)["temperature"])
    assert abs(np.mean(slopes) - shear) < 0.1 * shear
    assert abs(np.mean(temps) - 1.0) < 0.03


def test_le_rg2_of_a_chain_across_the_sheared_face(le_on):
    # radius of gyration from the unwrapped positions equals the one built by
    # walking the bonds with the sheared minimum image
    shear = 0.8
    le_on(shear)
    c = I.kg_lattice(6, 30, seed=4, jitter=0.05)
    st = O.State(c.box, c.x, I.maxwell_velocities(c.n, 1.0, seed=4), c.img, c.types, c.bonds)
    O.integrate(KG, st, 3000, 0.005, 1.0, 1.0, seed=4)
    assert np.abs(st.img[:, 2]).max() >= 1
    delta = shear * c.box[2] * st.time
    rg = []
    for m in range(6):
        ids = np.arange(30 * m, 30 * m + 30)
        pos = [st.x[ids[0]]]
        for a, b in zip(ids[:-1], ids[1:]):
            d = _le_images(c.box, delta, st.x[b], st.x[a])
            pos.append(pos[-1] + d[np.argmin((d ** 2).sum(axis=1))])
        pos = np.array(pos)
        rg.append(((pos - pos.mean(axis=0)) ** 2).sum(axis=1).mean())
    o = O.observables(KG, st)
    assert abs(o["rg2"] - np.mean(rg)) < 1e-9 * np.mean(rg)


def test_dpd_skips_excluded_bonded_pairs(dpd_on):
    # with 1-2 exclusions on (the learned CG model) a bonded pair gets no DPD
    # force: a lone FENE dimer moves exactly as without the thermostat
    dpd_on(1.2)
    box = np.array([10.0, 10.0, 10.0])
    x = np.array([[5.0, 5.0, 5.0], [5.9, 5.2, 5.1]])
    v = np.array([[0.4, -0.3, 0.1], [-0.2, 0.5, 0.3]])
    bonds = np.array([[0, 1]])
    fene = O.Model(1, {}, ("fene", 30.0, 1.5))
    runs = {}
    try:
        for excl, gamma in ((True, 4.5), (True, 0.0), (False, 4.5)):
            O.set_exclude_bonded(excl)
            st = O.State(box, x, v, None, None, bonds)
            O.integrate(fene, st, 50, 0.005, gamma, 0.0, seed=3)
            runs[(excl, gamma)] = st.v.copy()
    finally:
        O.set_exclude_bonded(False)
    assert np.array_equal(runs[(True, 4.5)], runs[(True, 0.0)])
    assert np.abs(runs[(False, 4.5)] - runs[(True, 0.0)]).max() > 1e-3


def test_pxz_symmetries():
    # the xz pressure changes sign under the mirror x -> -x and is unchanged
    # when the x and z axes are exchanged (a cubic box): a wrong component
    # (xx, zz) or a missing kinetic or virial part breaks one of the two
    c = I.lj_fcc(5, 5, 5, density=0.8442)
    g = np.random.default_rng(7)
    x = np.mod(c.x + g.normal(0, 0.1, c.x.shape), c.box)
    v = I.maxwell_velocities(c.n, 1.3, seed=7)
    st = O.State(c.box, x, v)
    o = O.observables(LJ_FLUID, st)
    assert abs(o["pxz"]) > 1e-3
    xm = x.copy()
    xm[:, 0] = np.mod(-xm[:, 0], c.box[0])
    vm = v.copy()
    vm[:, 0] = -vm[:, 0]
    om = O.observables(LJ_FLUID, O.State(c.box, xm, vm))
    assert abs(om["pxz"] + o["pxz"]) < 1e-10 * max(1.0, abs(o["pressure"]))
    assert abs(om["pressure"] - o["pressure"]) < 1e-10 * abs(o["pressure"])
    xs, vs = x[:, ::-1].copy(), v[:, ::-1].copy()   # (x, y, z) -> (z, y, x)
    os_ = O.observables(LJ_FLUID, O.State(c.box, xs, vs))
    assert abs(os_["pxz"] - o["pxz"]) < 1e-10 * max(1.0, abs(o["pressure"]))
    # the kinetic part alone: no pair within the cutoff
    far = O.State(np.array([40.0, 40.0, 40.0]), np.array([[5.0, 5.0, 5.0], [30.0, 30.0, 30.0]]),
                  np.array([[1.0, 0.0, 2.0], [0.5, 0.0, -1.0]]))
    assert abs(O.observables(LJ_FLUID, far)["pxz"] - (1.0 * 2.0 + 0.5 * -1.0) / 40.0 ** 3) < 1e-15
