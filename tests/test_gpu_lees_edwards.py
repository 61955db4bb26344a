"""GPU parity tests of Lees-Edwards boundary conditions (paper "State of the
field" and "New features": Lees-Edwards) through the C ABI against the
oracle: flow along x, gradient along z, offset delta = gdot Lz t.
Tolerances as for the periodic box: FP64 trajectories to 1e-10 in position
(sheared minimum image of the difference) and 1e-9 in velocity; FP32 one step
to a few float ulps and 1e-5 relative RMS; batched replicas and resumed runs
bit-identical."""
import numpy as np
import pytest

import oracle as O
from paper_2608_14911_gb300 import espp

from _systems import WCA_RC, kg_case, lj_case, rel_rms

pytestmark = pytest.mark.gpu

FP32, FP64 = espp.ESPP_FP32, espp.ESPP_FP64
DPD = espp.ESPP_THERMO_DPD


@pytest.fixture
def oracle_le():
    def on(shear, dpd_rc=None):
        O.set_lees_edwards(True, shear)
        if dpd_rc is not None:
            O.set_dpd(True, dpd_rc)
    yield on
    O.set_lees_edwards(False)
    O.set_dpd(False)


def le_diff(a, b, box, delta):
    """Sheared minimum image of a - b (rows)."""
    d = a - b
    k = np.rint(d[:, 2] / box[2])
    d[:, 2] -= k * box[2]
    d[:, 0] -= k * delta
    d[:, 0] -= np.rint(d[:, 0] / box[0]) * box[0]
    d[:, 1] -= np.rint(d[:, 1] / box[1]) * box[1]
    return d


def _run_pair(case, prec, shear, t0, nsteps, dt, gamma, kT, seed, dpd_rc=None):
    s = case.system(prec, seed=seed, build=False)
    s.set_lees_edwards(True, shear, t0)
    s.build_neighbors(case.rc_list, case.skin)
    if dpd_rc is not None:
        s.set_thermostat(DPD, dpd_rc)
    s.integrate(nsteps, dt, gamma, kT)
    st = case.oracle_state()
    st.time = t0
    O.integrate(case.model, st, nsteps, dt, gamma, kT, seed=seed)
    return s, st


@pytest.mark.parametrize("nsteps", [1, 7, 150])
def test_le_langevin_lj_fp64_matches_oracle(nsteps, oracle_le):
    case = lj_case()
    shear, t0 = 0.3, 3.7
    oracle_le(shear)
    s, st = _run_pair(case, FP64, shear, t0, nsteps, 0.005, 1.0, 0.72, 31)
    x, v, img = s.get_state()
    box = case.cfg.box
    _, _, t = s.lees_edwards()
    assert abs(t - (t0 + nsteps * 0.005)) < 1e-12 and abs(st.time - t) < 1e-12
    delta = shear * box[2] * t
    assert np.abs(le_diff(x, st.x, box, delta)).max() < 1e-10
    assert np.abs(v - st.v).max() < 1e-9
    assert np.array_equal(img, st.img)
    s.close()


@pytest.mark.parametrize("nsteps", [7, 150])
def test_le_dpd_kg_fp64_matches_oracle(nsteps, oracle_le):
    case = kg_case()
    shear = 0.5
    oracle_le(shear, WCA_RC)
    s, st = _run_pair(case, FP64, shear, 0.0, nsteps, 0.005, 4.5, 1.0, 17, dpd_rc=WCA_RC)
    x, v, img = s.get_state()
    box = case.cfg.box
    delta = shear * box[2] * st.time
    assert np.abs(le_diff(x, st.x, box, delta)).max() < 1e-10
    assert np.abs(v - st.v).max() < 1e-9
    assert np.array_equal(img, st.img)
    # observables of the sheared state, kinetic terms relative to the profile
    o = s.observables()
    oo = O.observables(case.model, st)
    for k in ("ke", "pe_pair", "pe_bond", "virial", "temperature", "pressure", "pxz", "mean_bond", "rg2"):
        assert abs(o[k] - oo[k]) <= 1e-9 * max(1.0, abs(oo[k])), (k, o[k], oo[k])
    s.close()


def test_le_fp32_single_step(oracle_le):
    case = lj_case()
    shear, t0 = 0.4, 11.3
    oracle_le(shear)
    s, st = _run_pair(case, FP32, shear, t0, 1, 0.005, 1.0, 0.72, 5)
    x, v, img = s.get_state()
    box = case.cfg.box
    ulp = np.spacing(np.float32(box.max()))
    delta = shear * box[2] * st.time
    assert np.abs(le_diff(x, st.x, box, delta)).max() <= 8 * ulp
    assert rel_rms(v, st.v) <= 1e-5
    s.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_le_neighbour_sets_match_oracle(prec, oracle_le):
    case = lj_case()
    shear, t = 0.7, 9.1
    oracle_le(shear)
    s = case.system(prec, build=False)
    s.set_lees_edwards(True, shear, t)
    s.build_neighbors(case.rc_list, case.skin)
    row, cols = s.get_neighbors()
    c = case.cfg
    rl = case.rc_list + case.skin
    orow, ocols = O.neighbors(c.box, c.x, rl, time=t)
    got = {(i, int(j)) for i in range(c.n) for j in cols[row[i]:row[i + 1]]}
    want = {(i, int(j)) for i in range(c.n) for j in ocols[orow[i]:orow[i + 1]]}
    if prec == FP64:
        assert got == want
    else:
        # FP32: only pairs within a float rounding of the list cutoff may differ
        delta = shear * c.box[2] * t
        for i, j in got ^ want:
            d = le_diff(c.x[i:i + 1], c.x[j:j + 1], c.box, delta)
            assert abs(np.sqrt((d ** 2).sum()) - rl) < 1e-5
    # every pair across a sheared face is there
    assert any(abs(c.x[i, 2] - c.x[j, 2]) > c.box[2] / 2 for i, j in want)
    s.close()


def test_le_zero_shear_is_the_periodic_box():
    case = lj_case()
    a = case.system(FP64, seed=3)
    a.integrate(100, 0.005, 1.0, 0.72)
    b = case.system(FP64, seed=3, build=False)
    b.set_lees_edwards(True, 0.0, 0.0)
    b.build_neighbors(case.rc_list, case.skin)
    b.integrate(100, 0.005, 1.0, 0.72)
    xa, va, ia = a.get_state()
    xb, vb, ib = b.get_state()
    assert np.abs(xa - xb).max() < 1e-10 and np.abs(va - vb).max() < 1e-9
    assert np.array_equal(ia, ib)


def test_le_batched_replicas_equal_standalone_runs():
    sizes = [(3, 40, 101), (11, 20, 202), (5, 77, 303)]
    cases_ = [kg_case(nc, nb, seed=sd, jitter=0.08) for nc, nb, sd in sizes]
    reps = [dict(box=c.cfg.box, n=c.cfg.n, types=c.cfg.types, bonds=c.cfg.bonds, seed=3000 + k)
            for k, c in enumerate(cases_)]
    shear, t0 = 0.6, 2.5
    b = espp.System(replicas=reps, precision=FP32)
    b.set_wca()
    b.set_fene()
    b.set_state(np.concatenate([c.cfg.x for c in cases_]), np.concatenate([c.v for c in cases_]),
                np.concatenate([c.cfg.img for c in cases_]))
    b.set_lees_edwards(True, shear, t0)
    b.build_neighbors(WCA_RC, 0.4)
    b.set_thermostat(DPD, WCA_RC)
    b.integrate(300, 0.005, 1.0, 1.0)
    xb, vb, ib = b.get_state()
    off = 0
    for k, c in enumerate(cases_):
        s = c.system(FP32, seed=3000 + k, build=False)
        s.set_lees_edwards(True, shear, t0)
        s.build_neighbors(WCA_RC, 0.4)
        s.set_thermostat(DPD, WCA_RC)
        s.integrate(300, 0.005, 1.0, 1.0)
        x, v, img = s.get_state()
        n = c.cfg.n
        assert np.array_equal(x, xb[off:off + n])
        assert np.array_equal(v, vb[off:off + n])
        assert np.array_equal(img, ib[off:off + n])
        off += n
        s.close()
    b.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_le_checkpoint_resume_is_bit_exact(prec, tmp_path):
    case = kg_case()
    path = str(tmp_path / "le.ckpt")

    def make():
        s = case.system(prec, seed=9, build=False)
        s.set_lees_edwards(True, 0.8, 1.25)
        s.build_neighbors(case.rc_list, case.skin)
        s.set_thermostat(DPD, WCA_RC)
        return s

    a = make()
    a.integrate(173, 0.005, 1.0, 1.0)
    a.checkpoint_save(path)
    a.integrate(211, 0.005, 1.0, 1.0)
    b = case.system(prec, seed=9)
    b.set_thermostat(DPD, WCA_RC)
    b.checkpoint_load(path)
    assert b.lees_edwards()[0] and abs(b.lees_edwards()[2] - (1.25 + 173 * 0.005)) < 1e-12
    b.integrate(211, 0.005, 1.0, 1.0)
    for p, q in zip(a.get_state(), b.get_state()):
        assert np.array_equal(p, q)
    a.close()
    b.close()


def test_le_direct_launches_equal_graphs():
    case = lj_case()
    out = []
    for chunk in (None, 0):
        s = case.system(FP32, seed=4, build=False)
        s.set_lees_edwards(True, 0.5, 0.0)
        s.build_neighbors(case.rc_list, case.skin)
        if chunk is not None:
            s.set_graph_chunk(chunk)
        s.integrate(150, 0.005, 1.0, 0.72)
        out.append(s.get_state())
        s.close()
    for p, q in zip(*out):
        assert np.array_equal(p, q)


def test_le_keeps_a_linear_profile_at_scale():
    # a 24,000-particle ideal DPD gas (density 3, rc 1, gamma 4.5, kT 1)
    # sheared through the boundaries, started on the linear profile: the mean
    # x velocity stays on gdot (z - Lz/2) in every slab, the temperature
    # relative to it stays at the bath's, the xz pressure is negative
    # (momentum flows down the gradient)
    from paper_2608_14911_gb300 import inputs as I
    L, shear = 20.0, 0.1
    box = np.array([L, L, L])
    n = int(3 * L ** 3)
    c = I.random_positions(n, box, seed=7)
    v = I.maxwell_velocities(n, 1.0, seed=7)
    v[:, 0] += shear * (c.x[:, 2] - L / 2)
    s = espp.System(box, n, c.types, c.bonds, precision=FP32, seed=7)
    s.set_lj(0.0, 1.0, 1.0, False)  # no conservative force
    s.set_state(c.x, v, c.img)
    s.set_lees_edwards(True, shear, 0.0)
    s.build_neighbors(1.0, 0.3)
    s.set_thermostat(DPD, 1.0)
    s.integrate(500, 0.01, 4.5, 1.0)
    slopes, temps, pxz, prof = [], [], [], []
    for _ in range(10):
        s.integrate(250, 0.01, 4.5, 1.0)
        x, vv, _ = s.get_state()
        slopes.append(np.polyfit(x[:, 2] - L / 2, vv[:, 0], 1)[0])
        b = np.minimum((x[:, 2] / L * 10).astype(int), 9)
        prof.append([vv[b == k, 0].mean() for k in range(10)])
        o = s.observables()
        temps.append(o["temperature"])
        pxz.append(o["pxz"])
    assert abs(np.mean(slopes) - shear) < 0.03 * shear, slopes
    line = shear * ((np.arange(10) + 0.5) * L / 10 - L / 2)
    assert np.abs(np.mean(prof, axis=0) - line).max() < 0.05 * shear * L
    assert abs(np.mean(temps) - 1.0) < 0.03, temps
    assert np.mean(pxz) < -5 * np.std(pxz) / np.sqrt(len(pxz)), pxz
    assert s.error_word == 0
    s.close()


def test_le_errors():
    case = lj_case()
    s = case.system(FP32)
    for bad in (float("nan"), float("inf")):
        with pytest.raises(espp.EsppError) as e:
            s.set_lees_edwards(True, bad, 0.0)
        assert e.value.code == espp.ESPP_ERR_ARG
    s.set_lees_edwards(True, 0.2, 0.0)
    import torch
    xo = torch.zeros((case.cfg.n // 4) * 3, dtype=torch.float64, device="cuda")
    fo = torch.zeros_like(xo)
    with pytest.raises(espp.EsppError) as e:
        s.cg_map(4, xo, fo)
    assert e.value.code == espp.ESPP_ERR_STATE
    s.set_lees_edwards(False)
    s.integrate(5, 0.005, 1.0, 0.72)
    s.close()


@pytest.mark.parametrize("method", [espp.ESPP_FORCES_VERLET, espp.ESPP_FORCES_CELLS])
def test_le_two_types_fp64_matches_oracle(method, oracle_le):
    # the general (several types) step-kernel variant across sheared faces,
    # over the Verlet list and over the cell stencil
    from _systems import two_type_case
    case = two_type_case()
    box = case.cfg.box
    # start where the offset is two whole boxes: the lattice start then meets
    # its sheared images without overlaps
    shear = 0.35
    t0 = 2 * box[0] / (shear * box[2])
    oracle_le(shear)
    s = case.system(FP64, seed=41, build=False)
    s.set_force_method(method)
    s.set_lees_edwards(True, shear, t0)
    s.build_neighbors(case.rc_list, case.skin)
    s.integrate(80, 0.005, 1.0, 1.0)
    x, v, img = s.get_state()
    st = case.oracle_state()
    st.time = t0
    O.integrate(case.model, st, 80, 0.005, 1.0, 1.0, seed=41)
    delta = shear * box[2] * st.time
    assert np.abs(le_diff(x, st.x, box, delta)).max() < 1e-10
    assert np.abs(v - st.v).max() < 1e-9
    o, oo = s.observables(), O.observables(case.model, st)
    for k in ("pe_pair", "virial", "pxz", "temperature"):
        assert abs(o[k] - oo[k]) <= 1e-9 * max(1.0, abs(oo[k])), (k, o[k], oo[k])
    s.close()
