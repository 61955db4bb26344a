"""GPU parity tests of the DPD thermostat (paper "Functionality": dissipative
particle dynamics) through the C ABI against the oracle.  Tolerances as for
the Langevin path: FP64 trajectories to 1e-10 in position and 1e-9 in
velocity, an FP32 step to a few float ulps in position and 1e-5 relative RMS
in velocity, batched replicas bit-identical to standalone runs."""
import numpy as np
import pytest

import oracle as O
from paper_2608_14911_gb300 import espp

from _systems import WCA_RC, kg_case, lj_case, rel_rms

pytestmark = pytest.mark.gpu

FP32, FP64 = espp.ESPP_FP32, espp.ESPP_FP64
DPD = espp.ESPP_THERMO_DPD
GAMMA, KT, DT = 4.5, 1.0, 0.005


@pytest.fixture
def oracle_dpd():
    def on(rc):
        O.set_dpd(True, rc)
    yield on
    O.set_dpd(False)


def _unwrapped(x, img, box):
    return x + img * box


def _drift(case, u=(0.02, -0.01, 0.005)):
    case.v = case.v + np.array(u)
    return case


CASES = {
    "lj": (lambda: lj_case(), 1.0),
    "kg": (lambda: kg_case(), WCA_RC),
}


@pytest.mark.parametrize("nsteps", [1, 7, 150])
@pytest.mark.parametrize("name", ["lj", "kg"])
def test_dpd_fp64_matches_oracle(name, nsteps, oracle_dpd):
    make, rc = CASES[name]
    case = make()
    s = case.system(FP64, seed=21)
    s.set_thermostat(DPD, rc)
    s.integrate(nsteps, DT, GAMMA, KT)
    x, v, img = s.get_state()
    oracle_dpd(rc)
    st = case.oracle_state()
    O.integrate(case.model, st, nsteps, DT, GAMMA, KT, seed=21)
    box = case.cfg.box
    assert np.abs(_unwrapped(x, img, box) - _unwrapped(st.x, st.img, box)).max() < 1e-10
    assert np.abs(v - st.v).max() < 1e-9
    s.close()


def test_dpd_fp32_single_step(oracle_dpd):
    case = lj_case()
    s = case.system(FP32, seed=5)
    s.set_thermostat(DPD, 1.0)
    s.integrate(1, DT, GAMMA, KT)
    x, v, img = s.get_state()
    oracle_dpd(1.0)
    st = case.oracle_state()
    O.integrate(case.model, st, 1, DT, GAMMA, KT, seed=5)
    box = case.cfg.box
    ulp = np.spacing(np.float32(box.max()))
    assert np.abs(_unwrapped(x, img, box) - _unwrapped(st.x, st.img, box)).max() <= 4 * ulp
    assert rel_rms(v, st.v) <= 1e-5
    s.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_dpd_conserves_momentum(prec):
    case = _drift(lj_case())
    s = case.system(prec, seed=8)
    s.set_thermostat(DPD, 1.0)
    p0 = case.v.sum(axis=0)
    s.integrate(400, DT, GAMMA, KT)
    _, v, _ = s.get_state()
    tol = 1e-9 if prec == FP64 else 2e-3
    assert np.abs(v.sum(axis=0) - p0).max() < tol
    # the Langevin thermostat on the same system does not conserve it
    s.set_thermostat(espp.ESPP_THERMO_LANGEVIN)
    s.integrate(400, DT, GAMMA, KT)
    _, v, _ = s.get_state()
    assert np.abs(v.sum(axis=0) - p0).max() > 1.0
    s.close()


def test_dpd_batched_replicas_equal_standalone_runs():
    sizes = [(3, 40, 101), (11, 20, 202), (5, 77, 303)]
    cases_ = [kg_case(nc, nb, seed=sd, jitter=0.08) for nc, nb, sd in sizes]
    reps = [dict(box=c.cfg.box, n=c.cfg.n, types=c.cfg.types, bonds=c.cfg.bonds, seed=2000 + k)
            for k, c in enumerate(cases_)]
    b = espp.System(replicas=reps, precision=FP32)
    b.set_wca()
    b.set_fene()
    b.set_state(np.concatenate([c.cfg.x for c in cases_]), np.concatenate([c.v for c in cases_]),
                np.concatenate([c.cfg.img for c in cases_]))
    b.build_neighbors(WCA_RC, 0.4)
    b.set_thermostat(DPD, WCA_RC)
    b.integrate(300, DT, GAMMA, KT)
    xb, vb, ib = b.get_state()
    off = 0
    for k, c in enumerate(cases_):
        s = c.system(FP32, seed=2000 + k)
        s.set_thermostat(DPD, WCA_RC)
        s.integrate(300, DT, GAMMA, KT)
        x, v, img = s.get_state()
        n = c.cfg.n
        assert np.array_equal(x, xb[off:off + n])
        assert np.array_equal(v, vb[off:off + n])
        assert np.array_equal(img, ib[off:off + n])
        off += n
        s.close()
    b.close()


def test_dpd_direct_launches_equal_graphs():
    case = lj_case()
    a = case.system(FP32, seed=4)
    a.set_thermostat(DPD, 1.0)
    a.integrate(120, DT, GAMMA, KT)
    b = case.system(FP32, seed=4)
    b.set_thermostat(DPD, 1.0)
    b.set_graph_chunk(0)
    b.integrate(120, DT, GAMMA, KT)
    for p, q in zip(a.get_state(), b.get_state()):
        assert np.array_equal(p, q)
    # one velocity-snapshot kernel per step on top of the Langevin path's
    c = case.system(FP32, seed=4)
    c.set_graph_chunk(0)
    c.integrate(120, DT, GAMMA, KT)
    deltas = []
    for s in (b, c):
        n0 = s.kernel_launches
        s.integrate(10, DT, GAMMA, KT)
        deltas.append(s.kernel_launches - n0)
    assert deltas[0] - deltas[1] == 10
    for s in (a, b, c):
        s.close()


def test_thermostat_switch_and_errors():
    case = lj_case()
    ref = case.system(FP64, seed=6)
    ref.integrate(50, DT, 1.0, KT)
    s = case.system(FP64, seed=6)
    s.set_thermostat(DPD, 1.0)
    s.set_thermostat(espp.ESPP_THERMO_LANGEVIN)
    s.integrate(50, DT, 1.0, KT)
    for p, q in zip(ref.get_state(), s.get_state()):
        assert np.array_equal(p, q)
    for kind, rc in ((7, 1.0), (DPD, 0.0), (DPD, -1.0), (DPD, float("nan"))):
        with pytest.raises(espp.EsppError) as e:
            s.set_thermostat(kind, rc)
        assert e.value.code == espp.ESPP_ERR_ARG
    # a DPD cutoff beyond the list cutoff (2.5) is refused at integrate
    s.set_thermostat(DPD, 2.6)
    with pytest.raises(espp.EsppError) as e:
        s.integrate(1, DT, GAMMA, KT)
    assert e.value.code == espp.ESPP_ERR_ARG
    s.set_thermostat(DPD, 2.5)
    s.integrate(3, DT, GAMMA, KT)
    ref.close()
    s.close()
