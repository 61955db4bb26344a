"""GPU parity tests of the list-free force method (pair forces from the cell
stencil, cells of rc / w, binned every step) through the C ABI: forces and
trajectories against the oracle with the same tolerances as the Verlet path
(FP32 forces 1e-5 relative RMS, FP64 1e-12; FP64 trajectories 1e-10), the
same trajectories as the Verlet list up to rounding, bit-identical batched
replicas and resumed runs."""
import numpy as np
import pytest

import oracle as O
from paper_2608_14911_gb300 import espp, inputs as I

from _systems import WCA_RC, capped_case, kg_case, lj_case, rel_rms, two_type_case

pytestmark = pytest.mark.gpu

FP32, FP64 = espp.ESPP_FP32, espp.ESPP_FP64
CELLS, VERLET = espp.ESPP_FORCES_CELLS, espp.ESPP_FORCES_VERLET
DPD = espp.ESPP_THERMO_DPD
FORCE_TOL = {FP32: 1e-5, FP64: 1e-12}


def cells_system(case, prec, seed=42, w=0):
    s = case.system(prec, seed=seed, build=False)
    s.set_force_method(CELLS)
    if w:
        s.set_cell_subdivision(w)
    s.build_neighbors(case.rc_list, case.skin)
    return s


def _unwrapped(x, img, box):
    return x + img * box


def cases():
    return [kg_case(), kg_case(7, 23, seed=5, jitter=0.1), lj_case(), two_type_case(), capped_case()]


@pytest.mark.parametrize("w", [1, 2])
@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", cases(), ids=lambda c: c.name)
def test_cell_forces_match_oracle(case, prec, w):
    s = cells_system(case, prec, w=w)
    f = s.compute_forces()
    c = case.cfg
    fo, _ = O.forces(case.model, c.box, c.x, c.types, c.bonds)
    assert rel_rms(f, fo) <= FORCE_TOL[prec]
    o = s.observables()
    oo = O.observables(case.model, case.oracle_state())
    tol = 1e-12 if prec == FP64 else 2e-6
    for k in ("pe_pair", "pe_bond", "virial", "pressure"):
        assert abs(o[k] - oo[k]) <= tol * max(1.0, abs(oo[k])), (k, o[k], oo[k])
    # the off-diagonal pressure is a sum of terms of both signs: gated
    # against the scale of the pressure
    assert abs(o["pxz"] - oo["pxz"]) <= 5 * tol * max(1.0, abs(oo["pressure"])), (o["pxz"], oo["pxz"])
    s.close()


@pytest.mark.parametrize("case_fn", [kg_case, lj_case, two_type_case], ids=["kg", "lj", "two"])
def test_cell_fp64_trajectory_matches_oracle(case_fn):
    case = case_fn()
    s = cells_system(case, FP64, seed=13)
    s.integrate(150, 0.005, 1.0, 1.0)
    x, v, img = s.get_state()
    st = case.oracle_state()
    O.integrate(case.model, st, 150, 0.005, 1.0, 1.0, seed=13)
    box = case.cfg.box
    assert np.abs(_unwrapped(x, img, box) - _unwrapped(st.x, st.img, box)).max() < 1e-10
    assert np.abs(v - st.v).max() < 1e-9
    s.close()


def test_cell_dpd_and_lees_edwards_match_oracle():
    case = kg_case()
    shear = 0.5
    O.set_lees_edwards(True, shear)
    O.set_dpd(True, WCA_RC)
    try:
        s = case.system(FP64, seed=19, build=False)
        s.set_force_method(CELLS)
        s.set_lees_edwards(True, shear, 0.7)
        s.build_neighbors(case.rc_list, case.skin)
        s.set_thermostat(DPD, WCA_RC)
        s.integrate(120, 0.005, 4.5, 1.0)
        x, v, img = s.get_state()
        st = case.oracle_state()
        st.time = 0.7
        O.integrate(case.model, st, 120, 0.005, 4.5, 1.0, seed=19)
        box = case.cfg.box
        delta = shear * box[2] * st.time
        d = x - st.x
        k = np.rint(d[:, 2] / box[2])
        d[:, 2] -= k * box[2]
        d[:, 0] -= k * delta
        d -= np.rint(d / box) * box
        assert np.abs(d).max() < 1e-10
        assert np.abs(v - st.v).max() < 1e-9
        assert np.array_equal(img, st.img)
        o = s.observables()
        oo = O.observables(case.model, st)
        for key in ("ke", "temperature", "pxz", "rg2", "virial"):
            assert abs(o[key] - oo[key]) <= 1e-9 * max(1.0, abs(oo[key])), key
        s.close()
    finally:
        O.set_lees_edwards(False)
        O.set_dpd(False)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_cells_and_verlet_give_the_same_run(prec):
    case = lj_case()
    a = case.system(prec, seed=8)
    a.integrate(100, 0.005, 1.0, 0.72)
    b = cells_system(case, prec, seed=8)
    b.integrate(100, 0.005, 1.0, 0.72)
    xa, va, ia = a.get_state()
    xb, vb, ib = b.get_state()
    box = case.cfg.box
    tol = 1e-10 if prec == FP64 else 2e-3
    assert np.abs(_unwrapped(xa, ia, box) - _unwrapped(xb, ib, box)).max() < tol
    assert b.list_stats() == (0, 0)
    assert b.n_rebuilds >= 100  # binned every step


def test_cell_batched_replicas_equal_standalone_runs():
    sizes = [(3, 40, 101), (11, 20, 202), (5, 77, 303)]
    cases_ = [kg_case(nc, nb, seed=sd, jitter=0.08) for nc, nb, sd in sizes]
    reps = [dict(box=c.cfg.box, n=c.cfg.n, types=c.cfg.types, bonds=c.cfg.bonds, seed=4000 + k)
            for k, c in enumerate(cases_)]
    b = espp.System(replicas=reps, precision=FP32)
    b.set_wca()
    b.set_fene()
    b.set_state(np.concatenate([c.cfg.x for c in cases_]), np.concatenate([c.v for c in cases_]),
                np.concatenate([c.cfg.img for c in cases_]))
    b.set_force_method(CELLS)
    b.build_neighbors(WCA_RC, 0.4)
    b.integrate(200, 0.005, 1.0, 1.0)
    xb, vb, ib = b.get_state()
    off = 0
    for k, c in enumerate(cases_):
        s = cells_system(c, FP32, seed=4000 + k)
        s.integrate(200, 0.005, 1.0, 1.0)
        x, v, img = s.get_state()
        n = c.cfg.n
        assert np.array_equal(x, xb[off:off + n])
        assert np.array_equal(v, vb[off:off + n])
        assert np.array_equal(img, ib[off:off + n])
        off += n
        s.close()
    b.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_cell_checkpoint_resume_is_bit_exact(prec, tmp_path):
    case = kg_case()
    a = cells_system(case, prec, seed=23)
    a.integrate(137, 0.005, 1.0, 1.0)
    path = str(tmp_path / "cells.ckpt")
    a.checkpoint_save(path)
    a.integrate(211, 0.005, 1.0, 1.0)
    b = cells_system(case, prec, seed=5)
    b.checkpoint_load(path)
    b.integrate(211, 0.005, 1.0, 1.0)
    for p, q in zip(a.get_state(), b.get_state()):
        assert np.array_equal(p, q)


def test_cell_direct_launches_equal_graphs():
    case = kg_case()
    out = []
    for chunk in (None, 0):
        s = cells_system(case, FP32, seed=4)
        if chunk is not None:
            s.set_graph_chunk(chunk)
        s.integrate(120, 0.005, 1.0, 1.0)
        out.append(s.get_state())
        s.close()
    for p, q in zip(*out):
        assert np.array_equal(p, q)


def test_tuner_times_both_and_keeps_the_state():
    case = kg_case()
    s = case.system(FP32, seed=2)
    s.integrate(50, 0.005, 1.0, 1.0)
    before = s.get_state()
    step = s.step
    ms, chosen = s.tune_force_method(40, 0.005, 1.0, 1.0)
    assert len(ms) == espp.FORCE_SHAPES and np.isfinite(ms[0]) and np.isfinite(ms[3]) and min(ms) > 0
    assert chosen == int(np.argmin(ms))
    assert s.step == step
    for p, q in zip(before, s.get_state()):
        assert np.array_equal(p, q)
    s.integrate(20, 0.005, 1.0, 1.0)
    assert s.error_word == 0
    s.close()


def test_cell_mode_errors():
    case = lj_case()
    s = cells_system(case, FP32)
    with pytest.raises(espp.EsppError) as e:
        s.get_neighbors()
    assert e.value.code == espp.ESPP_ERR_STATE
    with pytest.raises(espp.EsppError) as e:
        s.set_force_method(7)
    assert e.value.code == espp.ESPP_ERR_ARG
    # the RDF falls back to all pairs and still counts the same pairs
    got = s.rdf_counts(2.0, 40)
    exp = O.rdf_counts(case.cfg.box, case.cfg.x, 2.0, 40)
    assert got.sum() == exp.sum()
    s.set_force_method(VERLET)
    s.integrate(5, 0.005, 1.0, 0.72)
    assert s.list_stats()[0] > 0
    s.close()


def test_checkpoint_moves_between_force_methods(tmp_path):
    # a state saved in the list-free mode resumes on a Verlet-list handle and
    # the other way round, with forces equal to the oracle's at the saved state
    case = kg_case()
    path = str(tmp_path / "x.ckpt")
    for src, dst in ((CELLS, VERLET), (VERLET, CELLS)):
        a = case.system(FP64, seed=12, build=False)
        a.set_force_method(src)
        a.build_neighbors(case.rc_list, case.skin)
        a.integrate(77, 0.005, 1.0, 1.0)
        a.checkpoint_save(path)
        x, _, img = a.get_state()
        b = case.system(FP64, seed=12, build=False)
        b.set_force_method(dst)
        b.build_neighbors(case.rc_list, case.skin)
        b.checkpoint_load(path)
        f = b.compute_forces()
        fo, _ = O.forces(case.model, case.cfg.box, x, case.cfg.types, case.cfg.bonds)
        assert rel_rms(f, fo) <= FORCE_TOL[FP64]
        b.integrate(30, 0.005, 1.0, 1.0)
        assert b.error_word == 0
        a.close()
        b.close()
