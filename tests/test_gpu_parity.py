"""GPU parity tests: the CUDA path (through the C ABI) against the oracle on the
same seeded inputs.  Tolerances: neighbour sets exact outside a 1e-6 sigma band
at the list cutoff (FP32) or exact (FP64); single-step forces <= 1e-5 relative
RMS in FP32 and <= 1e-12 in FP64."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2608_14911_gb300 import espp, inputs as I

from _systems import (KG_BOND, KG_PAIR, LJ_PAIR, WCA_RC, Case, capped_case, kg_case, lj_case,
                      rel_rms, two_type_case)

pytestmark = pytest.mark.gpu

FP32, FP64 = espp.ESPP_FP32, espp.ESPP_FP64
FORCE_TOL = {FP32: 1e-5, FP64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available()


def cases():
    return [kg_case(), kg_case(7, 23, seed=5, jitter=0.1), lj_case(), two_type_case(),
            capped_case()]


# ---------------------------------------------------------------------------
def test_philox_stream_bit_exact():
    import torch
    for seed in (0, 42, (1 << 40) + 7):
        for step in (0, 1, 12345, (1 << 33) + 5):
            n = 1537
            out = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
            espp.espp_langevin_noise(seed, step, out)
            ref = O.langevin_noise(seed, step, n)
            assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", cases(), ids=lambda c: c.name)
def test_neighbour_sets_match_brute_force(case, prec):
    s = case.system(prec)
    row, cols = s.get_neighbors()
    c = case.cfg
    rl = case.rc_list + case.skin
    orow, ocols = O.neighbors(c.box, c.x, rl, method="brute")
    band = 1e-6 if prec == FP32 else 0.0
    for i in range(c.n):
        got = set(cols[row[i]:row[i + 1]].tolist())
        exp = set(ocols[orow[i]:orow[i + 1]].tolist())
        if got == exp:
            continue
        for j in got ^ exp:
            d = c.x[i] - c.x[j]
            d -= c.box * np.round(d / c.box)
            assert abs(np.linalg.norm(d) - rl) <= band, (i, j, np.linalg.norm(d))
    s.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", cases(), ids=lambda c: c.name)
def test_forces_match_oracle(case, prec):
    s = case.system(prec)
    f = s.compute_forces()
    c = case.cfg
    fo, _ = O.forces(case.model, c.box, c.x, c.types, c.bonds)
    assert rel_rms(f, fo) <= FORCE_TOL[prec]
    # a second explicit build (resort of an already sorted state) changes nothing
    s.build_neighbors(case.rc_list, case.skin)
    f2 = s.compute_forces()
    assert rel_rms(f2, fo) <= FORCE_TOL[prec]
    s.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_forces_device_pointers(prec):
    import torch
    case = kg_case()
    c = case.cfg
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=prec)
    s.set_wca()
    s.set_fene()
    x = torch.tensor(c.x, device="cuda")
    img = torch.tensor(c.img, device="cuda", dtype=torch.int32)
    s.set_state(x, None, img)
    s.build_neighbors(WCA_RC, 0.4)
    f = torch.zeros((c.n, 3), dtype=torch.float64, device="cuda")
    s.compute_forces(f)
    fo, _ = O.forces(case.model, c.box, c.x, c.types, c.bonds)
    assert rel_rms(f.cpu().numpy(), fo) <= FORCE_TOL[prec]
    xo = torch.zeros_like(x)
    vo = torch.zeros_like(x)
    io = torch.zeros_like(img)
    s.get_state((xo, vo, io))
    assert np.array_equal(xo.cpu().numpy(), c.x)
    assert np.array_equal(io.cpu().numpy(), c.img)
    s.close()


def _unwrapped(x, img, box):
    return x + img * box


@pytest.mark.parametrize("nsteps", [1, 7, 150])
@pytest.mark.parametrize("case_fn", [kg_case, lj_case, two_type_case], ids=["kg", "lj", "two"])
def test_integrate_fp64_matches_oracle(case_fn, nsteps):
    case = case_fn()
    s = case.system(FP64, seed=11)
    s.integrate(nsteps, 0.005, 1.0, 1.0)
    x, v, img = s.get_state()
    st = case.oracle_state()
    O.integrate(case.model, st, nsteps, 0.005, 1.0, 1.0, seed=11)
    box = case.cfg.box
    ux, uo = _unwrapped(x, img, box), _unwrapped(st.x, st.img, box)
    assert np.abs(ux - uo).max() < 1e-10
    assert np.abs(v - st.v).max() < 1e-9
    assert s.step == nsteps
    s.close()


def test_integrate_fp64_split_calls_equal_one_call():
    case = kg_case()
    a = case.system(FP64, seed=3)
    a.integrate(90, 0.005, 1.0, 1.0)
    b = case.system(FP64, seed=3)
    for k in (1, 2, 64, 23):
        b.integrate(k, 0.005, 1.0, 1.0)
    xa, va, ia = a.get_state()
    xb, vb, ib = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ia, ib)


@pytest.mark.parametrize("case_fn", [kg_case, lj_case], ids=["kg", "lj"])
def test_integrate_fp32_single_step(case_fn):
    case = case_fn()
    s = case.system(FP32, seed=5)
    s.integrate(1, 0.005, 1.0, 1.0)
    x, v, img = s.get_state()
    st = case.oracle_state()
    O.integrate(case.model, st, 1, 0.005, 1.0, 1.0, seed=5)
    box = case.cfg.box
    ulp = np.spacing(np.float32(box.max()))
    assert np.abs(_unwrapped(x, img, box) - _unwrapped(st.x, st.img, box)).max() <= 4 * ulp
    assert rel_rms(v, st.v) <= 1e-5


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case_fn", [kg_case, lj_case, two_type_case], ids=["kg", "lj", "two"])
def test_observables_match_oracle(case_fn, prec):
    case = case_fn()
    s = case.system(prec)
    o = s.observables()
    oo = O.observables(case.model, case.oracle_state())
    tol = 1e-12 if prec == FP64 else 2e-6
    for k in ("pe_pair", "pe_bond", "virial", "ke", "temperature", "pressure", "mean_bond", "rg2"):
        ref = oo[k]
        assert abs(o[k] - ref) <= tol * max(1.0, abs(ref)), (k, o[k], ref)
    assert o["n_molecules"] == int(oo["nmol"])


def _edge_pairs(box, x, rmax, nbins, band):
    """Per bin edge k (k = 0..nbins, edge k at k rmax / nbins): the number of
    unique pairs whose minimum-image distance lies within a relative `band`
    of that edge.  Only such pairs can land in different bins on two sides
    that round the distance differently."""
    n = x.shape[0]
    near = np.zeros(nbins + 1, dtype=np.int64)
    dr = rmax / nbins
    for i in range(n - 1):
        d = x[i] - x[i + 1:]
        d -= box * np.round(d / box)
        r = np.sqrt((d * d).sum(axis=1))
        r = r[r < rmax * (1 + band)]
        k = np.rint(r / dr).astype(np.int64)
        close = np.abs(r - k * dr) <= band * np.maximum(r, dr)
        np.add.at(near, k[close & (k <= nbins)], 1)
    return near


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_rdf_counts_match_oracle(prec):
    # counts equal the oracle's bin by bin, except for pairs the two sides
    # may round across a bin edge: those are counted and named (for the FP64
    # path the band is 1e-12 relative, and this seed has none, so the FP64
    # counts are compared exactly)
    case = lj_case((6, 6, 6))
    s = case.system(prec)
    c = case.cfg
    for rmax, nbins in ((3.0, 60), (4.5, 90)):   # from the list, then from all pairs
        got = s.rdf_counts(rmax, nbins)
        exp = O.rdf_counts(c.box, c.x, rmax, nbins)
        near = _edge_pairs(c.box, c.x, rmax, nbins, 1e-12 if prec == FP64 else 1e-6)
        if prec == FP64:
            assert near.sum() == 0
            assert np.array_equal(got, exp), np.nonzero(got != exp)
        else:
            # a pair near edge k moves between bins k - 1 and k; near the
            # outer edge it may drop out of the histogram
            slack = near[:-1] + near[1:]
            assert np.all(np.abs(got - exp) <= slack), (np.nonzero(np.abs(got - exp) > slack), near.sum())
            assert abs(int(got.sum()) - int(exp.sum())) <= near[-1]


def test_batched_replicas_equal_standalone_runs():
    sizes = [(3, 40, 101), (11, 20, 202), (5, 77, 303)]
    cases_ = [kg_case(nc, nb, seed=sd, jitter=0.08) for nc, nb, sd in sizes]
    reps = [dict(box=c.cfg.box, n=c.cfg.n, types=c.cfg.types, bonds=c.cfg.bonds, seed=1000 + k)
            for k, c in enumerate(cases_)]
    b = espp.System(replicas=reps, precision=FP32)
    b.set_wca()
    b.set_fene()
    b.set_state(np.concatenate([c.cfg.x for c in cases_]), np.concatenate([c.v for c in cases_]),
                np.concatenate([c.cfg.img for c in cases_]))
    b.build_neighbors(WCA_RC, 0.4)
    b.integrate(300, 0.005, 1.0, 1.0)
    xb, vb, ib = b.get_state()
    off = 0
    for k, c in enumerate(cases_):
        s = c.system(FP32, seed=1000 + k)
        s.integrate(300, 0.005, 1.0, 1.0)
        x, v, img = s.get_state()
        n = c.cfg.n
        assert np.array_equal(x, xb[off:off + n])
        assert np.array_equal(v, vb[off:off + n])
        assert np.array_equal(img, ib[off:off + n])
        off += n
    obs = b.observables()
    assert len(obs) == 3 and all(o["n"] == c.cfg.n for o, c in zip(obs, cases_))


def test_list_overflow_is_retried(monkeypatch):
    monkeypatch.setenv("ESPP_FAULT_LIST_CAP", "4")
    case = lj_case()
    s = case.system(FP32)
    assert s.list_capacity > 4
    f = s.compute_forces()
    fo, _ = O.forces(case.model, case.cfg.box, case.cfg.x, case.cfg.types, case.cfg.bonds)
    assert rel_rms(f, fo) <= 1e-5
    monkeypatch.setenv("ESPP_FAULT_LIST_CAP", "8")
    s2 = case.system(FP64)
    s2.integrate(40, 0.005, 1.0, 0.72)
    x, v, img = s2.get_state()
    st = case.oracle_state()
    O.integrate(case.model, st, 40, 0.005, 1.0, 0.72, seed=42)
    assert np.abs(_unwrapped(x, img, case.cfg.box) - _unwrapped(st.x, st.img, case.cfg.box)).max() < 1e-10


@pytest.mark.parametrize("w", [2, 3])
@pytest.mark.parametrize("case", [kg_case(), lj_case(), two_type_case()], ids=lambda c: c.name)
def test_cell_subdivision_keeps_the_list(case, w):
    # sub-cells (paper: cell sub-decomposition) change the search, not the list
    a = case.system(FP64)
    b = case.system(FP64, build=False)
    b.set_cell_subdivision(w)
    b.build_neighbors(case.rc_list, case.skin)
    ra, ca = a.get_neighbors()
    rb, cb = b.get_neighbors()
    assert np.array_equal(ra, rb)
    for i in range(case.cfg.n):
        assert set(ca[ra[i]:ra[i + 1]].tolist()) == set(cb[rb[i]:rb[i + 1]].tolist())
    assert rel_rms(b.compute_forces(), a.compute_forces()) <= 1e-13
    # a trajectory with sub-cells (rebuilds and resorts included) follows the oracle
    b.set_resort_interval(20)
    b.integrate(60, 0.005, 1.0, 0.72)
    x, v, img = b.get_state()
    st = case.oracle_state()
    O.integrate(case.model, st, 60, 0.005, 1.0, 0.72, seed=42)
    assert np.abs(_unwrapped(x, img, case.cfg.box) - _unwrapped(st.x, st.img, case.cfg.box)).max() < 1e-10
    with pytest.raises(espp.EsppError) as e:
        b.set_cell_subdivision(4)
    assert e.value.code == espp.ESPP_ERR_ARG


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_third_cells_keep_the_neighbour_sets(prec):
    # cells of (rc + skin) / 3, rows trimmed to the list sphere: the same
    # pairs as brute force (FP32: outside a 1e-6 band at the list radius)
    case = lj_case()
    s = case.system(prec, build=False)
    s.set_cell_subdivision(3)
    s.build_neighbors(case.rc_list, case.skin)
    row, cols = s.get_neighbors()
    c = case.cfg
    rl = case.rc_list + case.skin
    orow, ocols = O.neighbors(c.box, c.x, rl, method="brute")
    band = 1e-6 if prec == FP32 else 0.0
    for i in range(c.n):
        got = set(cols[row[i]:row[i + 1]].tolist())
        exp = set(ocols[orow[i]:orow[i + 1]].tolist())
        for j in got ^ exp:
            d = c.x[i] - c.x[j]
            d -= c.box * np.round(d / c.box)
            assert abs(np.linalg.norm(d) - rl) <= band, (i, j, np.linalg.norm(d))
    # the list-free mode takes whole or half cells only
    with pytest.raises(espp.EsppError) as e:
        s.set_force_method(espp.ESPP_FORCES_CELLS)
    assert e.value.code == espp.ESPP_ERR_ARG
    s.set_cell_subdivision(0)
    s.set_force_method(espp.ESPP_FORCES_CELLS)
    with pytest.raises(espp.EsppError) as e:
        s.set_cell_subdivision(3)
    assert e.value.code == espp.ESPP_ERR_ARG
    s.close()


def _store_pair(case, w, push, prec=FP32, le=False, excl=False):
    s = case.system(prec, build=False)
    s.set_cell_subdivision(w)
    s.set_list_store(push)
    if excl:
        s.set_exclude_bonded(True)
    if le:
        s.set_lees_edwards(True, 0.5, 0.25)
    s.build_neighbors(case.rc_list, case.skin)
    return s


@pytest.mark.parametrize("w", [1, 3])
@pytest.mark.parametrize("variant", ["plain", "lees_edwards", "exclusions"])
@pytest.mark.parametrize("case", [kg_case(), lj_case()], ids=lambda c: c.name)
def test_pushed_list_store_builds_the_same_lists(case, w, variant):
    # the two ways of storing hits in the build give the same lists in the
    # same order: FP32 force sums and trajectories (with rebuilds) bit for bit
    if variant != "plain" and case.name != kg_case().name:
        pytest.skip("sheared and excluded builds on the bonded melt")
    kw = dict(le=variant == "lees_edwards", excl=variant == "exclusions")
    a = _store_pair(case, w, espp.ESPP_LIST_STORE_PLACE, **kw)
    b = _store_pair(case, w, espp.ESPP_LIST_STORE_PUSH, **kw)
    ra, ca = a.get_neighbors()
    rb, cb = b.get_neighbors()
    assert np.array_equal(ra, rb) and np.array_equal(ca, cb)
    assert np.array_equal(a.compute_forces(), b.compute_forces())
    a.integrate(60, 0.005, 1.0, 1.0)
    b.integrate(60, 0.005, 1.0, 1.0)
    assert a.n_rebuilds == b.n_rebuilds and a.n_rebuilds >= 2
    for qa, qb in zip(a.get_state(), b.get_state()):
        assert np.array_equal(qa, qb)
    with pytest.raises(espp.EsppError) as e:
        b.set_list_store(2)
    assert e.value.code == espp.ESPP_ERR_ARG
    a.close()
    b.close()


def test_cell_subdivision_in_batches():
    # replicas of different sizes, each with its own sub-cell grid
    cases_ = [kg_case(), kg_case(4, 30, seed=3, jitter=0.08), kg_case(7, 23, seed=5, jitter=0.1)]
    reps = [dict(box=c.cfg.box, n=c.cfg.n, types=c.cfg.types, bonds=c.cfg.bonds, seed=42 + k)
            for k, c in enumerate(cases_)]
    b = espp.System(replicas=reps, precision=FP64)
    b.set_wca()
    b.set_fene()
    b.set_state(np.concatenate([c.cfg.x for c in cases_]), np.concatenate([c.v for c in cases_]),
                np.concatenate([c.cfg.img for c in cases_]))
    b.set_cell_subdivision(2)
    b.build_neighbors(WCA_RC, 0.4)
    f3 = b.compute_forces()
    b.set_cell_subdivision(1)
    f1 = b.compute_forces()
    assert rel_rms(f3, f1) <= 1e-13
    b.set_cell_subdivision(3)
    assert rel_rms(b.compute_forces(), f1) <= 1e-13
    off = 0
    for c in cases_:
        fo, _ = O.forces(c.model, c.cfg.box, c.cfg.x, c.cfg.types, c.cfg.bonds)
        assert rel_rms(f3[off:off + c.cfg.n], fo) <= 1e-12
        off += c.cfg.n


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_direct_launches_equal_graphs(prec):
    # the same kernels launched one by one (no CUDA graphs), or in graphs of
    # other step counts (a chunk limit of 5: graphs of 5, 4, 2 and 1 steps),
    # give the same bits, whatever the split of the run into calls
    case = kg_case()
    a = case.system(prec, seed=8)
    a.integrate(150, 0.005, 1.0, 1.0)
    xa, va, ia = a.get_state()
    for chunk, calls in ((0, (150,)), (5, (150,)), (64, (1, 2, 20, 3, 124)), (7, (33, 117))):
        b = case.system(prec, seed=8)
        b.set_graph_chunk(chunk)
        for k in calls:
            b.integrate(k, 0.005, 1.0, 1.0)
        xb, vb, ib = b.get_state()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ia, ib), (chunk, calls)
        assert a.n_rebuilds == b.n_rebuilds
        b.close()


@pytest.mark.parametrize("every", [0, 7, 40])
def test_resort_interval_does_not_change_fp64_physics(every):
    case = lj_case()
    s = case.system(FP64, seed=2)
    s.set_resort_interval(every)
    s.integrate(120, 0.005, 1.0, 0.72)
    x, v, img = s.get_state()
    st = case.oracle_state()
    O.integrate(case.model, st, 120, 0.005, 1.0, 0.72, seed=2)
    assert np.abs(_unwrapped(x, img, case.cfg.box) - _unwrapped(st.x, st.img, case.cfg.box)).max() < 1e-10


def test_broken_bond_is_reported():
    case = kg_case(4, 50)
    c = case.cfg
    c.x = c.x.copy()
    c.x[5] = np.mod(c.x[4] + np.array([1.6, 0.0, 0.0]), c.box)
    c.img = np.zeros_like(c.img)
    s = case.system(FP32)
    with pytest.raises(espp.EsppError) as e:
        s.compute_forces()
    assert e.value.code == espp.ESPP_ERR_BOND_BROKEN


def test_degenerate_inputs_are_rejected():
    # no particles, more than the 2^25 slots a handle can address, a bond to
    # itself, a zero box edge: ESPP_ERR_ARG before anything is allocated
    box = np.array([10.0, 10.0, 10.0])
    for n in (0, 1 << 25):
        with pytest.raises(espp.EsppError) as e:
            espp.System(box, n, precision=FP32)
        assert e.value.code == espp.ESPP_ERR_ARG
    with pytest.raises(espp.EsppError) as e:
        espp.System(box, 4, bonds=np.array([[1, 1]]), precision=FP32)
    assert e.value.code == espp.ESPP_ERR_ARG
    with pytest.raises(espp.EsppError) as e:
        espp.System(np.array([10.0, 0.0, 10.0]), 4, precision=FP32)
    assert e.value.code == espp.ESPP_ERR_ARG


def test_zero_steps_and_calls_before_setup():
    case = kg_case()
    s = espp.System(case.cfg.box, case.cfg.n, case.cfg.types, case.cfg.bonds, precision=FP32)
    s.set_wca()
    s.set_fene()
    with pytest.raises(espp.EsppError) as e:   # no state yet
        s.compute_forces()
    assert e.value.code == espp.ESPP_ERR_STATE
    s.set_state(case.cfg.x, case.v, case.cfg.img)
    with pytest.raises(espp.EsppError) as e:   # no list yet
        s.integrate(1, 0.005, 1.0, 1.0)
    assert e.value.code == espp.ESPP_ERR_STATE
    s.build_neighbors(WCA_RC, 0.4)
    x0, v0, i0 = s.get_state()
    s.integrate(0, 0.005, 1.0, 1.0)            # zero steps: nothing moves
    x1, v1, i1 = s.get_state()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1) and s.step == 0
    with pytest.raises(espp.EsppError) as e:   # a non-positive time step
        s.integrate(5, 0.0, 1.0, 1.0)
    assert e.value.code == espp.ESPP_ERR_ARG


def test_box_too_small_is_reported():
    s = espp.System(np.array([4.0, 4.0, 4.0]), 8, precision=FP32)
    s.set_wca()
    s.set_state(np.random.default_rng(0).random((8, 3)) * 4.0)
    with pytest.raises(espp.EsppError) as e:
        s.build_neighbors(WCA_RC, 0.4)
    assert e.value.code == espp.ESPP_ERR_BOX_TOO_SMALL


def test_cutoff_beyond_list_is_rejected():
    case = lj_case()
    s = case.system(FP32, build=False)
    with pytest.raises(espp.EsppError) as e:
        s.build_neighbors(2.0, 0.3)
    assert e.value.code == espp.ESPP_ERR_ARG


def test_refused_settings_leave_the_handle_unchanged():
    case = kg_case()
    s = case.system(FP32, seed=3)
    ref = case.system(FP32, seed=3)
    bad_bits = espp.to_bf16_bits(np.zeros(espp.MLP_NPARAMS))
    bad_bits[7] = 0x7FC0  # a BF16 NaN
    refusals = [
        lambda: s.set_lj(1.0, 1.0, float("inf")),
        lambda: s.set_wca(float("nan"), 1.0),
        lambda: s.set_fene(float("inf"), 1.5),
        lambda: s.set_mass(0, float("inf")),
        lambda: s.set_mlp(2.5, bad_bits),
        lambda: s.build_neighbors(0.5, 0.4),  # below the WCA cutoff
        lambda: s.integrate(5, 0.005, float("inf"), 1.0),
        lambda: s.integrate(5, 0.005, 1.0, float("nan")),
    ]
    for call in refusals:
        with pytest.raises(espp.EsppError) as e:
            call()
        assert e.value.code == espp.ESPP_ERR_ARG
    s.integrate(40, 0.005, 1.0, 1.0)
    ref.integrate(40, 0.005, 1.0, 1.0)
    xs, vs, is_ = s.get_state()
    xr, vr, ir = ref.get_state()
    assert np.array_equal(xs, xr) and np.array_equal(vs, vr) and np.array_equal(is_, ir)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_single_free_particle(prec):
    box = np.array([5.0, 6.0, 7.0])
    s = espp.System(box, 1, precision=prec, seed=9)
    s.set_wca()
    s.set_state(np.array([[4.9, 0.05, 3.5]]), np.array([[3.0, -2.0, 1.0]]))
    s.build_neighbors(WCA_RC, 0.4)
    assert np.array_equal(s.compute_forces(), np.zeros((1, 3)))
    s.integrate(100, 0.005, 1.0, 1.0)
    x, v, img = s.get_state()
    st = O.State(box, np.array([[4.9, 0.05, 3.5]]), np.array([[3.0, -2.0, 1.0]]))
    O.integrate(O.Model(1, KG_PAIR), st, 100, 0.005, 1.0, 1.0, seed=9)
    tol = 1e-12 if prec == FP64 else 1e-4
    assert np.abs(_unwrapped(x, img, box) - _unwrapped(st.x, st.img, box)).max() < tol
    assert np.abs(v - st.v).max() < tol


def test_ragged_tiles_and_types():
    # 257 particles: two full tiles plus a tail of one
    c = I.random_positions(257, (9.0, 9.5, 10.0), seed=4)
    c.types = (np.arange(257) % 3).astype(np.int32)
    pair = {(0, 0): ("wca", 1.0, 1.0), (0, 1): ("lj", 0.5, 1.0, 2.0, True),
            (1, 1): ("lj", 1.0, 0.8, 1.8, False), (0, 2): ("wca", 1.0, 0.9),
            (1, 2): ("lj_capped", 1.0, 1.0, 2.0, True, 0.85), (2, 2): ("lj", 0.3, 1.2, 2.0, True)}
    case = Case("ragged", c, pair, None, 2.0, 0.25, np.zeros((257, 3)))
    for prec in (FP32, FP64):
        s = case.system(prec)
        f = s.compute_forces()
        fo, _ = O.forces(case.model, c.box, c.x, c.types, c.bonds)
        assert rel_rms(f, fo) <= (1e-5 if prec == FP32 else 1e-12)


def test_capped_pushoff_runs_like_the_oracle():
    case = capped_case(800, 10.0)
    s = case.system(FP64, seed=4)
    s.integrate(200, 1e-4, 1.0, 1.0)
    x, v, img = s.get_state()
    st = case.oracle_state()
    O.integrate(case.model, st, 200, 1e-4, 1.0, 1.0, seed=4)
    assert np.abs(_unwrapped(x, img, case.cfg.box) - _unwrapped(st.x, st.img, case.cfg.box)).max() < 1e-9


def _tab_case():
    """KG chains with the WCA pair and the FENE bond given as tables (the
    table values are inputs: the closed forms sampled on the grid)."""
    c = I.kg_lattice(20, 50, seed=21, jitter=0.08)
    n = 2048
    r = np.linspace(0.0, WCA_RC, n)
    rs = np.maximum(r, 0.6)
    u = 4 * (rs ** -12 - rs ** -6) + 1.0
    f = 24 * (2 * rs ** -13 - rs ** -7)
    rb = np.linspace(0.0, 1.49, 1024)
    ub = -0.5 * 30.0 * 2.25 * np.log(1 - rb ** 2 / 2.25)
    fb = -30.0 * rb / (1 - rb ** 2 / 2.25)
    O.set_table(3, WCA_RC, u, f)
    O.set_table(4, 1.49, ub, fb)
    model = O.Model(1, {(0, 0): ("table", 3, WCA_RC)}, ("table", 4))
    return c, (WCA_RC, u, f), (1.49, ub, fb), model


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_tabulated_pair_and_bond_match_oracle(prec):
    c, tp, tb, model = _tab_case()
    v = I.maxwell_velocities(c.n, 1.0, seed=3)
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=prec, seed=6)
    s.set_table_pair(*tp)
    s.set_table_bond(*tb)
    s.set_state(c.x, v, c.img)
    s.build_neighbors(WCA_RC, 0.4)
    f = s.compute_forces()
    fo, en = O.forces(model, c.box, c.x, c.types, c.bonds)
    assert rel_rms(f, fo) <= FORCE_TOL[prec]
    o = s.observables()
    oo = O.observables(model, O.State(c.box, c.x, v, c.img, c.types, c.bonds))
    tol = 1e-12 if prec == FP64 else 2e-6
    for k in ("pe_pair", "pe_bond", "virial"):
        assert abs(o[k] - oo[k]) <= tol * max(1.0, abs(oo[k])), k
    if prec == FP64:
        s.integrate(60, 0.005, 1.0, 1.0)
        x1, v1, i1 = s.get_state()
        st = O.State(c.box, c.x, v, c.img, c.types, c.bonds)
        O.integrate(model, st, 60, 0.005, 1.0, 1.0, seed=6)
        assert np.abs(_unwrapped(x1, i1, c.box) - _unwrapped(st.x, st.img, c.box)).max() < 1e-10


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_checkpoint_resume_is_bit_exact(prec, tmp_path):
    case = kg_case()
    a = case.system(prec, seed=17)
    a.integrate(137, 0.005, 1.0, 1.0)
    path = str(tmp_path / "state.ckpt")
    a.checkpoint_save(path)
    a.integrate(300, 0.005, 1.0, 1.0)
    xa, va, ia = a.get_state()
    c = case.cfg
    b = espp.System(c.box, c.n, c.types, c.bonds, precision=prec, seed=999)
    b.set_wca()
    b.set_fene()
    b.build_neighbors(WCA_RC, 0.4)
    b.checkpoint_load(path)
    assert b.step == 137
    b.integrate(300, 0.005, 1.0, 1.0)
    xb, vb, ib = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ia, ib)


def test_checkpoint_rejects_other_handles(tmp_path):
    case = kg_case()
    a = case.system(FP32)
    path = str(tmp_path / "s.ckpt")
    a.checkpoint_save(path)
    other = lj_case()
    b = other.system(FP32)
    with pytest.raises(espp.EsppError):
        b.checkpoint_load(path)
    c64 = case.system(FP64)
    with pytest.raises(espp.EsppError):
        c64.checkpoint_load(path)


def test_failed_checkpoint_load_leaves_the_handle_unchanged(tmp_path):
    # a truncated file of a run with another seed: the load fails after the
    # per-replica records (seeds included) have been read; the handle must
    # keep its own seed and state
    case = kg_case()
    a = case.system(FP32, seed=17)
    a.integrate(20, 0.005, 1.0, 1.0)
    full = tmp_path / "full.ckpt"
    a.checkpoint_save(str(full))
    data = full.read_bytes()
    cut = tmp_path / "cut.ckpt"
    cut.write_bytes(data[: len(data) // 2])
    b = case.system(FP32, seed=5)
    ref = case.system(FP32, seed=5)
    with pytest.raises(espp.EsppError):
        b.checkpoint_load(str(cut))
    b.integrate(50, 0.005, 1.0, 1.0)
    ref.integrate(50, 0.005, 1.0, 1.0)
    xb, vb, ib = b.get_state()
    xr, vr, ir = ref.get_state()
    assert b.step == ref.step == 50
    assert np.array_equal(xb, xr) and np.array_equal(vb, vr) and np.array_equal(ib, ir)


# ---------------------------------------------------------------------------
# full sizes, sampled against the oracle one particle at a time
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [FP32, FP64])
def test_full_size_kg_1m_sampled_forces(prec):
    c = I.kg_lattice(1000, 1000, density=0.85, seed=42, jitter=0.05)
    case = Case("kg1m", c, KG_PAIR, KG_BOND, WCA_RC, 0.4)
    s = case.system(prec)
    f = s.compute_forces()
    sel = np.random.default_rng(0).choice(c.n, 4000, replace=False)
    fo = O.forces_subset(case.model, c.box, c.x, c.types, c.bonds, sel)
    assert rel_rms(f[sel], fo) <= FORCE_TOL[prec]
    # property at any size: Newton's third law
    assert np.abs(f.sum(axis=0)).max() <= (1e-3 if prec == FP32 else 1e-8) * np.abs(f).sum() / c.n
    s.close()


def _bench_melt_1m():
    """The KG melt as the benchmark runs it: 1000 random-walk chains of 1000
    beads (seed 42), the capped push-off, then plain WCA at dt 0.002 and
    0.005 (4400 steps), FP32."""
    c = I.kg_random_walk(1000, 1000, density=0.85, seed=42, bond=0.97)
    v = I.maxwell_velocities(c.n, 1.0, seed=42)
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=FP32, seed=42)
    s.set_fene(30.0, 1.5)
    s.set_lj_capped(1.0, 1.0, WCA_RC, 1.05)
    s.set_state(c.x, v, c.img)
    s.build_neighbors(WCA_RC, 0.4)
    for cap in (1.05, 1.0, 0.95, 0.9, 0.85, 0.8):
        s.set_lj_capped(1.0, 1.0, WCA_RC, cap)
        s.integrate(400, 1e-3, 1.0, 1.0)
    s.set_wca(1.0, 1.0)
    s.integrate(1000, 0.002, 1.0, 1.0)
    s.integrate(1000, 0.005, 1.0, 1.0)
    return s, c


def test_full_size_kg_1m_in_the_benchmark_state():
    # the timed workload itself, after the GPU has integrated it: rebuilds
    # inside the step graphs, list growth and a Hilbert resort (every 500
    # steps: the run crosses step 4500) have all happened at 1M beads; then
    # forces and neighbour sets of sampled particles against the oracle on
    # the stored positions
    s, c = _bench_melt_1m()
    rb0 = s.n_rebuilds
    s.integrate(300, 0.005, 1.0, 1.0)
    assert s.step == 4700 and s.n_rebuilds - rb0 >= 10
    x, _, img = s.get_state()
    # image counters: every bond of the unwrapped chains (no minimum image)
    # is shorter than R0 after hundreds of wraps at list builds
    u = x + img * c.box
    b = np.asarray(c.bonds)
    blen = np.sqrt(((u[b[:, 0]] - u[b[:, 1]]) ** 2).sum(axis=1))
    assert blen.max() < 1.5, (blen.max(), int((blen >= 1.5).sum()))
    f = s.compute_forces()
    sel = np.random.default_rng(3).choice(c.n, 4000, replace=False)
    model = O.Model(1, KG_PAIR, KG_BOND)
    fo = O.forces_subset(model, c.box, x, c.types, c.bonds, sel)
    assert rel_rms(f[sel], fo) <= FORCE_TOL[FP32], rel_rms(f[sel], fo)
    # neighbour sets of a list built now, for the stored positions, against
    # the oracle's cell search, exact outside the 1e-6 sigma band at rc + skin
    s.build_neighbors(WCA_RC, 0.4)
    row, cols = s.get_neighbors()
    orow, ocols = O.neighbors(c.box, x, WCA_RC + 0.4, method="cells")
    rl = WCA_RC + 0.4
    for i in sel[:1000]:
        got = set(cols[row[i]:row[i + 1]].tolist())
        exp = set(ocols[orow[i]:orow[i + 1]].tolist())
        for j in got ^ exp:
            d = x[i] - x[j]
            d -= c.box * np.round(d / c.box)
            assert abs(np.sqrt(d @ d) - rl) < 1e-6, (i, j)
    s.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_wrap_just_below_zero_keeps_the_unwrapped_position(prec):
    # a particle drifts to just below 0 by less than half an ulp of L in the
    # stored precision; the wrap at the next list build must keep it in its
    # own image (x + img L continuous), as the oracle does
    L = 10.0
    eps = 1e-7 if prec == FP32 else 1e-17
    box = np.array([L, L, L])
    s = espp.System(box, 2, None, None, precision=prec, seed=1)
    s.set_lj(1.0, 1.0, 2.5, True)
    x = np.array([[eps / 10, 5.0, 5.0], [5.0, 5.0, 5.0]])
    v = np.array([[-(eps + eps / 10) / 0.005, 0.0, 0.0], [0.0, 0.0, 0.0]])
    s.set_state(x, v)
    s.build_neighbors(2.5, 0.3)
    s.integrate(1, 0.005, 0.0, 0.0)
    s.build_neighbors(2.5, 0.3)  # wraps the stored positions
    xw, _, img = s.get_state()
    assert 0.0 <= xw[0, 0] < L
    assert abs(xw[0, 0] + img[0, 0] * L) < 1e-5, (xw[0, 0], img[0, 0])
    s.close()


def test_unwrapped_bonds_stay_short_over_a_long_run():
    # many wraps of a melt's chains at list builds: the unwrapped chains keep
    # every bond below R0
    c = I.kg_lattice(200, 100, density=0.85, seed=7, jitter=0.05)
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=FP32, seed=7)
    s.set_fene(30.0, 1.5)
    s.set_wca(1.0, 1.0)
    s.set_state(c.x, I.maxwell_velocities(c.n, 1.0, seed=7), c.img)
    s.build_neighbors(WCA_RC, 0.4)
    s.integrate(8000, 0.005, 1.0, 1.0)
    x, _, img = s.get_state()
    u = x + img * c.box
    b = np.asarray(c.bonds)
    assert np.sqrt(((u[b[:, 0]] - u[b[:, 1]]) ** 2).sum(axis=1)).max() < 1.5
    s.close()


def test_full_size_lj_4m_sampled_forces():
    case = lj_case((128, 128, 64), seed=2, noise=0.05)
    c = case.cfg
    s = case.system(FP32)
    f = s.compute_forces()
    sel = np.random.default_rng(1).choice(c.n, 4000, replace=False)
    fo = O.forces_subset(case.model, c.box, c.x, c.types, c.bonds, sel)
    assert rel_rms(f[sel], fo) <= 1e-5
    s.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_rdf_from_list_equals_all_pairs(prec):
    case = lj_case((6, 6, 6))
    s = case.system(prec)
    a = s.rdf_counts(2.5, 50)  # within rc + skin: from the Verlet list
    b = s.rdf_counts(4.5, 90)[:50]  # beyond it: all pairs, the same bins below 2.5
    if prec == FP64:
        assert np.array_equal(a, b)
    else:
        assert np.abs(a - b).max() <= 2 and abs(int(a.sum()) - int(b.sum())) <= 2


def test_cg_map_matches_numpy_mapping():
    import torch
    case = kg_case(20, 48, seed=3)
    s = case.system(FP32)
    s.integrate(50, 0.005, 1.0, 1.0)
    x, v, img = s.get_state()
    f = s.compute_forces()
    xs = torch.zeros((case.cfg.n // 4, 3), dtype=torch.float64, device="cuda")
    fs = torch.zeros_like(xs)
    s.cg_map(4, xs, fs)
    box = case.cfg.box
    u = (x + img * box).reshape(-1, 4, 3).mean(axis=1)
    u = np.mod(u, box)
    assert np.abs(xs.cpu().numpy() - u).max() < 1e-9
    assert np.abs(fs.cpu().numpy() - f.reshape(-1, 4, 3).sum(axis=1)).max() < 1e-9


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_non_finite_input_and_runaway_are_reported(prec):
    case = kg_case()
    c = case.cfg
    s = case.system(prec)
    # a non-finite input is refused and leaves no state behind
    for bad_x, bad_v in ((True, False), (False, True)):
        x, v = c.x.copy(), case.v.copy()
        if bad_x:
            x[5, 1] = np.nan
        if bad_v:
            v[7, 2] = np.inf
        with pytest.raises(espp.EsppError) as e:
            s.set_state(x, v, c.img)
        assert e.value.code == espp.ESPP_ERR_ARG
        with pytest.raises(espp.EsppError) as e:
            s.integrate(1, 0.005, 1.0, 1.0)
        assert e.value.code == espp.ESPP_ERR_STATE
    # a finite but runaway velocity carries a particle beyond any box in one
    # step: the step kernels stop and the call reports it
    v = case.v.copy()
    v[11] = [1e35, 0.0, 0.0]
    s.set_state(c.x, v, c.img)
    s.build_neighbors(case.rc_list, case.skin)
    with pytest.raises(espp.EsppError) as e:
        s.integrate(5, 0.005, 1.0, 1.0)
    assert e.value.code == espp.ESPP_ERR_NONFINITE
    # a fresh state clears the condition
    s.set_state(c.x, case.v, c.img)
    s.integrate(5, 0.005, 1.0, 1.0)
    assert s.error_word == 0
    s.close()


def _long_run_stats(step_fn, obs_fn, rdf_fn, nsamples=100, every=100):
    T, B, G = [], [], []
    for _ in range(nsamples):
        step_fn(every)
        o = obs_fn()
        T.append(o["temperature"])
        B.append(o["mean_bond"])
        G.append(rdf_fn())
    return np.array(T), np.array(B), np.array(G, dtype=float)


def _block_mean(x, nb=10):
    m = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
    return m.mean(), m.std(ddof=1) / np.sqrt(nb)


def test_long_run_statistics_match_oracle():
    # FP32 on the GPU and the FP64 oracle (different noise streams) sample the
    # same ensemble: temperature and mean bond length within 4 combined block
    # errors, g(r) within 4x the seed-to-seed L2 (0.0038 from two oracle runs)
    case = kg_case()
    c = case.cfg
    s = case.system(FP32, seed=101)
    s.integrate(2000, 0.005, 1.0, 1.0)
    g_run = _long_run_stats(lambda k: s.integrate(k, 0.005, 1.0, 1.0), s.observables,
                            lambda: s.rdf_counts(2.5, 25))
    st = case.oracle_state()
    O.integrate(case.model, st, 2000, 0.005, 1.0, 1.0, seed=202)

    def ostep(k):
        O.integrate(case.model, st, k, 0.005, 1.0, 1.0, seed=202)

    o_run = _long_run_stats(ostep, lambda: O.observables(case.model, st), lambda: O.rdf_counts(c.box, st.x, 2.5, 25))
    for k in range(2):
        mg, sg = _block_mean(g_run[k])
        mo, so = _block_mean(o_run[k])
        assert abs(mg - mo) <= 4 * np.hypot(sg, so) + 1e-4, (k, mg, mo, sg, so)
    gg, go = g_run[2].mean(axis=0), o_run[2].mean(axis=0)
    assert np.sqrt(((gg - go) ** 2).sum() / (go ** 2).sum()) < 0.015
    # (Rg^2 is not compared: 50-bead chains from a lattice start relax over
    # far more than these 60 time units; two oracle seeds differ by 5 block
    # errors)
    s.close()


@pytest.mark.parametrize("thermo", ["langevin", "dpd"])
def test_two_masses_match_oracle(thermo):
    # a particle type of mass 2.5 next to mass 1: friction, noise amplitude,
    # kicks and kinetic energy all carry the mass
    case = two_type_case()
    c = case.cfg
    s = case.system(FP64, seed=27)
    s.set_mass(1, 2.5)
    if thermo == "dpd":
        s.set_thermostat(espp.ESPP_THERMO_DPD, 1.2)
        O.set_dpd(True, 1.2)
    try:
        s.integrate(120, 0.005, 1.3, 1.0)
        x, v, img = s.get_state()
        model = O.Model(2, case.pair, None, masses=[1.0, 2.5])
        st = case.oracle_state()
        O.integrate(model, st, 120, 0.005, 1.3, 1.0, seed=27)
    finally:
        O.set_dpd(False)
    box = c.box
    assert np.abs(_unwrapped(x, img, box) - _unwrapped(st.x, st.img, box)).max() < 1e-10
    assert np.abs(v - st.v).max() < 1e-9
    o, oo = s.observables(), O.observables(model, st)
    for k in ("ke", "temperature", "px", "pressure"):
        assert abs(o[k] - oo[k]) <= 1e-9 * max(1.0, abs(oo[k])), (k, o[k], oo[k])
    s.close()


# ---------------------------------------------------------------------------
# launch shapes of the step kernel (autotuned): the same trajectory bit for bit
# ---------------------------------------------------------------------------
def test_every_step_shape_gives_the_same_trajectory():
    # 1000 + 1288 + 333 beads in three replicas: tile counts 8 + 11 + 3 = 22, so
    # blocks of 2, 3, 4 and 5 tiles end on a partial block and mix replicas
    sizes = [(20, 50, 11), (23, 56, 12), (9, 37, 13)]
    cases_ = [kg_case(nc, nb, seed=sd, jitter=0.06) for nc, nb, sd in sizes]
    reps = [dict(box=c.cfg.box, n=c.cfg.n, types=c.cfg.types, bonds=c.cfg.bonds, seed=70 + k)
            for k, c in enumerate(cases_)]
    out = []
    for shape in range(espp.STEP_SHAPES):
        b = espp.System(replicas=reps, precision=FP32)
        b.set_wca()
        b.set_fene()
        b.set_state(np.concatenate([c.cfg.x for c in cases_]), np.concatenate([c.v for c in cases_]),
                    np.concatenate([c.cfg.img for c in cases_]))
        b.build_neighbors(WCA_RC, 0.4)
        b.set_step_shape(shape)
        b.integrate(150, 0.005, 1.0, 1.0)
        out.append(b.get_state())
        b.close()
    for shape in range(1, espp.STEP_SHAPES):
        for a, c in zip(out[0], out[shape]):
            assert np.array_equal(a, c), shape


def test_step_shape_tuner_restores_the_state():
    case = kg_case()
    s = case.system(FP32, seed=8)
    ref = case.system(FP32, seed=8)
    shape_ms, resort_ms, (shape, resort) = s.tune_step_shape(20, 0.005, 1.0, 1.0)
    assert len(shape_ms) == espp.STEP_SHAPES and len(resort_ms) == 3
    assert all(np.isfinite(shape_ms)) and 0 <= shape < espp.STEP_SHAPES and resort in (250, 500, 1000)
    assert s.step == 0
    s.set_step_shape(0)
    s.integrate(50, 0.005, 1.0, 1.0)
    ref.integrate(50, 0.005, 1.0, 1.0)
    for a, b in zip(s.get_state(), ref.get_state()):
        assert np.array_equal(a, b)
    with pytest.raises(espp.EsppError):
        s.set_step_shape(espp.STEP_SHAPES)


def test_full_size_lj_4m_in_the_benchmark_state():
    # the 4M LJ fluid as the benchmark runs it: the force-path tuner (third
    # cells win there) and the step-shape tuner, then steps with rebuilds;
    # sampled forces and neighbour sets against the oracle on the stored state
    case = lj_case((128, 128, 64), seed=2, noise=0.05)
    c = case.cfg
    s = case.system(FP32)
    s.integrate(100, 0.005, 1.0, 0.72)
    s.tune_force_method(50, 0.005, 1.0, 0.72)
    s.tune_step_shape(50, 0.005, 1.0, 0.72)
    rb0 = s.n_rebuilds
    s.integrate(300, 0.005, 1.0, 0.72)
    assert s.n_rebuilds - rb0 >= 10
    x, _, _ = s.get_state()
    f = s.compute_forces()
    sel = np.random.default_rng(5).choice(c.n, 3000, replace=False)
    fo = O.forces_subset(case.model, c.box, x, c.types, c.bonds, sel)
    assert rel_rms(f[sel], fo) <= 1e-5, rel_rms(f[sel], fo)
    s.build_neighbors(case.rc_list, case.skin)
    row, cols = s.get_neighbors()
    rl = case.rc_list + case.skin
    orow, ocols = O.neighbors(c.box, x, rl, method="cells")
    for i in sel[:300]:
        got = set(cols[row[i]:row[i + 1]].tolist())
        exp = set(ocols[orow[i]:orow[i + 1]].tolist())
        for j in got ^ exp:
            d = x[i] - x[j]
            d -= c.box * np.round(d / c.box)
            assert abs(np.sqrt(d @ d) - rl) < 1e-6, (i, j)
    s.close()


def test_full_size_batched_512_replicas_sampled_forces():
    # the 512 uneven replicas of the batched benchmark (11.6M beads, lattice
    # starts), tuned and stepped as the benchmark does; three replicas (the
    # smallest, the largest and one between) against the oracle
    sizes = I.replica_sizes(512, seed=42)
    cfgs = [I.kg_lattice(nc, nb, density=0.85, seed=42 + r, jitter=0.05) for r, (nc, nb) in enumerate(sizes)]
    reps = [dict(box=q.box, n=q.n, types=q.types, bonds=q.bonds, seed=42 + r) for r, q in enumerate(cfgs)]
    s = espp.System(replicas=reps, precision=FP32)
    s.set_wca()
    s.set_fene()
    s.set_state(np.concatenate([q.x for q in cfgs]), I.maxwell_velocities(s.n, 1.0, seed=7),
                np.concatenate([q.img for q in cfgs]))
    s.build_neighbors(WCA_RC, 0.4)
    s.integrate(100, 0.005, 1.0, 1.0)
    s.tune_force_method(50, 0.005, 1.0, 1.0)
    s.tune_step_shape(50, 0.005, 1.0, 1.0)
    s.integrate(200, 0.005, 1.0, 1.0)
    x, _, _ = s.get_state()
    f = s.compute_forces()
    off = np.concatenate([[0], np.cumsum([q.n for q in cfgs])])
    ns = np.array([q.n for q in cfgs])
    model = O.Model(1, KG_PAIR, KG_BOND)
    for r in (int(ns.argmin()), int(ns.argmax()), 255):
        q = cfgs[r]
        xr, fr = x[off[r]:off[r + 1]], f[off[r]:off[r + 1]]
        sel = np.random.default_rng(r).choice(q.n, min(q.n, 2000), replace=False)
        fo = O.forces_subset(model, q.box, xr, q.types, q.bonds, sel)
        assert rel_rms(fr[sel], fo) <= 1e-5, (r, rel_rms(fr[sel], fo))
    s.close()


def test_largest_handle_2_to_the_25_minus_1_particles():
    # the most particles a handle addresses (2^25 - 1 = 31 x 601 x 1801): the
    # list's padding slot is then the largest index an entry can hold; forces
    # of sampled particles against the oracle, then steps with rebuilds
    n_chains, n_beads = 31 * 601, 1801
    c = I.kg_lattice(n_chains, n_beads, density=0.85, seed=13, jitter=0.05)
    assert c.n == (1 << 25) - 1
    case = Case("kg_max", c, KG_PAIR, KG_BOND, WCA_RC, 0.4)
    s = case.system(FP32)
    f = s.compute_forces()
    sel = np.random.default_rng(13).choice(c.n, 1000, replace=False)
    fo = O.forces_subset(case.model, c.box, c.x, c.types, c.bonds, sel)
    assert rel_rms(f[sel], fo) <= FORCE_TOL[FP32], rel_rms(f[sel], fo)
    s.integrate(20, 0.002, 1.0, 1.0)
    assert s.error_word == 0 and s.step == 20
    s.close()
