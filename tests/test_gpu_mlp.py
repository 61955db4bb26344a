"""The learned CG pair potential on the tensor cores against the oracle's
double-precision evaluation of the same network (BF16 weights upcast).

Tolerances.  FP32 handles run the network on the tensor cores: the radial
features and the first-layer activations are rounded to BF16 (unit roundoff
2^-8, so about 2.3e-3 relative RMS per rounding) before FP32-accumulated
GEMMs.  Two such roundings in sequence, each spread over 32 or 64 terms of
mixed sign, give a per-pair error in u and du/dr of a few 1e-3 of the
function's scale; the per-pair scan is gated at 1e-2 of that scale
(MLP_PAIR_TOL).  Summed forces add ~20 such pair errors of both signs per
site, so their relative RMS error stays at the per-pair level: gated at
MLP_SUM_TOL.  FP64 handles evaluate the same network in double and are gated
at 1e-12 like every other FP64 path."""
import numpy as np
import pytest

import oracle as O
from paper_2608_14911_gb300 import espp, inputs as I

from _systems import rel_rms

pytestmark = pytest.mark.gpu
RC = 3.5
SKIN = 0.5
MLP_PAIR_TOL = 1e-2   # per pair, relative to max |u| and max |du/dr| over the scan
MLP_SUM_TOL = 1e-2    # summed forces, relative RMS (FP32 handle, BF16 tensor cores)
MLP_E_TOL = 5e-3      # pair energy sum, relative (FP32 handle)
FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _weights(seed=0):
    g = np.random.default_rng(seed)
    w = np.concatenate([
        g.normal(0, 1.0 / np.sqrt(32), 64 * 32), g.normal(0, 0.1, 64),
        g.normal(0, 1.0 / np.sqrt(64), 64 * 64), g.normal(0, 0.1, 64),
        g.normal(0, 0.5 / np.sqrt(64), 64), [0.05]])
    bits = espp.to_bf16_bits(w)
    return bits, espp.bf16_bits_to_float(bits)


def _cg_system(nchains=60, nbeads=50, seed=3):
    """CG chains at the site density of the 4:1 mapped melt (0.2125)."""
    return I.kg_lattice(nchains, nbeads, density=0.2125, seed=seed, jitter=0.3)


def _bond_table():
    rb = np.linspace(0.0, 4.0, 801)
    return 4.0, 5.0 * (rb - 2.0) ** 2, -10.0 * (rb - 2.0)


@pytest.mark.parametrize("prec", [espp.ESPP_FP32, espp.ESPP_FP64])
def test_mlp_forces_and_energy_match_oracle(prec):
    c = _cg_system()
    bits, wd = _weights(1)
    rmax, ub, fb = _bond_table()
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=prec, seed=5)
    s.set_mlp(RC, bits)
    s.set_table_bond(rmax, ub, fb)
    s.set_exclude_bonded(True)
    s.set_state(c.x, None, c.img)
    s.build_neighbors(RC, SKIN)
    f = s.compute_forces()
    o = s.observables()
    O.set_mlp(wd, RC)
    O.set_table(7, rmax, ub, fb)
    O.set_exclude_bonded(True)
    try:
        model = O.Model(1, {(0, 0): ("mlp", RC)}, ("table", 7))
        fo, en = O.forces(model, c.box, c.x, c.types, c.bonds)
    finally:
        O.set_exclude_bonded(False)
    fp64 = prec == espp.ESPP_FP64
    assert rel_rms(f, fo) <= (FP64_TOL if fp64 else MLP_SUM_TOL), rel_rms(f, fo)
    assert abs(o["pe_pair"] - en[0]) <= (FP64_TOL if fp64 else MLP_E_TOL) * abs(en[0]), (o["pe_pair"], en[0])
    assert abs(o["pe_bond"] - en[1]) <= (FP64_TOL if fp64 else 1e-5) * abs(en[1])
    if fp64:
        assert abs(o["virial"] - en[2]) <= FP64_TOL * abs(en[2])
    # each pair is evaluated from both ends with identical arithmetic
    assert np.abs(f.sum(axis=0)).max() <= 1e-4 * np.abs(f).sum()


@pytest.mark.parametrize("prec", [espp.ESPP_FP32, espp.ESPP_FP64])
def test_mlp_single_pair_scan_matches_oracle(prec):
    # u(r) and du/dr of one pair, element by element, over (0, rc): a dimer
    # in a large box, its energy from the observables and -du/dr from the
    # force on the particle at larger x
    bits, wd = _weights(6)
    O.set_mlp(wd, RC)
    box = np.array([20.0, 20.0, 20.0])
    s = espp.System(box, 2, None, None, precision=prec, seed=1)
    s.set_mlp(RC, bits)
    rs = np.linspace(0.02, RC - 0.02, 171)
    u_dev, du_dev, u_orc, du_orc = [], [], [], []
    x = np.zeros((2, 3))
    for k, r in enumerate(rs):
        x[0] = (5.0, 5.0, 5.0)
        x[1] = (5.0 + r, 5.0, 5.0)
        s.set_state(x)
        if k == 0:
            s.build_neighbors(RC, SKIN)
        f = s.compute_forces()
        u_dev.append(s.observables()["pe_pair"])
        du_dev.append(-f[1, 0])
        # the stored separation (FP32 handles round the positions)
        xs, _, _ = s.get_state()
        u, du = O.mlp_pair(float(xs[1, 0] - xs[0, 0]))
        u_orc.append(u)
        du_orc.append(du)
    s.close()
    u_dev, du_dev, u_orc, du_orc = map(np.array, (u_dev, du_dev, u_orc, du_orc))
    eu = np.abs(u_dev - u_orc).max() / np.abs(u_orc).max()
    ed = np.abs(du_dev - du_orc).max() / np.abs(du_orc).max()
    tol = FP64_TOL if prec == espp.ESPP_FP64 else MLP_PAIR_TOL
    assert eu <= tol and ed <= tol, (eu, ed)


def test_mlp_dynamics_runs_and_thermalises():
    c = _cg_system(40, 50, seed=9)
    bits, _ = _weights(2)
    rmax, ub, fb = _bond_table()
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=espp.ESPP_FP32, seed=11)
    s.set_mlp(RC, bits)
    s.set_table_bond(rmax, ub, fb)
    s.set_exclude_bonded(True)
    s.set_state(c.x, I.maxwell_velocities(c.n, 1.0, seed=2), c.img)
    s.build_neighbors(RC, SKIN)
    s.integrate(400, 0.005, 1.0, 1.0)
    o = s.observables()
    assert 0.8 < o["temperature"] < 1.2
    assert np.isfinite(o["pe_pair"]) and o["error_word"] == 0


def _mlp_system(c, bits, prec=espp.ESPP_FP32, seed=5, replicas=None):
    rmax, ub, fb = _bond_table()
    if replicas is None:
        s = espp.System(c.box, c.n, c.types, c.bonds, precision=prec, seed=seed)
    else:
        s = espp.System(replicas=replicas, precision=prec)
    s.set_mlp(RC, bits)
    s.set_table_bond(rmax, ub, fb)
    s.set_exclude_bonded(True)
    return s


def test_mlp_batched_replicas_equal_standalone():
    # pair records carry their replica; each pair is evaluated once and summed
    # in list order, so a replica in a batch gets the standalone forces exactly
    cs = [_cg_system(12, 50, seed=31), _cg_system(20, 40, seed=32), _cg_system(9, 60, seed=33)]
    bits, _ = _weights(4)
    reps = [dict(box=c.box, n=c.n, types=c.types, bonds=c.bonds, seed=50 + k) for k, c in enumerate(cs)]
    b = _mlp_system(None, bits, replicas=reps)
    b.set_state(np.concatenate([c.x for c in cs]), None, np.concatenate([c.img for c in cs]))
    b.build_neighbors(RC, SKIN)
    fb = b.compute_forces()
    off = 0
    for k, c in enumerate(cs):
        s = _mlp_system(c, bits, seed=50 + k)
        s.set_state(c.x, None, c.img)
        s.build_neighbors(RC, SKIN)
        assert np.array_equal(s.compute_forces(), fb[off:off + c.n])
        off += c.n


def test_mlp_survives_list_growth(monkeypatch):
    # a list overflow reallocates the list and the learned potential's
    # per-entry buffers, then rebuilds: the forces are those of a roomy list
    c = _cg_system(15, 50, seed=41)
    bits, _ = _weights(5)
    ref = _mlp_system(c, bits)
    ref.set_state(c.x, None, c.img)
    ref.build_neighbors(RC, SKIN)
    monkeypatch.setenv("ESPP_FAULT_LIST_CAP", "8")
    s = _mlp_system(c, bits)
    s.set_state(c.x, None, c.img)
    s.build_neighbors(RC, SKIN)
    assert s.list_capacity > 8
    assert np.array_equal(s.compute_forces(), ref.compute_forces())


def test_mlp_and_table_switch_on_one_handle():
    # the learned potential, then its own table, then the learned potential again
    c = _cg_system(12, 50, seed=51)
    bits, _ = _weights(6)
    s = _mlp_system(c, bits)
    s.set_state(c.x, None, c.img)
    s.build_neighbors(RC, SKIN)
    f_mlp = s.compute_forces()
    rt = np.linspace(0.0, RC, 4096)
    box = np.array([20.0, 20.0, 20.0])
    probe = espp.System(box, 2, None, None, precision=espp.ESPP_FP64)
    probe.set_mlp(RC, bits)
    ut, ft = np.zeros(rt.size), np.zeros(rt.size)
    xs = np.zeros((2, 3))
    for k, r in enumerate(rt):
        xs[0] = (5.0, 5.0, 5.0)
        xs[1] = (5.0 + max(r, 1e-3), 5.0, 5.0)
        probe.set_state(xs)
        if k == 0:
            probe.build_neighbors(RC, SKIN)
        ft[k] = probe.compute_forces()[1, 0]
        ut[k] = probe.observables()["pe_pair"]
    s.set_table_pair(RC, ut, ft)
    f_tab = s.compute_forces()
    assert rel_rms(f_tab, f_mlp) < 2e-2
    s.set_mlp(RC, bits)
    assert np.array_equal(s.compute_forces(), f_mlp)


def test_tensor_core_wait_timeout_is_reported(monkeypatch):
    # host-side fault injection: the tensor-core kernel issues no MMA, its
    # bounded mbarrier wait runs out, it releases its tensor memory and the
    # host reads ESPP_ERR_TIMEOUT; the GPU context stays usable
    c = _cg_system(12, 50, seed=61)
    bits, _ = _weights(7)
    monkeypatch.setenv("ESPP_FAULT_TC_TIMEOUT", "1")
    s = _mlp_system(c, bits)
    s.set_state(c.x, None, c.img)
    s.build_neighbors(RC, SKIN)
    with pytest.raises(espp.EsppError) as e:
        s.compute_forces()
    assert e.value.code == espp.ESPP_ERR_TIMEOUT
    monkeypatch.delenv("ESPP_FAULT_TC_TIMEOUT")
    ok = _mlp_system(c, bits)
    ok.set_state(c.x, None, c.img)
    ok.build_neighbors(RC, SKIN)
    assert np.isfinite(ok.compute_forces()).all()


def test_mlp_requires_weights():
    c = _cg_system(10, 50)
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=espp.ESPP_FP32)
    s.set_interaction(espp.ESPP_MLP, 0, 0, (RC,))
    s.set_state(c.x, None, c.img)
    s.build_neighbors(RC, SKIN)
    with pytest.raises(espp.EsppError):
        s.compute_forces()


def _frames(c, nframes, seed, noise=0.25):
    g = np.random.default_rng(seed)
    X = np.stack([I.f32(np.mod(c.x + g.normal(0, noise, c.x.shape), c.box)) for _ in range(nframes)])
    X[X >= c.box] = 0.0
    return X


def test_mlp_training_gradient_matches_oracle():
    import torch
    c = _cg_system(16, 25, seed=21)
    bits, wd = _weights(3)
    rmax, ub, fb = _bond_table()
    X = _frames(c, 2, 22)
    Y = np.random.default_rng(23).normal(0, 1.0, X.shape)
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=espp.ESPP_FP32, seed=5)
    s.set_mlp(RC, bits)
    s.set_table_bond(rmax, ub, fb)
    s.set_exclude_bonded(True)
    s.set_state(X[0], None, None)
    s.build_neighbors(RC, SKIN)
    loss, grad = s.mlp_loss_grad(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"))
    O.set_mlp(wd, RC)
    O.set_table(8, rmax, ub, fb)
    O.set_exclude_bonded(True)
    try:
        lo, go = O.mlp_loss_grad(O.Model(1, {}, ("table", 8)), c.box, X, Y, c.types, c.bonds)
    finally:
        O.set_exclude_bonded(False)
    go = go[:-1]  # b3 has no gradient
    assert abs(loss - lo) <= 2e-2 * lo
    assert np.linalg.norm(grad - go) <= 5e-2 * np.linalg.norm(go), np.linalg.norm(grad - go) / np.linalg.norm(go)
    # each block of parameters separately
    for lo_, hi_ in ((0, 2048), (2048, 2112), (2112, 6208), (6208, 6272), (6272, 6336)):
        ref = go[lo_:hi_]
        assert np.linalg.norm(grad[lo_:hi_] - ref) <= 8e-2 * np.linalg.norm(ref) + 1e-9, (lo_, hi_)


def test_mlp_training_is_deterministic_and_learns_a_known_potential():
    import torch
    # targets: forces of a smooth repulsive pair potential (a fine table)
    c = I.random_positions(500, (13.5, 13.5, 13.5), seed=31)
    rt = np.linspace(0.0, RC, 4096)
    fc = 0.5 * (np.cos(np.pi * rt / RC) + 1)
    ut = 3.0 * np.exp(-1.5 * rt) * fc
    dfc = -0.5 * np.pi / RC * np.sin(np.pi * rt / RC)
    ft = -(3.0 * (-1.5) * np.exp(-1.5 * rt) * fc + 3.0 * np.exp(-1.5 * rt) * dfc)
    O.set_table(10, RC, ut, ft)
    tmodel = O.Model(1, {(0, 0): ("table", 10, RC)})
    X = _frames(c, 8, 32, noise=0.6)
    Y = np.stack([O.forces(tmodel, c.box, x, c.types, c.bonds)[0] for x in X])
    bits, _ = _weights(4)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    runs = []
    for _ in range(2):
        s = espp.System(c.box, c.n, c.types, c.bonds, precision=espp.ESPP_FP32, seed=5)
        s.set_mlp(RC, bits)
        s.set_state(X[0])
        s.build_neighbors(RC, SKIN)
        loss = s.mlp_train(Xd, Yd, batch_frames=4, epochs=150, lr=2e-3, seed=9)
        runs.append((loss, s.mlp_weights()))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    loss = runs[0][0]
    assert loss[-1] < 0.05 * loss[0], (loss[0], loss[-1])
    # the trained network reproduces the target forces
    s.set_state(X[1])
    f = s.compute_forces()
    assert rel_rms(f, Y[1]) < 0.25


def test_mlp_with_dpd_matches_oracle():
    # the learned potential with all-zero weights (no pair force at all) and
    # the DPD thermostat: the DPD pass over the list (1-2 bonded pairs
    # excluded, as in the list) and the bonds give the oracle's trajectory
    c = _cg_system(20, 30, seed=7)
    zeros = np.zeros(espp.MLP_NPARAMS)
    s = _mlp_system(c, espp.to_bf16_bits(zeros), prec=espp.ESPP_FP64, seed=9)
    v = I.maxwell_velocities(c.n, 1.0, seed=9)
    s.set_state(c.x, v, c.img)
    s.build_neighbors(RC, SKIN)
    s.set_thermostat(espp.ESPP_THERMO_DPD, 2.0)
    s.integrate(60, 0.005, 4.5, 1.0)
    x, vv, img = s.get_state()
    rmax, ub, fb = _bond_table()
    O.set_mlp(zeros, RC)
    O.set_table(7, rmax, ub, fb)
    O.set_exclude_bonded(True)
    O.set_dpd(True, 2.0)
    try:
        model = O.Model(1, {(0, 0): ("mlp", RC)}, ("table", 7))
        st = O.State(c.box, c.x, v, c.img, c.types, c.bonds)
        O.integrate(model, st, 60, 0.005, 4.5, 1.0, seed=9)
    finally:
        O.set_exclude_bonded(False)
        O.set_dpd(False)
    box = c.box
    assert np.abs((x + img * box) - (st.x + st.img * box)).max() < 1e-10
    assert np.abs(vv - st.v).max() < 1e-9
    # with real weights the pass conserves momentum as well
    bits, _ = _weights(3)
    s2 = _mlp_system(c, bits, seed=4)
    v2 = v + np.array([0.05, -0.02, 0.01])
    s2.set_state(c.x, v2, c.img)
    s2.build_neighbors(RC, SKIN)
    s2.set_thermostat(espp.ESPP_THERMO_DPD, 2.0)
    s2.integrate(200, 0.005, 4.5, 1.0)
    _, v3, _ = s2.get_state()
    assert np.abs(v3.sum(axis=0) - v2.sum(axis=0)).max() < 1e-3 * c.n ** 0.5


def test_mlp_refuses_sheared_and_list_free_modes():
    c = _cg_system(seed=2)
    bits, _ = _weights(1)
    s = _mlp_system(c, bits)
    s.set_state(c.x, None, c.img)
    s.build_neighbors(RC, SKIN)
    for call in (lambda: s.set_lees_edwards(True, 0.1, 0.0), lambda: s.set_force_method(espp.ESPP_FORCES_CELLS)):
        with pytest.raises(espp.EsppError) as e:
            call()
        assert e.value.code == espp.ESPP_ERR_STATE
    s.compute_forces()


def test_full_size_cg_4m_sampled_forces():
    # the 4M-site CG melt of the learned-potential benchmark (16,000 chains of
    # 250 sites at density 0.2125), stepped with the learned potential on the
    # tensor cores; sampled summed forces against the oracle's double
    # evaluation of the same BF16 weights on the stored positions
    c = I.kg_lattice(16000, 250, density=0.2125, seed=44, jitter=0.1)
    bits, wd = _weights(4)
    rmax, ub, fb = _bond_table()
    s = espp.System(c.box, c.n, None, c.bonds, precision=espp.ESPP_FP32, seed=45)
    s.set_mlp(RC, bits)
    s.set_table_bond(rmax, ub, fb)
    s.set_exclude_bonded(True)
    s.set_state(c.x, I.maxwell_velocities(c.n, 1.0, seed=46), c.img)
    s.build_neighbors(RC, SKIN)
    s.integrate(100, 0.005, 1.0, 1.0)
    x, _, _ = s.get_state()
    f = s.compute_forces()
    s.close()
    O.set_mlp(wd, RC)
    O.set_table(7, rmax, ub, fb)
    O.set_exclude_bonded(True)
    try:
        model = O.Model(1, {(0, 0): ("mlp", RC)}, ("table", 7))
        sel = np.random.default_rng(8).choice(c.n, 1500, replace=False)
        fo = O.forces_subset(model, c.box, x, c.types, c.bonds, sel)
    finally:
        O.set_exclude_bonded(False)
    assert rel_rms(f[sel], fo) <= MLP_SUM_TOL, rel_rms(f[sel], fo)


def test_training_gradient_over_many_tiles_matches_oracle():
    # a frame of 10k sites (200 chains of 50 at density 0.2125): about 180k
    # pairs, so every gradient CTA accumulates several 128-pair tiles in tensor
    # memory (the small case above gives each CTA at most one); the loss and
    # its weight gradient against the oracle's double evaluation (the oracle
    # needs minutes for a whole 100k-site frame, whose gradient is a sum over
    # every pair and cannot be sampled)
    import torch
    c = I.kg_lattice(200, 50, density=0.2125, seed=31, jitter=0.3)
    bits, wd = _weights(5)
    rmax, ub, fb = _bond_table()
    X = _frames(c, 1, 32)
    Y = np.random.default_rng(33).normal(0, 1.0, X.shape)
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=espp.ESPP_FP32, seed=5)
    s.set_mlp(RC, bits)
    s.set_table_bond(rmax, ub, fb)
    s.set_exclude_bonded(True)
    s.set_state(X[0], None, None)
    s.build_neighbors(RC, 0.0)
    loss, grad = s.mlp_loss_grad(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"))
    s.close()
    O.set_mlp(wd, RC)
    O.set_table(8, rmax, ub, fb)
    O.set_exclude_bonded(True)
    try:
        lo, go = O.mlp_loss_grad(O.Model(1, {}, ("table", 8)), c.box, X, Y, c.types, c.bonds)
    finally:
        O.set_exclude_bonded(False)
    go = go[:-1]  # b3 has no gradient
    assert abs(loss - lo) <= 2e-2 * lo
    assert np.linalg.norm(grad - go) <= 5e-2 * np.linalg.norm(go), np.linalg.norm(grad - go) / np.linalg.norm(go)
