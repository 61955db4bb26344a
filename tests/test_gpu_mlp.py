"""The learned CG pair potential on the tensor cores against the oracle's
double-precision evaluation of the same network (BF16 weights upcast).

Tolerance: the GPU rounds the radial features and the first-layer
activations to BF16 (relative 2^-9 each) before FP32-accumulated GEMMs, so a
pair's du/dr carries a relative error of order 1e-2 at worst; the summed
forces are checked at 3e-2 relative RMS and the energies at 1e-2."""
import numpy as np
import pytest

import oracle as O
from paper_2608_14911_gb300 import espp, inputs as I

from _systems import rel_rms

pytestmark = pytest.mark.gpu
RC = 3.5
SKIN = 0.5


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
    assert rel_rms(f, fo) <= 3e-2, rel_rms(f, fo)
    assert abs(o["pe_pair"] - en[0]) <= 1e-2 * abs(en[0])
    assert abs(o["pe_bond"] - en[1]) <= 1e-5 * abs(en[1])
    # each pair is evaluated from both ends with identical arithmetic
    assert np.abs(f.sum(axis=0)).max() <= 1e-4 * np.abs(f).sum()


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


def test_mlp_requires_weights():
    c = _cg_system(10, 50)
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=espp.ESPP_FP32)
    s.set_interaction(espp.ESPP_MLP, 0, 0, (RC,))
    s.set_state(c.x, None, c.img)
    s.build_neighbors(RC, SKIN)
    with pytest.raises(espp.EsppError):
        s.compute_forces()
