"""H5MD output and input: files the library writes, parsed by the test-side
HDF5 reader (every checksum verified), hold the handle's state in the H5MD
1.1 layout; a run resumed from such a file continues the trajectory (the
Philox stream restored by the seeds and the step)."""
import numpy as np
import pytest

from paper_2608_14911_gb300 import espp

import _h5read as H
from _systems import WCA_RC, kg_case

pytestmark = pytest.mark.gpu

FP32, FP64 = espp.ESPP_FP32, espp.ESPP_FP64
DT = 0.005


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available()


def _string(a):
    return a.reshape(-1)[0].decode() if a.shape else a.item().decode()


def _bond_set(bonds):
    return {tuple(sorted(map(int, b))) for b in np.asarray(bonds).reshape(-1, 2)}


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_written_file_holds_the_state_in_the_h5md_layout(prec, tmp_path):
    case = kg_case()
    c = case.cfg
    s = case.system(prec, seed=23)
    s.integrate(113, DT, 1.0, 1.0)
    path = tmp_path / "state.h5"
    s.h5md_write(path)
    x, v, img = s.get_state()
    f = H.read(path)
    assert list(f["h5md"].attrs["version"]) == [1, 1]
    assert _string(f["h5md/author"].attrs["name"])
    assert _string(f["h5md/creator"].attrs["name"]) and _string(f["h5md/creator"].attrs["version"])
    box = f["particles/all/box"]
    assert int(box.attrs["dimension"]) == 3
    assert [b.decode() for b in box.attrs["boundary"]] == ["periodic"] * 3
    assert np.array_equal(f["particles/all/box/edges"].value, c.box)
    for name, ref in (("position", x), ("velocity", v), ("image", img)):
        el = f["particles/all/" + name]
        assert el["step"].value.tolist() == [113]
        assert el["time"].value.tolist() == [113 * DT]
        assert el["value"].value.shape == (1, c.n, 3)
        assert np.array_equal(el["value"].value[0], ref)
    assert f["particles/all/image/value"].value.dtype == np.int32
    fel = f["particles/all/force"]
    assert fel["step"].value.tolist() == [113] and fel["value"].value.shape == (1, c.n, 3)
    assert np.isfinite(fel["value"].value).all() and np.abs(fel["value"].value).max() > 0
    assert np.array_equal(f["particles/all/species"].value, c.types)
    assert _bond_set(f["connectivity/all/bonds"].value) == _bond_set(c.bonds)
    par = f["parameters/espp"]
    assert int(par.attrs["step"]) == 113 and float(par.attrs["time"]) == 113 * DT
    # the handle-free inspection reads the same file
    assert espp.h5md_inspect(path) == {"replicas": 1, "particles": c.n, "step": 113, "precision": prec}
    assert int(par.attrs["precision"]) == prec and int(par.attrs["lees_edwards"]) == 0
    assert par["seeds"].value.tolist() == [23]
    # the wrapped positions lie in the box; unwrapping restores the chains
    xv = f["particles/all/position/value"].value[0]
    assert (xv >= 0).all() and (xv < c.box).all()
    u = xv + f["particles/all/image/value"].value[0] * c.box
    b = np.asarray(c.bonds)
    assert np.linalg.norm(u[b[:, 0]] - u[b[:, 1]], axis=1).max() < 1.5
    s.close()


def test_state_without_a_step_has_no_force_element(tmp_path):
    case = kg_case()
    s = case.system(FP64)
    path = tmp_path / "fresh.h5"
    s.h5md_write(path)
    f = H.read(path)
    assert "force" not in f["particles/all"].children
    assert f["particles/all/position/step"].value.tolist() == [0]
    # a run resumed from it equals one started from the same set_state
    b = case.system(FP64)
    b.h5md_read(path)
    s.integrate(30, DT, 1.0, 1.0)
    b.integrate(30, DT, 1.0, 1.0)
    xs, vs, _ = s.get_state()
    xb, vb, _ = b.get_state()
    assert np.abs(xs - xb).max() <= 1e-12 and np.abs(vs - vb).max() <= 1e-12
    s.close()
    b.close()


def test_batched_replicas_write_one_group_each(tmp_path):
    cases_ = [kg_case(3, 40, seed=101, jitter=0.08), kg_case(5, 30, seed=202, jitter=0.08)]
    reps = [dict(box=k.cfg.box, n=k.cfg.n, types=k.cfg.types, bonds=k.cfg.bonds, seed=500 + i)
            for i, k in enumerate(cases_)]
    b = espp.System(replicas=reps, precision=FP32)
    b.set_wca()
    b.set_fene()
    b.set_state(np.concatenate([k.cfg.x for k in cases_]), np.concatenate([k.v for k in cases_]),
                np.concatenate([k.cfg.img for k in cases_]))
    b.build_neighbors(WCA_RC, 0.4)
    b.integrate(40, DT, 1.0, 1.0)
    path = tmp_path / "batch.h5"
    b.h5md_write(path)
    x, v, img = b.get_state()
    f = H.read(path)
    assert sorted(f["particles"].children) == ["replica_0", "replica_1"]
    off = 0
    for r, k in enumerate(cases_):
        n = k.cfg.n
        g = "particles/replica_%d/" % r
        assert np.array_equal(f[g + "box/edges"].value, k.cfg.box)
        assert np.array_equal(f[g + "position/value"].value[0], x[off:off + n])
        assert np.array_equal(f[g + "velocity/value"].value[0], v[off:off + n])
        assert np.array_equal(f[g + "image/value"].value[0], img[off:off + n])
        assert _bond_set(f["connectivity/replica_%d/bonds" % r].value) == _bond_set(k.cfg.bonds)
        off += n
    assert f["parameters/espp/seeds"].value.tolist() == [500, 501]
    info = espp.h5md_inspect(path)
    assert info["replicas"] == 2 and info["particles"] == sum(k.cfg.n for k in cases_) and info["step"] == 40
    b.close()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-9), (FP32, 2e-3)])
def test_resume_from_h5md_continues_the_trajectory(prec, tol, tmp_path):
    # FP64: the resumed run differs from the uninterrupted one by the order of
    # force sums only (the list is rebuilt from the file); over 40 steps that
    # stays far below 1e-9.  FP32: the same at single-precision rounding.
    case = kg_case()
    c = case.cfg
    a = case.system(prec, seed=31)
    a.integrate(97, DT, 1.0, 1.0)
    path = tmp_path / "resume.h5"
    a.h5md_write(path)
    a.integrate(40, DT, 1.0, 1.0)
    xa, va, ia = a.get_state()
    b = espp.System(c.box, c.n, c.types, c.bonds, precision=prec, seed=999)
    b.set_wca()
    b.set_fene()
    b.set_state(c.x, case.v, c.img)
    b.build_neighbors(WCA_RC, 0.4)
    b.h5md_read(path)
    assert b.step == 97
    b.integrate(40, DT, 1.0, 1.0)
    xb, vb, ib = b.get_state()
    assert b.step == a.step == 137
    ua, ub = xa + ia * c.box, xb + ib * c.box
    assert np.abs(ua - ub).max() <= tol
    assert np.abs(va - vb).max() <= 10 * tol
    # a handle with the file's seed but without the file diverges at once:
    # the restored stream is the file's, not the handle's own
    assert np.abs(va).max() > 0
    a.close()
    b.close()


def test_read_refuses_other_handles_and_broken_files(tmp_path):
    case = kg_case()
    a = case.system(FP32, seed=3)
    a.integrate(10, DT, 1.0, 1.0)
    path = tmp_path / "a.h5"
    a.h5md_write(path)
    # another particle count
    other = kg_case(7, 23, seed=5, jitter=0.1)
    o = other.system(FP32)
    with pytest.raises(espp.EsppError):
        o.h5md_read(path)
    # a header byte changed: the object-header checksum fails
    data = bytearray(path.read_bytes())
    k = data.find(b"OHDR", 100)
    data[k + 12] ^= 0x40
    bad = tmp_path / "bad.h5"
    bad.write_bytes(bytes(data))
    b = case.system(FP32, seed=3)
    x0, v0, i0 = b.get_state()
    with pytest.raises(espp.EsppError):
        b.h5md_read(bad)
    with pytest.raises(espp.EsppError):
        b.h5md_read(tmp_path / "missing.h5")
    # not an HDF5 file at all
    junk = tmp_path / "junk.h5"
    junk.write_bytes(b"not hdf5" * 20)
    with pytest.raises(espp.EsppError):
        b.h5md_read(junk)
    x1, v1, i1 = b.get_state()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1) and np.array_equal(i0, i1)
    assert b.step == 0
    # and the intact file loads
    b.h5md_read(path)
    assert b.step == 10
    a.close()
    b.close()
    o.close()


def test_resume_under_lees_edwards(tmp_path):
    # a sheared run: the file keeps the shear rate and the simulated time (the
    # offset delta = gdot Lz t), and the resumed run continues the trajectory;
    # positions compared through the sheared minimum image
    case = kg_case()
    c = case.cfg

    def make(seed):
        s = case.system(FP64, seed=seed, build=False)
        s.set_lees_edwards(True, 0.8, 1.25)
        s.build_neighbors(case.rc_list, case.skin)
        return s

    a = make(9)
    a.integrate(120, DT, 1.0, 1.0)
    path = tmp_path / "le.h5"
    a.h5md_write(path)
    f = H.read(path)
    par = f["parameters/espp"]
    assert int(par.attrs["lees_edwards"]) == 1 and float(par.attrs["shear_rate"]) == 0.8
    assert float(par.attrs["time"]) == pytest.approx(1.25 + 120 * DT, abs=1e-12)
    a.integrate(40, DT, 1.0, 1.0)
    b = make(77)
    b.h5md_read(path)
    assert b.step == 120 and b.lees_edwards()[2] == pytest.approx(1.25 + 120 * DT, abs=1e-12)
    b.integrate(40, DT, 1.0, 1.0)
    xa, va, _ = a.get_state()
    xb, vb, _ = b.get_state()
    delta = 0.8 * c.box[2] * (1.25 + 160 * DT)
    d = xa - xb
    k = np.rint(d[:, 2] / c.box[2])
    d[:, 2] -= k * c.box[2]
    d[:, 0] -= k * delta
    d[:, 0] -= np.rint(d[:, 0] / c.box[0]) * c.box[0]
    d[:, 1] -= np.rint(d[:, 1] / c.box[1]) * c.box[1]
    assert np.abs(d).max() <= 1e-9
    dv = va - vb
    dv[:, 0] -= k * 0.8 * c.box[2]
    assert np.abs(dv).max() <= 1e-8
    # a handle without shear refuses the sheared file
    p = case.system(FP64, seed=9)
    with pytest.raises(espp.EsppError):
        p.h5md_read(path)
    a.close()
    b.close()
    p.close()
