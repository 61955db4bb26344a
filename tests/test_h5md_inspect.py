"""The library's H5MD reader on files written by the test-side HDF5 writer
(tests/_h5write.py, from the HDF5 specification): a well-formed file is read
back by espp_h5md_inspect (host code, no GPU), and files with planted faults
(shapes larger than their data, addresses past the end or wrapping around,
links that form a cycle or reach one object twice, a truncated file) are
refused with ESPP_ERR_IO instead of being read out of bounds."""
import struct

import numpy as np
import pytest

import _h5read as R
import _h5write as W
from paper_2608_14911_gb300 import espp

N = 5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()


def _h5md(n=N, seeds=(77,), seeds_dims=None, position_dims=None, position=None, extra_root=None,
          extra_links=(), step=123, precision=espp.ESPP_FP64):
    """The H5MD tree the reader expects for one replica of n particles (the
    layout espp_h5md_write produces), with optional planted faults."""
    rng = np.random.default_rng(5)
    box = np.array([4.0, 5.0, 6.0])
    x = rng.uniform(0, 4.0, (1, n, 3))
    v = rng.normal(size=(1, n, 3))
    img = np.zeros((1, n, 3), np.int32)
    species = np.zeros(n, np.int32)
    value = lambda dtype, arr, dims=None: W.Group({"value": W.Dataset(dtype, dims or arr.shape, arr.tobytes())})
    particles = W.Group({
        "box": W.Group({"edges": W.Dataset(W.t_f64(), [3], box.tobytes())}),
        "position": W.Group({"value": W.Dataset(W.t_f64(), position_dims or x.shape,
                                                 (x if position is None else position).tobytes())}),
        "velocity": value(W.t_f64(), v),
        "image": value(W.t_int(4), img),
        "species": W.Dataset(W.t_int(4), [n], species.tobytes()),
    })
    s = np.array(seeds, np.uint64)
    espp_par = W.Group({"seeds": W.Dataset(W.t_int(8, False), seeds_dims or [len(s)], s.tobytes())}, attrs=[
        W.attribute("step", W.t_int(8), [], struct.pack("<q", step), scalar=True),
        W.attribute("time", W.t_f64(), [], struct.pack("<d", 0.005 * step), scalar=True),
        W.attribute("precision", W.t_int(4), [], struct.pack("<i", precision), scalar=True),
        W.attribute("lees_edwards", W.t_int(4), [], struct.pack("<i", 0), scalar=True),
        W.attribute("shear_rate", W.t_f64(), [], struct.pack("<d", 0.0), scalar=True),
    ])
    root = W.Group({
        "h5md": W.Group(attrs=[W.attribute("version", W.t_int(4), [2], struct.pack("<ii", 1, 1))]),
        "particles": W.Group({"all": particles}),
        "parameters": W.Group({"espp": espp_par}),
    }, links=list(extra_links))
    if extra_root:
        root.children.update(extra_root)
    return root, particles


def _write(tmp_path, root, name="f.h5", root_addr=None):
    path = tmp_path / name
    path.write_bytes(W.File().bytes(root, root_addr))
    return path


def _refused(path):
    with pytest.raises(espp.EsppError) as e:
        espp.h5md_inspect(path)
    assert e.value.code == espp.ESPP_ERR_IO
    return str(e.value)


def test_well_formed_file_is_read(tmp_path):
    root, _ = _h5md()
    path = _write(tmp_path, root)
    # the test writer's file passes the test reader (every checksum) ...
    f = R.read(path)
    assert f["particles/all/position/value"].value.shape == (1, N, 3)
    assert list(f["h5md"].attrs["version"]) == [1, 1]
    # ... and the library's reader
    info = espp.h5md_inspect(path)
    assert info == {"replicas": 1, "particles": N, "step": 123, "precision": espp.ESPP_FP64}


def test_missing_file_and_null_path():
    assert "cannot open" in _refused("/nonexistent/espp.h5")
    with pytest.raises(espp.EsppError) as e:
        espp._check(espp.lib().espp_h5md_inspect(None, None, None, None, None))
    assert e.value.code == espp.ESPP_ERR_ARG


def test_shape_larger_than_its_data_is_refused(tmp_path):
    # the seeds claim 1000 replicas over 8 bytes of data
    root, _ = _h5md(seeds_dims=[1000])
    assert "seeds" in _refused(_write(tmp_path, root))
    # positions claim 10^6 particles over N
    root, _ = _h5md(position_dims=[1, 10 ** 6, 3])
    _refused(_write(tmp_path, root, "p.h5"))


def test_shape_whose_element_count_overflows_is_refused(tmp_path):
    # 2^62 x 2^2 x 3 elements wrap around 64 bits; the data are N x 3 doubles
    root, _ = _h5md(position_dims=[2 ** 62, 4, 3])
    _refused(_write(tmp_path, root))
    root, _ = _h5md(seeds_dims=[2 ** 61])  # 8 * 2^61 wraps to 0
    _refused(_write(tmp_path, root, "s.h5"))


def test_addresses_past_the_end_or_wrapping_are_refused(tmp_path):
    # a link past the end of the file, and one that wraps around 64 bits
    for k, addr in enumerate((10 ** 9, W.UNDEF - 7)):
        root, _ = _h5md(extra_links=[("far", addr)])
        assert "object header" in _refused(_write(tmp_path, root, "l%d.h5" % k))
    # a dataset whose data address + size wraps around
    root, particles = _h5md()
    particles.children["species"] = W.Dataset(W.t_int(4), [N], np.zeros(N, np.int32).tobytes(),
                                              addr=W.UNDEF - 8, size=16)
    assert "readable data" in _refused(_write(tmp_path, root, "d.h5"))
    # the root group's address past the end
    root, _ = _h5md()
    _refused(_write(tmp_path, root, "r.h5", root_addr=W.UNDEF - 3))


def test_links_that_cycle_or_share_an_object_are_refused(tmp_path):
    # a group linking to itself: read once, not walked again and again
    root, _ = _h5md(extra_links=[("loop", "self")])
    assert "twice" in _refused(_write(tmp_path, root))
    # one dataset linked from two groups
    shared = W.Dataset(W.t_f64(), [3], np.zeros(3).tobytes())
    root, _ = _h5md(extra_root={"a": W.Group({"x": shared})})
    root.children["b"] = W.Group(links=[("x", shared)])
    assert "twice" in _refused(_write(tmp_path, root, "s.h5"))


def test_truncated_or_corrupted_file_is_refused(tmp_path):
    root, _ = _h5md()
    data = W.File().bytes(root)
    for k, cut in enumerate((30, 47, len(data) // 2, len(data) - 3)):
        p = tmp_path / ("t%d.h5" % k)
        p.write_bytes(data[:cut])
        _refused(p)
    # every single-byte change inside an object header fails its checksum
    k = data.find(b"OHDR", 48)
    for off in (6, 9, 20):
        bad = bytearray(data)
        bad[k + off] ^= 0x5A
        p = tmp_path / ("c%d.h5" % off)
        p.write_bytes(bytes(bad))
        _refused(p)
