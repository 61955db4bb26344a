"""CPU-only checks of the CUDA library: it builds, loads, exports every symbol
the C header declares, and its host-side Hilbert ordering is a bijection whose
consecutive cells are face neighbours.  No GPU work is issued."""
import os
import re

import numpy as np
import pytest

from paper_2608_14911_gb300 import build as pbuild
from paper_2608_14911_gb300 import espp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return espp.lib()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "espp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(espp_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(lib):
    syms = header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(espp.EXPORTS) == syms


def header_constants():
    txt = open(os.path.join(ROOT, "include", "espp.h")).read()
    return {k: int(v) for k, v in re.findall(r"#define\s+(ESPP_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", txt)}


def test_binding_constants_equal_the_header():
    # every integer the header defines and the binding names has one value;
    # the shape tables have as many rows as the header's shape counts
    consts = header_constants()
    assert len(consts) >= 30
    matched = 0
    for name, value in consts.items():
        for alias in (name, name[len("ESPP_"):]):
            if hasattr(espp, alias):
                assert getattr(espp, alias) == value, (name, alias)
                matched += 1
    assert matched >= 30
    assert len(espp.FORCE_SHAPE_NAMES) == consts["ESPP_FORCE_SHAPES"] == espp.FORCE_SHAPES
    assert len(espp.STEP_SHAPE_TABLE) == consts["ESPP_STEP_SHAPES"] == espp.STEP_SHAPES
    assert espp.MLP_NPARAMS == consts["ESPP_MLP_NPARAMS"]


@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_hilbert_ranks_bijective_and_adjacent(lib, n):
    rank = espp.espp_hilbert_ranks(n, n, n)
    assert np.array_equal(np.sort(rank), np.arange(n ** 3))
    order = np.argsort(rank)
    z, rem = np.divmod(order, n * n)
    y, x = np.divmod(rem, n)
    steps = np.abs(np.diff(x)) + np.abs(np.diff(y)) + np.abs(np.diff(z))
    assert np.all(steps == 1)


@pytest.mark.parametrize("dims", [(3, 5, 7), (69, 69, 69), (76, 76, 38)])
def test_hilbert_ranks_non_power_of_two(lib, dims):
    rank = espp.espp_hilbert_ranks(*dims)
    assert np.array_equal(np.sort(rank), np.arange(np.prod(dims)))
    # locality: consecutive cells are mostly face neighbours
    nx, ny, nz = dims
    order = np.argsort(rank)
    z, rem = np.divmod(order, nx * ny)
    y, x = np.divmod(rem, nx)
    steps = np.abs(np.diff(x)) + np.abs(np.diff(y)) + np.abs(np.diff(z))
    assert np.mean(steps == 1) > 0.9


def test_hilbert_rejects_bad_grid(lib):
    with pytest.raises(espp.EsppError):
        espp.espp_hilbert_ranks(0, 3, 3)


def test_create_without_gpu_fails_loudly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(espp.EsppError):
        espp.System(np.array([10.0, 10.0, 10.0]), 10)


def test_plain_c_client_builds_and_runs(lib, tmp_path):
    # the header is valid C99 and the library links and runs from C alone
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_client")
    libdir = os.path.dirname(pbuild.LIB)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_client.c"),
                    "-L", libdir, "-lespp_gb", "-Wl,-rpath," + libdir, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.startswith(("create refused:", "ok"))


# Every documented argument error of the allocation-free histogram is caught
# on the host before any GPU work, so these calls need no GPU: the pointers
# are never dereferenced.
_BOX = (10.0, 10.0, 10.0)
NOALLOC_REFUSALS = {
    "n_negative": dict(n=-1),
    "n_above_limit": dict(n=espp.NOALLOC_MAX_N + 1),
    "nbins_zero": dict(nbins=0),
    "nbins_above_limit": dict(nbins=espp.NOALLOC_MAX_BINS + 1),
    "rmax_zero": dict(rmax=0.0),
    "rmax_negative": dict(rmax=-1.0),
    "rmax_half_box": dict(rmax=5.0),
    "rmax_nan": dict(rmax=float("nan")),
    "box_edge_zero": dict(box=(10.0, 0.0, 10.0)),
    "null_positions": dict(x=0),
    "null_counts": dict(counts=0),
    "null_box": dict(box=None),
}


def _noalloc_raw(L, n=10, nbins=16, rmax=2.0, box=_BOX, x=0x1000, counts=0x2000):
    import ctypes
    b = None if box is None else (ctypes.c_double * 3)(*box)
    return L.espp_rdf_counts_noalloc(ctypes.c_void_p(x), n, b, rmax, nbins, ctypes.c_void_p(counts),
                                     ctypes.c_void_p(0))


@pytest.mark.parametrize("case", sorted(NOALLOC_REFUSALS))
def test_noalloc_refuses_bad_arguments_on_the_host(lib, case):
    assert _noalloc_raw(lib, **NOALLOC_REFUSALS[case]) == espp.ESPP_ERR_ARG


def test_noalloc_binding_refuses_wrong_tensors_before_the_call(lib):
    torch = pytest.importorskip("torch")
    # host tensors are refused by the binding (the library would read them
    # as device memory); so are the wrong dtypes and shapes, checked first
    with pytest.raises(ValueError):
        espp.espp_rdf_counts_noalloc(torch.zeros((4, 3), dtype=torch.float32), _BOX, 2.0,
                                     torch.zeros(8, dtype=torch.int64))
    with pytest.raises(ValueError):
        espp.espp_rdf_counts_noalloc(np.zeros((4, 3)), _BOX, 2.0, np.zeros(8, dtype=np.int64))
