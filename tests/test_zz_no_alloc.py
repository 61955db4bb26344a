"""The allocation-free pair-distance histogram (espp_rdf_counts_noalloc).

Callers that cannot call cudaMalloc (a framework that owns a fixed device
memory pool, a latency-critical loop that cannot take cudaMalloc's implicit
synchronisation) use this entry point; its working buffer is a fixed array
inside the library.  The tests check, through the C ABI, that it gives the
same counts as the handle-based espp_rdf_counts on the same positions (the
all-pairs path of a plain periodic box, which both count the same way), on
two calls in a row (the shared array must be cleared between calls), that
every documented argument error is refused with the caller's counts left
untouched, and that the binding refuses tensors of the wrong type, shape or
device.  This file sorts last so that a run stopping at the first failure has
run every other test first."""
import numpy as np
import pytest

from paper_2608_14911_gb300 import espp, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _positions():
    c = I.lj_fcc(6, 6, 6, density=0.8442)
    g = np.random.default_rng(7)
    c.x = I.f32(np.mod(c.x + g.normal(0, 0.08, c.x.shape), c.box))
    c.x[c.x >= c.box] = 0.0
    return c


def test_noalloc_histogram_matches_handle_path_twice():
    import torch
    c = _positions()
    s = espp.System(c.box, c.n, c.types, c.bonds, precision=espp.ESPP_FP64)
    s.set_lj(1.0, 1.0, 2.5, True)
    s.set_state(c.x, None, c.img)
    for rmax, nbins in ((3.0, 60), (2.5, 500)):
        ref = s.rdf_counts(rmax, nbins)
        x, _, _ = s.get_state()
        xd = torch.tensor(x, device="cuda")
        for _ in range(2):
            out = torch.full((nbins,), -1, dtype=torch.int64, device="cuda")
            espp.espp_rdf_counts_noalloc(xd, c.box, rmax, out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), ref)
    s.close()


def test_noalloc_rejects_too_many_bins():
    import torch
    c = _positions()
    xd = torch.tensor(c.x, device="cuda")
    out = torch.zeros(espp.NOALLOC_MAX_BINS + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(espp.EsppError) as e:
        espp.espp_rdf_counts_noalloc(xd, c.box, 2.0, out)
    assert e.value.code == espp.ESPP_ERR_ARG


REFUSALS = {
    "n_negative": dict(n=-1),
    "n_above_limit": dict(n=espp.NOALLOC_MAX_N + 1),
    "nbins_zero": dict(nbins=0),
    "rmax_zero": dict(rmax=0.0),
    "rmax_half_box": dict(rmax=None),
    "box_edge_negative": dict(box=(-1.0, 1.0, 1.0)),
    "null_positions": dict(x=0),
}


@pytest.mark.parametrize("case", sorted(REFUSALS))
def test_noalloc_refusal_leaves_counts_untouched(case):
    import ctypes

    import torch
    c = _positions()
    xd = torch.tensor(c.x, device="cuda")
    nbins = 32
    out = torch.full((nbins,), -7, dtype=torch.int64, device="cuda")
    kw = dict(n=c.n, nbins=nbins, rmax=2.0, box=tuple(c.box), x=xd.data_ptr())
    kw.update(REFUSALS[case])
    if kw["rmax"] is None:
        kw["rmax"] = 0.5 * float(min(c.box))
    b = (ctypes.c_double * 3)(*kw["box"])
    rc = espp.lib().espp_rdf_counts_noalloc(ctypes.c_void_p(kw["x"]), kw["n"], b, kw["rmax"], kw["nbins"],
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    torch.cuda.synchronize()
    assert rc == espp.ESPP_ERR_ARG
    assert bool((out == -7).all())


def test_noalloc_binding_refuses_wrong_tensors():
    import torch
    c = _positions()
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    bad_x = (torch.tensor(c.x, device="cuda", dtype=torch.float32),      # float32
             torch.tensor(c.x, device="cuda").reshape(-1),               # (3n,)
             torch.tensor(c.x, device="cuda").t(),                       # not contiguous, (3, n)
             torch.tensor(c.x))                                          # host memory
    for x in bad_x:
        with pytest.raises(ValueError):
            espp.espp_rdf_counts_noalloc(x, c.box, 2.0, out)
    xd = torch.tensor(c.x, device="cuda")
    for cnt in (torch.zeros(16, dtype=torch.int32, device="cuda"), torch.zeros(16, dtype=torch.int64)):
        with pytest.raises(ValueError):
            espp.espp_rdf_counts_noalloc(xd, c.box, 2.0, cnt)
