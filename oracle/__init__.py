"""Python access to the double-precision CPU oracle (oracle/orc.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py, never by the product package.  The oracle shares
no code with the CUDA library.

Interaction descriptions are plain dicts so that the test code states every
parameter explicitly:
    pair = {(ta, tb): ("lj", eps, sigma, rc, shift) | ("wca", eps, sigma)
                      | ("lj_capped", eps, sigma, rc, shift, caprad)
                      | ("table", slot, rc)}
    bond = ("fene", K, R0) | ("table", slot) | None
Tables are registered with set_table(slot, rmax, u, f).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

PAIR_STRIDE = 8
BOND_STRIDE = 4
NOBS = 13
OBS_NAMES = ("ke", "pe_pair", "pe_bond", "virial", "px", "py", "pz",
             "temperature", "pressure", "mean_bond", "rg2", "nmol", "pxz")

_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_uniform_centered.argtypes = [ctypes.c_uint32]
        L.orc_uniform_centered.restype = ctypes.c_double
        L.orc_uniform_fill.argtypes = [_u32p, ctypes.c_int64, _dp]
        L.orc_langevin_noise.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, _dp]
        L.orc_pair_eval.argtypes = [_dp, ctypes.c_double, _dp, _dp]
        L.orc_bond_eval.argtypes = [_dp, ctypes.c_double, _dp, _dp]
        L.orc_bond_eval.restype = ctypes.c_int
        L.orc_forces.argtypes = [ctypes.c_int64, _dp, _dp, _i32p, ctypes.c_int, _dp,
                                 ctypes.c_int64, _i64p, _dp, _dp, _dp]
        L.orc_forces.restype = ctypes.c_int
        L.orc_set_table.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]
        L.orc_set_table.restype = ctypes.c_int
        L.orc_set_mlp.argtypes = [_dp, ctypes.c_int64, ctypes.c_double]
        L.orc_set_mlp.restype = ctypes.c_int
        L.orc_mlp_pair.argtypes = [ctypes.c_double, _dp, _dp, _dp, _dp]
        L.orc_set_exclude_bonded.argtypes = [ctypes.c_int]
        L.orc_set_dpd.argtypes = [ctypes.c_int, ctypes.c_double]
        L.orc_dpd_theta.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        L.orc_dpd_theta.restype = ctypes.c_double
        L.orc_set_lees_edwards.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_le_get_time.restype = ctypes.c_double
        L.orc_mlp_loss_grad.argtypes = [ctypes.c_int64, _dp, ctypes.c_int64, _dp, _dp, _i32p,
                                        ctypes.c_int64, _i64p, _dp, _dp, _dp]
        L.orc_mlp_loss_grad.restype = ctypes.c_int
        L.orc_forces_subset.argtypes = [ctypes.c_int64, _dp, _dp, _i32p, ctypes.c_int, _dp,
                                        ctypes.c_int64, _i64p, _dp, ctypes.c_int64, _i64p, _dp]
        L.orc_forces_subset.restype = ctypes.c_int
        for fn in (L.orc_neighbors_brute, L.orc_neighbors_cells):
            fn.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, _i64p, _i64p, ctypes.c_int64]
            fn.restype = ctypes.c_int64
        L.orc_integrate.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _i32p, _i32p, _dp, ctypes.c_int,
                                    _dp, ctypes.c_int64, _i64p, _dp, _dp, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
        L.orc_integrate.restype = ctypes.c_int
        L.orc_observables.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _i32p, _i32p, _dp, ctypes.c_int,
                                      _dp, ctypes.c_int64, _i64p, _dp, _dp]
        L.orc_observables.restype = ctypes.c_int
        L.orc_rdf_counts.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_int, _i64p]
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


WCA_RC = 2.0 ** (1.0 / 6.0)


def pair_table(pair: dict, ntypes: int) -> np.ndarray:
    """Flatten a {(ta, tb): spec} dict into the oracle's pair records."""
    t = np.zeros((ntypes, ntypes, PAIR_STRIDE), dtype=np.float64)
    for (a, b), spec in pair.items():
        kind = spec[0]
        if kind == "lj":
            _, eps, sig, rc, shift = spec
            rec = [1, eps, sig, rc, 1.0 if shift else 0.0, 0.0]
        elif kind == "wca":
            _, eps, sig = spec
            rec = [1, eps, sig, WCA_RC * sig, 1.0, 0.0]
        elif kind == "lj_capped":
            _, eps, sig, rc, shift, cap = spec
            rec = [2, eps, sig, rc, 1.0 if shift else 0.0, cap]
        elif kind == "table":
            _, slot, rc = spec
            rec = [3, slot, 0.0, rc, 0.0, 0.0]
        elif kind == "mlp":
            _, rc = spec
            rec = [4, 0.0, 0.0, rc, 0.0, 0.0]
        else:
            raise ValueError(kind)
        t[a, b, :6] = rec
        t[b, a, :6] = rec
    return t.reshape(-1)


def bond_table(bond) -> np.ndarray:
    b = np.zeros(BOND_STRIDE, dtype=np.float64)
    if bond is None:
        return b
    if bond[0] == "fene":
        b[:3] = [1, bond[1], bond[2]]
        return b
    if bond[0] == "table":
        b[:2] = [2, bond[1]]
        return b
    raise ValueError(bond[0])


MLP_NPARAMS = 64 * 32 + 64 + 64 * 64 + 64 + 64 + 1


def set_mlp(params, rc):
    """Register the learned pair potential (parameters in double; the caller
    upcasts BF16 weights)."""
    p = _f64(params)
    if lib().orc_set_mlp(_p(p, _dp), p.size, rc) != 0:
        raise ValueError("bad MLP parameters")


def mlp_pair(r, want_grad=False):
    """u(r), du/dr and (optionally) their gradients w.r.t. the parameters."""
    u, du = ctypes.c_double(), ctypes.c_double()
    g = np.zeros(MLP_NPARAMS) if want_grad else None
    gu = np.zeros(MLP_NPARAMS) if want_grad else None
    lib().orc_mlp_pair(r, ctypes.byref(u), ctypes.byref(du),
                       _p(g, _dp) if want_grad else None, _p(gu, _dp) if want_grad else None)
    if want_grad:
        return u.value, du.value, g, gu
    return u.value, du.value


def mlp_loss_grad(model, box, frames_x, frames_y, types, bonds):
    """Force-matching loss and its parameter gradient (pair potential = the
    registered MLP, bonds as in `model`)."""
    _le(0.0)
    X = _f64(frames_x)
    Y = _f64(frames_y)
    nf = X.shape[0]
    n = X.shape[1]
    L = _f64(box)
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = np.ascontiguousarray(bonds, dtype=np.int64).reshape(-1, 2)
    loss = ctypes.c_double()
    g = np.zeros(MLP_NPARAMS)
    st = lib().orc_mlp_loss_grad(n, _p(L, _dp), nf, _p(X, _dp), _p(Y, _dp), _p(t, _i32p), b.shape[0],
                                 _p(b, _i64p), _p(model.bond, _dp), ctypes.byref(loss), _p(g, _dp))
    if st != 0:
        raise RuntimeError("oracle loss failed (%d)" % st)
    return loss.value, g


def set_exclude_bonded(on):
    lib().orc_set_exclude_bonded(1 if on else 0)


# Lees-Edwards setting of the calls below (flow x, gradient z, shear rate)
_LE = {"on": False, "shear": 0.0}


def set_lees_edwards(on, shear=0.0):
    """Lees-Edwards boundary conditions for the following calls; the offset
    is shear * Lz * t with t the State's (or the call's) simulated time."""
    _LE["on"] = bool(on)
    _LE["shear"] = float(shear)


def _le(time):
    lib().orc_set_lees_edwards(1 if _LE["on"] else 0, _LE["shear"], float(time))


def set_dpd(on, rc=0.0):
    """Use the DPD thermostat (pair cutoff rc) instead of Langevin in integrate."""
    lib().orc_set_dpd(1 if on else 0, float(rc))


def dpd_theta(seed, a, b, step):
    """The pair noise theta_ab of a step (symmetric in a, b)."""
    return lib().orc_dpd_theta(int(seed), int(a), int(b), int(step))


def set_table(slot, rmax, u, f):
    """Register a table: u and F = -dU/dr at r_k = k rmax / (n - 1)."""
    u = _f64(u)
    f = _f64(f)
    if lib().orc_set_table(slot, rmax, u.size, _p(u, _dp), _p(f, _dp)) != 0:
        raise ValueError("bad table")


class Model:
    """The interaction set of one system as the oracle sees it."""

    def __init__(self, ntypes=1, pair=None, bond=None, masses=None):
        self.ntypes = ntypes
        self.pair = pair_table(pair or {}, ntypes)
        self.bond = bond_table(bond)
        self.masses = _f64(masses if masses is not None else np.ones(ntypes))


def philox(ctr, key):
    out = np.zeros(4, dtype=np.uint32)
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def uniform_centered(words) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32).reshape(-1)
    out = np.empty(w.size, dtype=np.float64)
    lib().orc_uniform_fill(_p(w, _u32p), w.size, _p(out, _dp))
    return out


def langevin_noise(seed: int, step: int, n: int) -> np.ndarray:
    out = np.empty((n, 3), dtype=np.float64)
    lib().orc_langevin_noise(seed, step, n, _p(out, _dp))
    return out


def pair_eval(model: Model, ta: int, tb: int, r2: float):
    u, fr = ctypes.c_double(), ctypes.c_double()
    rec = model.pair[PAIR_STRIDE * (ta * model.ntypes + tb):][:PAIR_STRIDE].copy()
    lib().orc_pair_eval(_p(rec, _dp), r2, ctypes.byref(u), ctypes.byref(fr))
    return u.value, fr.value


def bond_eval(model: Model, r2: float):
    u, fr = ctypes.c_double(), ctypes.c_double()
    rc = lib().orc_bond_eval(_p(model.bond, _dp), r2, ctypes.byref(u), ctypes.byref(fr))
    return u.value, fr.value, rc


def forces(model: Model, box, x, types, bonds, time=0.0):
    """Conservative forces and (PE_pair, PE_bond, virial, virial_xz); raises
    on a broken bond.  time: simulated time (Lees-Edwards offset)."""
    _le(time)
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    L = _f64(box)
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = np.ascontiguousarray(bonds, dtype=np.int64).reshape(-1, 2)
    f = np.zeros((n, 3), dtype=np.float64)
    en = np.zeros(4, dtype=np.float64)
    st = lib().orc_forces(n, _p(L, _dp), _p(x, _dp), _p(t, _i32p), model.ntypes,
                          _p(model.pair, _dp), b.shape[0], _p(b, _i64p),
                          _p(model.bond, _dp), _p(f, _dp), _p(en, _dp))
    if st != 0:
        raise RuntimeError("oracle: bond broken (status %d)" % st)
    return f, en


def forces_subset(model: Model, box, x, types, bonds, sel, time=0.0):
    """Conservative forces on the particles `sel` only (same definition)."""
    _le(time)
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    L = _f64(box)
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = np.ascontiguousarray(bonds, dtype=np.int64).reshape(-1, 2)
    s = np.ascontiguousarray(sel, dtype=np.int64)
    f = np.zeros((s.size, 3), dtype=np.float64)
    st = lib().orc_forces_subset(n, _p(L, _dp), _p(x, _dp), _p(t, _i32p), model.ntypes,
                                 _p(model.pair, _dp), b.shape[0], _p(b, _i64p),
                                 _p(model.bond, _dp), s.size, _p(s, _i64p), _p(f, _dp))
    if st != 0:
        raise RuntimeError("oracle: bond broken (status %d)" % st)
    return f


def neighbors(box, x, rcut, method="cells", time=0.0):
    """Neighbour sets as CSR (row_ptr, cols) in id order."""
    _le(time)
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    L = _f64(box)
    cap = max(64, n * 16)
    fn = lib().orc_neighbors_cells if method == "cells" else lib().orc_neighbors_brute
    while True:
        row = np.zeros(n + 1, dtype=np.int64)
        cols = np.zeros(cap, dtype=np.int64)
        m = fn(n, _p(L, _dp), _p(x, _dp), rcut, _p(row, _i64p), _p(cols, _i64p), cap)
        if m >= 0:
            return row, cols[:m]
        cap *= 4


class State:
    """Particle state in id order: x, v (n,3) float64, img (n,3) int32."""

    def __init__(self, box, x, v=None, img=None, types=None, bonds=None):
        self.box = _f64(box).copy()
        self.x = _f64(x, (-1, 3)).copy()
        n = self.x.shape[0]
        self.v = _f64(v, (-1, 3)).copy() if v is not None else np.zeros((n, 3))
        self.img = (np.ascontiguousarray(img, dtype=np.int32).reshape(-1, 3).copy()
                    if img is not None else np.zeros((n, 3), dtype=np.int32))
        self.types = (np.ascontiguousarray(types, dtype=np.int32).copy()
                      if types is not None else np.zeros(n, dtype=np.int32))
        self.bonds = (np.ascontiguousarray(bonds, dtype=np.int64).reshape(-1, 2).copy()
                      if bonds is not None else np.zeros((0, 2), dtype=np.int64))
        self.f = np.zeros((n, 3), dtype=np.float64)
        self.f_valid = False
        self.step = 0
        self.time = 0.0  # simulated time (Lees-Edwards offset)

    @property
    def n(self):
        return self.x.shape[0]


def integrate(model: Model, st: State, nsteps: int, dt: float, gamma: float, kT: float,
              seed: int):
    _le(st.time)
    rc = lib().orc_integrate(st.n, _p(st.box, _dp), _p(st.x, _dp), _p(st.v, _dp),
                             _p(st.img, _i32p), _p(st.types, _i32p), _p(model.masses, _dp),
                             model.ntypes, _p(model.pair, _dp), st.bonds.shape[0],
                             _p(st.bonds, _i64p), _p(model.bond, _dp), _p(st.f, _dp),
                             1 if st.f_valid else 0, dt, gamma, kT, seed, st.step, nsteps)
    if rc != 0:
        raise RuntimeError("oracle integrate failed with status %d" % rc)
    st.f_valid = True
    st.step += nsteps
    st.time = lib().orc_le_get_time()
    return st


def observables(model: Model, st: State) -> dict:
    _le(st.time)
    out = np.zeros(NOBS, dtype=np.float64)
    rc = lib().orc_observables(st.n, _p(st.box, _dp), _p(st.x, _dp), _p(st.v, _dp),
                               _p(st.img, _i32p), _p(st.types, _i32p), _p(model.masses, _dp),
                               model.ntypes, _p(model.pair, _dp), st.bonds.shape[0],
                               _p(st.bonds, _i64p), _p(model.bond, _dp), _p(out, _dp))
    if rc != 0:
        raise RuntimeError("oracle observables failed with status %d" % rc)
    return dict(zip(OBS_NAMES, out.tolist()))


def rdf_counts(box, x, rmax, nbins, time=0.0):
    _le(time)
    x = _f64(x, (-1, 3))
    L = _f64(box)
    c = np.zeros(nbins, dtype=np.int64)
    lib().orc_rdf_counts(x.shape[0], _p(L, _dp), _p(x, _dp), rmax, nbins, _p(c, _i64p))
    return c
