"""Thin ctypes binding of libespp_gb.so (include/espp.h).

The functions below carry the C names and only marshal arguments; every step of
the MD path runs in the library's CUDA kernels.  `System` is a convenience
wrapper over one handle that accepts numpy arrays (host) or CUDA torch tensors
(device).  There is no CPU fallback: if the library is missing or no GPU is
visible, the first call raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libespp_gb.so")

ESPP_OK = 0
ESPP_ERR_ARG = -1
ESPP_ERR_CUDA = -2
ESPP_ERR_LIST_OVERFLOW = -3
ESPP_ERR_BOND_BROKEN = -4
ESPP_ERR_NONFINITE = -5
ESPP_ERR_TIMEOUT = -6
ESPP_ERR_BOX_TOO_SMALL = -7
ESPP_ERR_STATE = -8
ESPP_ERR_IO = -9

ESPP_FP32 = 1
ESPP_FP64 = 2
ESPP_HOST = 0
ESPP_DEVICE = 1

ESPP_NONE = 0
ESPP_LJ = 1
ESPP_WCA = 2
ESPP_LJ_CAPPED = 3
ESPP_FENE = 4
ESPP_TAB_PAIR = 5
ESPP_TAB_BOND = 6
ESPP_MLP = 7
MLP_NPARAMS = 6337
ESPP_THERMO_LANGEVIN = 0
ESPP_THERMO_DPD = 1
ESPP_FORCES_VERLET = 0
ESPP_FORCES_CELLS = 1
STEP_SHAPES = 8
FORCE_SHAPES = 6
FORCE_SHAPE_NAMES = ("verlet_whole_cells", "verlet_half_cells", "verlet_third_cells", "cells",
                     "verlet_whole_cells_push", "verlet_third_cells_push")
ESPP_LIST_STORE_PLACE, ESPP_LIST_STORE_PUSH = 0, 1
# (int4 list groups per batch, resident blocks per SM, tiles per block) of each
# step-kernel shape, as include/espp.h lists them
STEP_SHAPE_TABLE = ((1, 8, 1), (2, 8, 1), (1, 12, 1), (1, 10, 1), (1, 5, 2), (1, 3, 3), (1, 2, 4), (1, 2, 5))

ERROR_NAMES = {
    ESPP_ERR_ARG: "ESPP_ERR_ARG", ESPP_ERR_CUDA: "ESPP_ERR_CUDA",
    ESPP_ERR_LIST_OVERFLOW: "ESPP_ERR_LIST_OVERFLOW", ESPP_ERR_BOND_BROKEN: "ESPP_ERR_BOND_BROKEN",
    ESPP_ERR_NONFINITE: "ESPP_ERR_NONFINITE", ESPP_ERR_TIMEOUT: "ESPP_ERR_TIMEOUT",
    ESPP_ERR_BOX_TOO_SMALL: "ESPP_ERR_BOX_TOO_SMALL", ESPP_ERR_STATE: "ESPP_ERR_STATE",
    ESPP_ERR_IO: "ESPP_ERR_IO",
}

# every symbol include/espp.h declares
EXPORTS = (
    "espp_system_create", "espp_batch_create", "espp_system_destroy", "espp_set_state",
    "espp_get_state", "espp_set_step", "espp_set_interaction", "espp_set_mass",
    "espp_build_neighbors", "espp_get_neighbors", "espp_compute_forces", "espp_integrate",
    "espp_observables", "espp_observables_batch", "espp_rdf_counts", "espp_checkpoint_save",
    "espp_checkpoint_load", "espp_last_error", "espp_error_word", "espp_num_particles",
    "espp_num_replicas", "espp_num_rebuilds", "espp_step", "espp_list_capacity",
    "espp_kernel_launches", "espp_langevin_noise", "espp_hilbert_ranks",
    "espp_set_kernel_timing", "espp_kernel_timing", "espp_set_graph_chunk", "espp_list_stats",
    "espp_rdf_counts_noalloc", "espp_set_resort_interval", "espp_mlp_set_weights",
    "espp_set_exclude_bonded", "espp_mlp_get_weights", "espp_mlp_train", "espp_mlp_loss_grad",
    "espp_cg_map", "espp_set_cell_subdivision", "espp_set_thermostat",
    "espp_set_lees_edwards", "espp_get_lees_edwards", "espp_set_force_method",
    "espp_tune_force_method", "espp_set_step_shape", "espp_tune_step_shape",
    "espp_h5md_write", "espp_h5md_read", "espp_h5md_inspect", "espp_set_list_store",
)
NOALLOC_MAX_BINS = 4096
NOALLOC_MAX_N = 200000


class EsppError(RuntimeError):
    def __init__(self, code, msg):
        self.code = code
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "?"), code, msg))


class ReplicaDesc(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("n", ctypes.c_int64),
                ("types", ctypes.c_void_p), ("n_bonds", ctypes.c_int64),
                ("bonds", ctypes.c_void_p), ("seed", ctypes.c_uint64)]


class Obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("n", ctypes.c_int64),
                ("ke", ctypes.c_double), ("pe_pair", ctypes.c_double),
                ("pe_bond", ctypes.c_double), ("virial", ctypes.c_double),
                ("px", ctypes.c_double), ("py", ctypes.c_double), ("pz", ctypes.c_double),
                ("temperature", ctypes.c_double), ("pressure", ctypes.c_double),
                ("mean_bond", ctypes.c_double), ("rg2", ctypes.c_double),
                ("n_molecules", ctypes.c_int64), ("n_rebuilds", ctypes.c_int64),
                ("error_word", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("pxz", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None


def lib(path: str = LIB_PATH):
    """Load libespp_gb.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libespp_gb.so is not built (%s); run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    vp, dp, i64, i32 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int32
    sig = {
        "espp_system_create": ([dp, i64, vp, i64, vp, ctypes.c_int, ctypes.c_uint64, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "espp_batch_create": ([i32, ctypes.POINTER(ReplicaDesc), ctypes.c_int, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "espp_system_destroy": ([vp], ctypes.c_int),
        "espp_set_state": ([vp, vp, vp, vp, ctypes.c_int], ctypes.c_int),
        "espp_get_state": ([vp, vp, vp, vp, ctypes.c_int], ctypes.c_int),
        "espp_set_step": ([vp, i64], ctypes.c_int),
        "espp_set_interaction": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, i64], ctypes.c_int),
        "espp_set_mass": ([vp, ctypes.c_int, ctypes.c_double], ctypes.c_int),
        "espp_build_neighbors": ([vp, ctypes.c_double, ctypes.c_double], ctypes.c_int),
        "espp_get_neighbors": ([vp, vp, vp, i64], ctypes.c_int),
        "espp_compute_forces": ([vp, vp, ctypes.c_int], ctypes.c_int),
        "espp_integrate": ([vp, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double], ctypes.c_int),
        "espp_observables": ([vp, ctypes.POINTER(Obs)], ctypes.c_int),
        "espp_observables_batch": ([vp, ctypes.POINTER(Obs), i32], ctypes.c_int),
        "espp_rdf_counts": ([vp, i32, ctypes.c_double, i32, vp], ctypes.c_int),
        "espp_checkpoint_save": ([vp, ctypes.c_char_p], ctypes.c_int),
        "espp_checkpoint_load": ([vp, ctypes.c_char_p], ctypes.c_int),
        "espp_last_error": ([vp], ctypes.c_char_p),
        "espp_error_word": ([vp], ctypes.c_uint32),
        "espp_num_particles": ([vp], i64),
        "espp_num_replicas": ([vp], i32),
        "espp_num_rebuilds": ([vp], i64),
        "espp_step": ([vp], i64),
        "espp_list_capacity": ([vp], i32),
        "espp_kernel_launches": ([vp], i64),
        "espp_langevin_noise": ([ctypes.c_uint64, i64, i64, vp, vp], ctypes.c_int),
        "espp_hilbert_ranks": ([i32, i32, i32, vp], ctypes.c_int),
        "espp_set_kernel_timing": ([vp, ctypes.c_int], ctypes.c_int),
        "espp_kernel_timing": ([vp, dp, ctypes.c_int], ctypes.c_int),
        "espp_set_graph_chunk": ([vp, i32], ctypes.c_int),
        "espp_list_stats": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i32)], ctypes.c_int),
        "espp_rdf_counts_noalloc": ([vp, i64, dp, ctypes.c_double, i32, vp, vp], ctypes.c_int),
        "espp_set_resort_interval": ([vp, i64], ctypes.c_int),
        "espp_set_cell_subdivision": ([vp, ctypes.c_int32], ctypes.c_int),
        "espp_set_thermostat": ([vp, ctypes.c_int32, ctypes.c_double], ctypes.c_int),
        "espp_set_lees_edwards": ([vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double], ctypes.c_int),
        "espp_get_lees_edwards": ([vp, ctypes.POINTER(ctypes.c_int32), dp, dp], ctypes.c_int),
        "espp_set_force_method": ([vp, ctypes.c_int32], ctypes.c_int),
        "espp_tune_force_method": ([vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
                                    ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "espp_set_step_shape": ([vp, ctypes.c_int32], ctypes.c_int),
        "espp_set_list_store": ([vp, ctypes.c_int32], ctypes.c_int),
        "espp_h5md_write": ([vp, ctypes.c_char_p], ctypes.c_int),
        "espp_h5md_read": ([vp, ctypes.c_char_p], ctypes.c_int),
        "espp_h5md_inspect": ([ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "espp_tune_step_shape": ([vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
                                  ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "espp_mlp_set_weights": ([vp, vp, i64], ctypes.c_int),
        "espp_set_exclude_bonded": ([vp, ctypes.c_int], ctypes.c_int),
        "espp_mlp_get_weights": ([vp, vp, i64], ctypes.c_int),
        "espp_mlp_train": ([vp, vp, vp, i32, i32, i32, ctypes.c_double, ctypes.c_uint64, vp], ctypes.c_int),
        "espp_mlp_loss_grad": ([vp, vp, vp, i32, vp, vp], ctypes.c_int),
        "espp_cg_map": ([vp, i32, vp, vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc, h=None):
    if rc != ESPP_OK:
        msg = lib().espp_last_error(h)
        raise EsppError(rc, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, where) for a numpy array or a torch tensor."""
    if a is None:
        return None, ESPP_HOST
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            return ctypes.c_void_p(a.data_ptr()), ESPP_DEVICE
        return ctypes.c_void_p(a.data_ptr()), ESPP_HOST
    return a.ctypes.data_as(ctypes.c_void_p), ESPP_HOST


# ---- the C calls, by name --------------------------------------------------------
def h5md_inspect(path):
    """What an H5MD file written by the library holds, without a handle (host
    only): {"replicas", "particles" (in total), "step", "precision"}.  A file
    the reader refuses raises EsppError (ESPP_ERR_IO)."""
    r, p = ctypes.c_int32(0), ctypes.c_int32(0)
    n, st = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().espp_h5md_inspect(os.fspath(path).encode(), ctypes.byref(r), ctypes.byref(n), ctypes.byref(st),
                                   ctypes.byref(p)))
    return {"replicas": r.value, "particles": n.value, "step": st.value, "precision": p.value}


def espp_hilbert_ranks(nx, ny, nz):
    out = np.zeros(nx * ny * nz, dtype=np.int32)
    _check(lib().espp_hilbert_ranks(nx, ny, nz, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def espp_langevin_noise(seed, step, out_tensor, stream=0):
    n = out_tensor.numel() // 3
    _check(lib().espp_langevin_noise(seed, step, n, ctypes.c_void_p(out_tensor.data_ptr()),
                                     ctypes.c_void_p(stream)))


def to_bf16_bits(a):
    """float -> BF16 bit patterns (round to nearest even), as uint16."""
    f = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (f + 0x7FFF + ((f >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def bf16_bits_to_float(b):
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def espp_rdf_counts_noalloc(x_device, box, rmax, counts_device, stream=0):
    """Pair-distance histogram from device positions into device counts,
    without any allocation inside the library (see include/espp.h).

    x_device: contiguous CUDA float64 tensor of shape (n, 3); counts_device:
    contiguous CUDA int64 tensor on the same device, one entry per bin.  The
    library reads and writes these buffers by raw address, so anything else is
    refused here (ValueError) before the call."""
    import torch
    if not (isinstance(x_device, torch.Tensor) and isinstance(counts_device, torch.Tensor)):
        raise ValueError("x_device and counts_device must be torch tensors")
    if not (x_device.is_cuda and counts_device.is_cuda) or x_device.device != counts_device.device:
        raise ValueError("x_device and counts_device must be CUDA tensors on the same device")
    if x_device.dtype != torch.float64 or x_device.dim() != 2 or x_device.shape[1] != 3 \
            or not x_device.is_contiguous():
        raise ValueError("x_device must be a contiguous float64 tensor of shape (n, 3)")
    if counts_device.dtype != torch.int64 or counts_device.dim() != 1 or not counts_device.is_contiguous():
        raise ValueError("counts_device must be a contiguous one-dimensional int64 tensor")
    n = x_device.shape[0]
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    _check(lib().espp_rdf_counts_noalloc(ctypes.c_void_p(x_device.data_ptr()), n, b, float(rmax),
                                         counts_device.numel(),
                                         ctypes.c_void_p(counts_device.data_ptr()),
                                         ctypes.c_void_p(stream)))


class System:
    """One handle: a single system or a batch of independent replicas."""

    def __init__(self, box=None, n=None, types=None, bonds=None, precision=ESPP_FP32, seed=42,
                 stream=0, replicas=None):
        L = lib()
        self._h = ctypes.c_void_p()
        self.precision = precision
        keep = []
        if replicas is None:
            replicas = [dict(box=box, n=n, types=types, bonds=bonds, seed=seed)]
        descs = (ReplicaDesc * len(replicas))()
        self.rep_n = []
        for k, r in enumerate(replicas):
            t = None if r.get("types") is None else np.ascontiguousarray(r["types"], dtype=np.int32)
            b = None
            if r.get("bonds") is not None and len(r["bonds"]) > 0:
                b = np.ascontiguousarray(r["bonds"], dtype=np.int64).reshape(-1, 2)
            keep += [t, b]
            d = descs[k]
            for c in range(3):
                d.box[c] = float(np.asarray(r["box"], dtype=np.float64)[c])
            d.n = int(r["n"])
            d.types = t.ctypes.data if t is not None else None
            d.n_bonds = 0 if b is None else b.shape[0]
            d.bonds = b.ctypes.data if b is not None else None
            d.seed = int(r.get("seed", 42))
            self.rep_n.append(int(r["n"]))
        rc = L.espp_batch_create(len(replicas), descs, precision, ctypes.c_void_p(stream),
                                 ctypes.byref(self._h))
        _check(rc, None)
        self.n = sum(self.rep_n)
        self.R = len(replicas)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().espp_system_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, rc):
        _check(rc, self._h)

    # state
    def set_state(self, x, v=None, img=None):
        if not hasattr(x, "data_ptr"):
            x = np.ascontiguousarray(x, dtype=np.float64)
            v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
            img = None if img is None else np.ascontiguousarray(img, dtype=np.int32)
        px, where = _ptr(x)
        pv, _ = _ptr(v)
        pi, _ = _ptr(img)
        self._c(lib().espp_set_state(self._h, px, pv, pi, where))

    def get_state(self, out=None):
        if out is not None:
            x, v, img = out
            px, where = _ptr(x)
            self._c(lib().espp_get_state(self._h, px, _ptr(v)[0], _ptr(img)[0], where))
            return out
        x = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        img = np.zeros((self.n, 3), dtype=np.int32)
        self._c(lib().espp_get_state(self._h, _ptr(x)[0], _ptr(v)[0], _ptr(img)[0], ESPP_HOST))
        return x, v, img

    def set_step(self, step):
        self._c(lib().espp_set_step(self._h, int(step)))

    # interactions
    def set_interaction(self, kind, ta=0, tb=0, params=()):
        p = (ctypes.c_double * max(1, len(params)))(*params)
        self._c(lib().espp_set_interaction(self._h, kind, ta, tb, p, len(params)))

    def set_lj(self, eps, sigma, rc, shift=True, ta=0, tb=0):
        self.set_interaction(ESPP_LJ, ta, tb, (eps, sigma, rc, 1.0 if shift else 0.0))

    def set_wca(self, eps=1.0, sigma=1.0, ta=0, tb=0):
        self.set_interaction(ESPP_WCA, ta, tb, (eps, sigma))

    def set_lj_capped(self, eps, sigma, rc, caprad, shift=True, ta=0, tb=0):
        self.set_interaction(ESPP_LJ_CAPPED, ta, tb, (eps, sigma, rc, 1.0 if shift else 0.0, caprad))

    def set_fene(self, K=30.0, R0=1.5):
        self.set_interaction(ESPP_FENE, 0, 0, (K, R0))

    def set_table_pair(self, rc, u, f, ta=0, tb=0):
        """Tabulated pair potential: u and F = -dU/dr at r_k = k rc / (n-1)."""
        u = np.asarray(u, dtype=np.float64)
        f = np.asarray(f, dtype=np.float64)
        self.set_interaction(ESPP_TAB_PAIR, ta, tb, [rc, float(u.size)] + u.tolist() + f.tolist())

    def set_table_bond(self, rmax, u, f):
        u = np.asarray(u, dtype=np.float64)
        f = np.asarray(f, dtype=np.float64)
        self.set_interaction(ESPP_TAB_BOND, 0, 0, [rmax, float(u.size)] + u.tolist() + f.tolist())

    def set_mlp(self, rc, bf16_bits):
        """Learned pair potential: cutoff rc and ESPP_MLP_NPARAMS BF16 weights."""
        b = np.ascontiguousarray(bf16_bits, dtype=np.uint16)
        self._c(lib().espp_mlp_set_weights(self._h, b.ctypes.data_as(ctypes.c_void_p), b.size))
        self.set_interaction(ESPP_MLP, 0, 0, (rc,))

    def cg_map(self, beads_per_site, x_out, f_out):
        """Map onto sites of consecutive beads into CUDA float64 tensors."""
        self._c(lib().espp_cg_map(self._h, beads_per_site, ctypes.c_void_p(x_out.data_ptr()),
                                  ctypes.c_void_p(f_out.data_ptr())))

    def mlp_weights(self):
        out = np.zeros(MLP_NPARAMS, dtype=np.uint16)
        self._c(lib().espp_mlp_get_weights(self._h, out.ctypes.data_as(ctypes.c_void_p), MLP_NPARAMS))
        return out

    def mlp_train(self, frames_x, frames_f, batch_frames, epochs, lr, seed=4):
        """frames_x, frames_f: CUDA float64 tensors (nframes, n, 3)."""
        loss = np.zeros(epochs)
        self._c(lib().espp_mlp_train(self._h, ctypes.c_void_p(frames_x.data_ptr()),
                                     ctypes.c_void_p(frames_f.data_ptr()), frames_x.shape[0], batch_frames,
                                     epochs, lr, seed, loss.ctypes.data_as(ctypes.c_void_p)))
        return loss

    def mlp_loss_grad(self, frames_x, frames_f):
        loss = np.zeros(1)
        grad = np.zeros(MLP_NPARAMS - 1, dtype=np.float32)
        self._c(lib().espp_mlp_loss_grad(self._h, ctypes.c_void_p(frames_x.data_ptr()),
                                         ctypes.c_void_p(frames_f.data_ptr()), frames_x.shape[0],
                                         loss.ctypes.data_as(ctypes.c_void_p),
                                         grad.ctypes.data_as(ctypes.c_void_p)))
        return float(loss[0]), grad.astype(np.float64)

    def set_exclude_bonded(self, on=True):
        self._c(lib().espp_set_exclude_bonded(self._h, 1 if on else 0))

    def set_mass(self, t, m):
        self._c(lib().espp_set_mass(self._h, t, m))

    # neighbours, forces, dynamics
    def build_neighbors(self, rc, skin):
        self._c(lib().espp_build_neighbors(self._h, rc, skin))

    def get_neighbors(self):
        row = np.zeros(self.n + 1, dtype=np.int64)
        rc = lib().espp_get_neighbors(self._h, _ptr(row)[0], None, 0)
        need = int(row[-1])
        cols = np.zeros(max(need, 1), dtype=np.int64)
        self._c(lib().espp_get_neighbors(self._h, _ptr(row)[0], _ptr(cols)[0], cols.size))
        return row, cols[:need]

    def compute_forces(self, out=None):
        if out is None:
            out = np.zeros((self.n, 3))
        p, where = _ptr(out)
        self._c(lib().espp_compute_forces(self._h, p, where))
        return out

    def integrate(self, nsteps, dt, gamma, kT):
        self._c(lib().espp_integrate(self._h, int(nsteps), dt, gamma, kT))

    def observables(self, replica=None):
        out = (Obs * self.R)()
        self._c(lib().espp_observables_batch(self._h, out, self.R))
        if replica is None:
            return out[0].as_dict() if self.R == 1 else [o.as_dict() for o in out]
        return out[replica].as_dict()

    def rdf_counts(self, rmax, nbins, replica=0):
        c = np.zeros(nbins, dtype=np.int64)
        self._c(lib().espp_rdf_counts(self._h, replica, rmax, nbins, _ptr(c)[0]))
        return c

    def h5md_write(self, path):
        """The state as an H5MD file (see include/espp.h)."""
        self._c(lib().espp_h5md_write(self._h, os.fspath(path).encode()))

    def h5md_read(self, path):
        self._c(lib().espp_h5md_read(self._h, os.fspath(path).encode()))

    def checkpoint_save(self, path):
        self._c(lib().espp_checkpoint_save(self._h, path.encode()))

    def checkpoint_load(self, path):
        self._c(lib().espp_checkpoint_load(self._h, path.encode()))

    # timing
    def set_kernel_timing(self, enable=True):
        self._c(lib().espp_set_kernel_timing(self._h, 1 if enable else 0))

    def kernel_timing(self, reset=False):
        out = (ctypes.c_double * 4)()
        self._c(lib().espp_kernel_timing(self._h, out, 1 if reset else 0))
        return dict(step_ms=out[0], step_launches=int(out[1]), rebuild_ms=out[2], steps=int(out[3]))

    def list_stats(self):
        t, m = ctypes.c_int64(), ctypes.c_int32()
        self._c(lib().espp_list_stats(self._h, ctypes.byref(t), ctypes.byref(m)))
        return int(t.value), int(m.value)

    def set_resort_interval(self, steps):
        self._c(lib().espp_set_resort_interval(self._h, int(steps)))

    def set_cell_subdivision(self, w):
        self._c(lib().espp_set_cell_subdivision(self._h, int(w)))

    def set_thermostat(self, kind, rc=0.0):
        """ESPP_THERMO_LANGEVIN, or ESPP_THERMO_DPD with pair cutoff rc."""
        self._c(lib().espp_set_thermostat(self._h, int(kind), float(rc)))

    def set_lees_edwards(self, on, shear_rate=0.0, time=None):
        """Lees-Edwards shear (flow x, gradient z); time defaults to the
        handle's current simulated time."""
        if time is None:
            time = self.lees_edwards()[2]
        self._c(lib().espp_set_lees_edwards(self._h, 1 if on else 0, float(shear_rate), float(time)))

    def lees_edwards(self):
        """(on, shear_rate, simulated time)."""
        on, sh, t = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
        self._c(lib().espp_get_lees_edwards(self._h, ctypes.byref(on), ctypes.byref(sh), ctypes.byref(t)))
        return bool(on.value), sh.value, t.value

    def set_force_method(self, method):
        """ESPP_FORCES_VERLET (the list) or ESPP_FORCES_CELLS (list-free)."""
        self._c(lib().espp_set_force_method(self._h, int(method)))

    def tune_force_method(self, nsteps, dt, gamma, kT):
        """Time the FORCE_SHAPES shapes (Verlet over whole, half or third
        cells, list-free cells, whole and third cells with pushed list
        stores) from the current state and keep the fastest; returns (ms per
        step of each, chosen shape index)."""
        ms = (ctypes.c_double * FORCE_SHAPES)()
        ch = ctypes.c_int32()
        self._c(lib().espp_tune_force_method(self._h, int(nsteps), float(dt), float(gamma), float(kT), ms,
                                             ctypes.byref(ch)))
        return list(ms), int(ch.value)

    def set_step_shape(self, shape):
        self._c(lib().espp_set_step_shape(self._h, int(shape)))

    def set_list_store(self, push):
        """ESPP_LIST_STORE_PLACE or ESPP_LIST_STORE_PUSH (the same lists)."""
        self._c(lib().espp_set_list_store(self._h, int(push)))

    def tune_step_shape(self, nsteps, dt, gamma, kT):
        """Time the step kernel's launch shapes, then the resort intervals
        (250, 500, 1000 steps), from the current state and keep the fastest;
        returns (ms per step of each shape, ms per step of each interval,
        (shape kept, interval kept))."""
        ms = (ctypes.c_double * (STEP_SHAPES + 3))()
        ch = (ctypes.c_int32 * 2)()
        self._c(lib().espp_tune_step_shape(self._h, int(nsteps), float(dt), float(gamma), float(kT), ms, ch))
        return list(ms)[:STEP_SHAPES], list(ms)[STEP_SHAPES:], (int(ch[0]), int(ch[1]))

    def set_graph_chunk(self, steps):
        self._c(lib().espp_set_graph_chunk(self._h, int(steps)))

    # diagnostics
    @property
    def error_word(self):
        return int(lib().espp_error_word(self._h))

    @property
    def step(self):
        return int(lib().espp_step(self._h))

    @property
    def n_rebuilds(self):
        return int(lib().espp_num_rebuilds(self._h))

    @property
    def list_capacity(self):
        return int(lib().espp_list_capacity(self._h))

    @property
    def kernel_launches(self):
        return int(lib().espp_kernel_launches(self._h))
