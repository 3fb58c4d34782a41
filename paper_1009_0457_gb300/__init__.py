"""Python binding of libhmc, the GB300 (sm_103a) hybrid Monte Carlo library.

Argument marshalling only: every step of the method runs in the CUDA kernels
behind the C ABI declared in ``include/hmc.h``.  The functions below carry the
C names (``hmc_create``, ``hmc_set_orientations``, ``hmc_mpm_steps``,
``hmc_mc_sweeps``, ``hmc_texture_histogram``, ...) and take numpy arrays;
``HMC`` wraps one handle.  Importing this module loads ``libhmc.so`` and raises
if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhmc.so")

HMC_OK, HMC_ERR_ARG, HMC_ERR_CUDA, HMC_ERR_OOM, HMC_ERR_STATE, HMC_ERR_NONFINITE, HMC_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
HMC_BC_UNIAXIAL, HMC_BC_STRAIN6, HMC_BC_TRACTION = 0, 1, 2
HMC_ELASTIC_OFF, HMC_ELASTIC_TRACTION, HMC_ELASTIC_ZONE1, HMC_ELASTIC_STRAIN = 0, 1, 2, 3
HMC_TRIAL_NEIGHBOR, HMC_TRIAL_UNIFORM_Q = 0, 1
HMC_FP64, HMC_FP32 = 0, 1
HMC_HIST_PER_Q, HMC_HIST_ANGLE_100, HMC_HIST_YOUNG = 0, 1, 2


class hmc_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("n_orient", C.c_int32),
        ("J", C.c_double), ("kT", C.c_double),
        ("c11", C.c_double), ("c12", C.c_double), ("c44", C.c_double),
        ("bc", C.c_int32),
        ("load_axis", C.c_double * 3),
        ("strain", C.c_double),
        ("strain6", C.c_double * 6),
        ("elastic_scale", C.c_double),
        ("elastic", C.c_int32),
        ("trial", C.c_int32),
        ("mpm_steps_per_mcs", C.c_int32),
        ("dt", C.c_double), ("damping", C.c_double),
        ("precision", C.c_int32),
        ("seed", C.c_uint64),
        ("replica", C.c_uint32),
        ("stream", C.c_void_p),
        ("stress", C.c_double),
        ("store_stress", C.c_int32),
    ]


class hmc_info(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("damping", C.c_double), ("elastic_scale", C.c_double),
        ("strain_bar", C.c_double * 6),
        ("mcs", C.c_uint32), ("u_buffer", C.c_int32),
        ("n_sites", C.c_int64), ("n_nodes", C.c_int64),
        ("zone_trials", C.c_int64),
    ]


class HMCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hmc status {status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhmc.so not built ({LIB_PATH}); run paper_1009_0457_gb300/build.py "
                          "or __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    H = C.c_void_p
    st = C.c_int
    dp, i64p, u16p = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_uint16)
    sig = {
        "hmc_default_params": (None, [C.POINTER(hmc_params)]),
        "hmc_create": (st, [C.POINTER(hmc_params), C.POINTER(H)]),
        "hmc_create_batch": (st, [C.POINTER(hmc_params), C.c_int32, C.POINTER(H)]),
        "hmc_select_replica": (st, [H, C.c_int32]),
        "hmc_get_tuning": (st, [H, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "hmc_get_sweep_tuning": (st, [H, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "hmc_fma_peak": (st, [C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
        "hmc_destroy": (None, [H]),
        "hmc_set_orientations": (st, [H, dp, u16p]),
        "hmc_set_spins": (st, [H, u16p]),
        "hmc_get_spins": (st, [H, u16p]),
        "hmc_mpm_steps": (st, [H, C.c_int32, dp]),
        "hmc_mpm_steps_plain": (st, [H, C.c_int32]),
        "hmc_compute_stress": (st, [H, dp, dp]),
        "hmc_sweep_half": (st, [H, C.c_int32, i64p]),
        "hmc_sweep_half_margins": (st, [H, C.c_int32, dp, i64p]),
        "hmc_end_mcs": (st, [H]),
        "hmc_mc_sweeps": (st, [H, C.c_int32, i64p]),
        "hmc_texture_histogram": (st, [H, C.c_int32, C.c_int32, dp, i64p]),
        "hmc_energy": (st, [H, i64p, dp, dp]),
        "hmc_grain_count": (st, [H, i64p]),
        "hmc_get_stress": (st, [H, dp]),
        "hmc_set_stress": (st, [H, dp]),
        "hmc_get_nodal": (st, [H, dp, dp]),
        "hmc_set_nodal": (st, [H, dp, dp]),
        "hmc_get_strain": (st, [H, dp]),
        "hmc_set_strain": (st, [H, dp]),
        "hmc_set_spins_dev": (st, [H, C.c_void_p]),
        "hmc_get_spins_dev": (st, [H, C.c_void_p]),
        "hmc_set_orientations_dev": (st, [H, dp, C.c_void_p]),
        "hmc_set_load": (st, [H, C.c_double]),
        "hmc_get_info": (st, [H, C.POINTER(hmc_info)]),
        "hmc_get_state": (st, [H, C.c_void_p, C.POINTER(C.c_size_t)]),
        "hmc_set_state": (st, [H, C.c_void_p, C.c_size_t]),
        "hmc_synchronize": (st, [H]),
        "hmc_adjoint_forward": (st, [H, C.c_int32, C.c_int32, dp, dp]),
        "hmc_adjoint_backward": (st, [H, C.c_double, dp, dp]),
        "hmc_stress_noalloc": (st, [C.c_void_p, C.c_void_p, C.c_void_p, dp, C.c_int32, C.c_int32, C.c_int32,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
        "hmc_last_error": (C.c_char_p, [H]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def _check(h, status):
    if status != HMC_OK:
        raise HMCError(status, lib.hmc_last_error(h).decode())


# --- thin wrappers with the C names ------------------------------------------

def hmc_default_params(**overrides) -> hmc_params:
    p = hmc_params()
    lib.hmc_default_params(C.byref(p))
    for k, v in overrides.items():
        if k in ("load_axis", "strain6"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = float(x)
        else:
            setattr(p, k, v)
    return p


def hmc_create(p: hmc_params):
    h = C.c_void_p()
    _check(None, lib.hmc_create(C.byref(p), C.byref(h)))
    return h


def hmc_create_batch(params):
    """One handle over len(params) replicas (a sequence of hmc_params)."""
    arr = (hmc_params * len(params))(*params)
    h = C.c_void_p()
    _check(None, lib.hmc_create_batch(arr, len(params), C.byref(h)))
    return h


def hmc_select_replica(h, r):
    _check(h, lib.hmc_select_replica(h, int(r)))


def hmc_fma_peak(precision, iters=4096):
    """Measured peak FMA rate of the current device in TFLOP/s (FP32 or FP64)."""
    t = C.c_double(0.0)
    _check(None, lib.hmc_fma_peak(int(precision), int(iters), C.byref(t)))
    return t.value


def hmc_get_sweep_tuning(h):
    """(threads per sweep CTA, 1 if the sweeps read stored stress else 0)."""
    c, st_ = C.c_int32(0), C.c_int32(0)
    _check(h, lib.hmc_get_sweep_tuning(h, C.byref(c), C.byref(st_)))
    return c.value, st_.value


def hmc_get_tuning(h):
    s, g = C.c_int32(), C.c_int32()
    _check(h, lib.hmc_get_tuning(h, C.byref(s), C.byref(g)))
    return s.value, g.value


def hmc_destroy(h):
    lib.hmc_destroy(h)


def hmc_set_orientations(h, euler, spins):
    e = np.ascontiguousarray(euler, dtype=np.float64)
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    _check(h, lib.hmc_set_orientations(h, _ptr(e, C.c_double), _ptr(s, C.c_uint16)))


def hmc_set_spins(h, spins):
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    _check(h, lib.hmc_set_spins(h, _ptr(s, C.c_uint16)))


def hmc_set_spins_dev(h, d_spins):
    """d_spins: device address (int) of N uint16 values, e.g. a tensor's data_ptr()."""
    _check(h, lib.hmc_set_spins_dev(h, C.c_void_p(int(d_spins))))


def hmc_get_spins_dev(h, d_spins):
    _check(h, lib.hmc_get_spins_dev(h, C.c_void_p(int(d_spins))))


def hmc_set_orientations_dev(h, euler, d_spins):
    e = np.ascontiguousarray(euler, dtype=np.float64)
    _check(h, lib.hmc_set_orientations_dev(h, _ptr(e, C.c_double), C.c_void_p(int(d_spins))))


def hmc_get_spins(h, out):
    assert out.dtype == np.uint16 and out.flags.c_contiguous
    _check(h, lib.hmc_get_spins(h, _ptr(out, C.c_uint16)))
    return out


def hmc_mpm_steps(h, nsteps, want_energy=False):
    e = np.zeros(1) if want_energy else None
    _check(h, lib.hmc_mpm_steps(h, int(nsteps), _ptr(e, C.c_double)))
    return None if e is None else float(e[0])


def hmc_mpm_steps_plain(h, nsteps):
    _check(h, lib.hmc_mpm_steps_plain(h, int(nsteps)))


def hmc_compute_stress(h):
    m, e = np.zeros(6), np.zeros(1)
    _check(h, lib.hmc_compute_stress(h, _ptr(m, C.c_double), _ptr(e, C.c_double)))
    return m, float(e[0])


def hmc_sweep_half(h, colour):
    a = np.zeros(1, dtype=np.int64)
    _check(h, lib.hmc_sweep_half(h, int(colour), _ptr(a, C.c_int64)))
    return int(a[0])


def hmc_sweep_half_margins(h, colour, n_sites):
    """(accepted, margin): margin[i] = (H - t) / max(1, |t|) of site i's elastic trial, NaN elsewhere."""
    a = np.zeros(1, dtype=np.int64)
    m = np.empty(n_sites)
    _check(h, lib.hmc_sweep_half_margins(h, int(colour), _ptr(m, C.c_double), _ptr(a, C.c_int64)))
    return int(a[0]), m


def hmc_end_mcs(h):
    _check(h, lib.hmc_end_mcs(h))


def hmc_mc_sweeps(h, n_mcs, want_accepted=True):
    a = np.zeros(1, dtype=np.int64) if want_accepted else None
    _check(h, lib.hmc_mc_sweeps(h, int(n_mcs), _ptr(a, C.c_int64)))
    return None if a is None else int(a[0])


def hmc_texture_histogram(h, kind, nbins, n_orient):
    f = np.zeros(nbins)
    c = np.zeros(n_orient, dtype=np.int64)
    _check(h, lib.hmc_texture_histogram(h, int(kind), int(nbins), _ptr(f, C.c_double), _ptr(c, C.c_int64)))
    return f, c


def hmc_energy(h):
    u = np.zeros(1, dtype=np.int64)
    e = np.zeros(1)
    m = np.zeros(6)
    _check(h, lib.hmc_energy(h, _ptr(u, C.c_int64), _ptr(e, C.c_double), _ptr(m, C.c_double)))
    return int(u[0]), float(e[0]), m


def hmc_grain_count(h):
    n = np.zeros(1, dtype=np.int64)
    _check(h, lib.hmc_grain_count(h, _ptr(n, C.c_int64)))
    return int(n[0])


def hmc_get_stress(h, n_sites):
    out = np.zeros((n_sites, 6))
    _check(h, lib.hmc_get_stress(h, _ptr(out, C.c_double)))
    return out


def hmc_set_stress(h, sigma):
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    _check(h, lib.hmc_set_stress(h, _ptr(s, C.c_double)))


def hmc_get_nodal(h, n_nodes):
    u, v = np.zeros((n_nodes, 3)), np.zeros((n_nodes, 3))
    _check(h, lib.hmc_get_nodal(h, _ptr(u, C.c_double), _ptr(v, C.c_double)))
    return u, v


def hmc_set_nodal(h, u, v):
    u = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    _check(h, lib.hmc_set_nodal(h, _ptr(u, C.c_double), _ptr(v, C.c_double)))


def hmc_get_strain(h):
    e = np.zeros(6)
    _check(h, lib.hmc_get_strain(h, _ptr(e, C.c_double)))
    return e


def hmc_set_strain(h, e):
    e = np.ascontiguousarray(e, dtype=np.float64)
    _check(h, lib.hmc_set_strain(h, _ptr(e, C.c_double)))


def hmc_set_load(h, value):
    _check(h, lib.hmc_set_load(h, float(value)))


def hmc_get_info(h) -> hmc_info:
    i = hmc_info()
    _check(h, lib.hmc_get_info(h, C.byref(i)))
    return i


def hmc_get_state(h) -> bytes:
    n = C.c_size_t(0)
    _check(h, lib.hmc_get_state(h, None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(h, lib.hmc_get_state(h, buf, C.byref(n)))
    return buf.raw[:n.value]


def hmc_set_state(h, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(h, lib.hmc_set_state(h, buf, len(blob)))


def hmc_stress_noalloc(d_spins, d_u, d_ctab, strain_bar, nx, ny, nz, d_sigma, d_mean, d_energy, stream=None):
    """Allocation-free stress pass on caller-owned device buffers (integer device
    pointers, e.g. ``tensor.data_ptr()``); see include/hmc.h."""
    e = np.ascontiguousarray(strain_bar, dtype=np.float64)
    _check(None, lib.hmc_stress_noalloc(d_spins, d_u, d_ctab, _ptr(e, C.c_double), int(nx), int(ny), int(nz),
                                        d_sigma, d_mean, d_energy, stream))


def hmc_adjoint_forward(h, nsteps, checkpoint_every, n_sites=None):
    """Run the MPM map keeping checkpoints; returns (W, w field or None)."""
    W = np.zeros(1)
    w = None if n_sites is None else np.zeros(n_sites)
    _check(h, lib.hmc_adjoint_forward(h, int(nsteps), int(checkpoint_every), _ptr(W, C.c_double), _ptr(w, C.c_double)))
    return float(W[0]), w


def hmc_adjoint_backward(h, gW, g_field=None):
    """d(gW W + g.w)/d(C11, C12, C44, Ebar_1..6) after hmc_adjoint_forward."""
    g = None if g_field is None else np.ascontiguousarray(g_field, dtype=np.float64).reshape(-1)
    out = np.zeros(9)
    _check(h, lib.hmc_adjoint_backward(h, float(gW), _ptr(g, C.c_double), _ptr(out, C.c_double)))
    return out


def hmc_last_error(h=None) -> str:
    return lib.hmc_last_error(h).decode()


def hmc_synchronize(h):
    _check(h, lib.hmc_synchronize(h))


class HMC:
    """One replica behind one handle.  ``shape`` is (nz, ny, nx)."""

    def __init__(self, shape, n_orient, **params):
        nz, ny, nx = shape
        self.shape = tuple(shape)
        self.n_orient = n_orient
        self.p = hmc_default_params(nx=nx, ny=ny, nz=nz, n_orient=n_orient, **params)
        self.h = hmc_create(self.p)
        self.n_sites = nx * ny * nz
        self.n_nodes = self.n_sites // 8

    def tuning(self):
        return hmc_get_tuning(self.h)

    def sweep_tuning(self):
        return hmc_get_sweep_tuning(self.h)

    def adjoint_forward(self, nsteps, checkpoint_every, want_field=True):
        return hmc_adjoint_forward(self.h, nsteps, checkpoint_every, self.n_sites if want_field else None)

    def adjoint_backward(self, gW, g_field=None):
        return hmc_adjoint_backward(self.h, gW, g_field)

    def close(self):
        if self.h:
            hmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_orientations(self, euler, spins):
        hmc_set_orientations(self.h, euler, np.asarray(spins).reshape(-1))

    def set_spins(self, spins):
        hmc_set_spins(self.h, np.asarray(spins).reshape(-1))

    def spins(self):
        return hmc_get_spins(self.h, np.zeros(self.n_sites, dtype=np.uint16)).reshape(self.shape)

    def mpm_steps(self, n, want_energy=False):
        return hmc_mpm_steps(self.h, n, want_energy)

    def mpm_steps_plain(self, n):
        hmc_mpm_steps_plain(self.h, n)

    def compute_stress(self):
        return hmc_compute_stress(self.h)

    def sweep_half(self, colour):
        return hmc_sweep_half(self.h, colour)

    def sweep_half_margins(self, colour):
        acc, m = hmc_sweep_half_margins(self.h, colour, self.n_sites)
        return acc, m.reshape(self.shape)

    def end_mcs(self):
        hmc_end_mcs(self.h)

    def mc_sweeps(self, n):
        return hmc_mc_sweeps(self.h, n)

    def texture_histogram(self, kind, nbins):
        return hmc_texture_histogram(self.h, kind, nbins, self.n_orient)

    def energy(self):
        return hmc_energy(self.h)

    def grain_count(self):
        return hmc_grain_count(self.h)

    def stress(self):
        return hmc_get_stress(self.h, self.n_sites)

    def set_stress(self, sigma):
        hmc_set_stress(self.h, sigma)

    def nodal(self):
        return hmc_get_nodal(self.h, self.n_nodes)

    def set_nodal(self, u, v):
        hmc_set_nodal(self.h, u, v)

    def strain(self):
        return hmc_get_strain(self.h)

    def set_strain(self, e):
        hmc_set_strain(self.h, e)

    def set_load(self, value):
        hmc_set_load(self.h, value)

    def info(self):
        return hmc_get_info(self.h)

    def state(self):
        return hmc_get_state(self.h)

    def set_state(self, blob):
        hmc_set_state(self.h, blob)

    def synchronize(self):
        hmc_synchronize(self.h)


class HMCBatch:
    """A batched ensemble: replica r has shape shapes[r] = (nz, ny, nx) and the
    keyword overrides per_replica[r]; ``common`` applies to all."""

    def __init__(self, shapes, n_orient, per_replica=None, **common):
        self.shapes = [tuple(s) for s in shapes]
        self.n_orient = n_orient
        per_replica = per_replica or [{} for _ in shapes]
        self.params = []
        for (nz, ny, nx), kw in zip(self.shapes, per_replica):
            d = dict(common)
            d.update(kw)
            self.params.append(hmc_default_params(nx=nx, ny=ny, nz=nz, n_orient=n_orient, **d))
        self.h = hmc_create_batch(self.params)
        self.sel = 0

    def close(self):
        if self.h:
            hmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def select(self, r):
        hmc_select_replica(self.h, r)
        self.sel = r

    def set_orientations(self, euler, spins_list):
        flat = np.concatenate([np.asarray(s, dtype=np.uint16).reshape(-1) for s in spins_list])
        hmc_set_orientations(self.h, euler, flat)

    def spins(self, r):
        self.select(r)
        n = int(np.prod(self.shapes[r]))
        return hmc_get_spins(self.h, np.zeros(n, dtype=np.uint16)).reshape(self.shapes[r])

    def nodal(self, r):
        self.select(r)
        return hmc_get_nodal(self.h, int(np.prod(self.shapes[r])) // 8)

    def strain(self, r):
        self.select(r)
        return hmc_get_strain(self.h)

    def mc_sweeps(self, n):
        return hmc_mc_sweeps(self.h, n)

    def mpm_steps(self, n):
        return hmc_mpm_steps(self.h, n)

    def tuning(self):
        return hmc_get_tuning(self.h)

    def sweep_tuning(self):
        return hmc_get_sweep_tuning(self.h)

    def synchronize(self):
        hmc_synchronize(self.h)
