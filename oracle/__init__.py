"""FP64 CPU oracle of the hybrid Monte Carlo hot path (test infrastructure).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU leg
of ``bench.py`` may import this package; the product path never does.  It shares
no code with the CUDA library.  Scalar loops live in ``hmc_oracle.c`` (plain C,
double precision, compiled by ``oracle/build.py``); this module marshals numpy
arrays into them and writes out, in numpy, the small host-side formulas:
calibration (Eqs. 11-13), the loading control, the texture measures, and the
Monte Carlo step schedule.

Paper: Zhang, Bartel & Lusk, "Parallelized Hybrid Monte Carlo Simulation of
Stress-Induced Texture Evolution".  Readings of silent or garbled passages are
the ones listed in the design notes: periodic lattice, 6 neighbours, bonds
counted once, neighbour-copy trial state, constant-traction sign that grows the
softer grain, total-form stress, mixed uniaxial loading control.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building if needed) the oracle's shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        u16p = C.POINTER(C.c_uint16)
        u32p = C.POINTER(C.c_uint32)
        i64p = C.POINTER(C.c_int64)
        u8p = C.POINTER(C.c_uint8)
        i = C.c_int
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_euler_zyz_to_A.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.orc_rotated_stiffness.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
        L.orc_invert6.argtypes = [dp, dp]
        L.orc_invert6.restype = C.c_int
        L.orc_point_strain.argtypes = [i, i, i, dp, dp, i, i, i, dp]
        L.orc_point_stress.argtypes = [i, i, i, u16p, dp, dp, dp, i, i, i, dp]
        L.orc_internal_force.argtypes = [i, i, i, u16p, dp, dp, dp, dp]
        L.orc_lumped_mass.argtypes = [i, i, i, dp]
        L.orc_strain_field.argtypes = [i, i, i, dp, dp, dp]
        L.orc_node_force.argtypes = [i, i, i, u16p, dp, dp, dp, i, i, i, dp]
        L.orc_mpm_step.argtypes = [i, i, i, u16p, dp, dp, dp, dp, C.c_double, C.c_double, dp, dp]
        L.orc_stress_field.argtypes = [i, i, i, u16p, dp, dp, dp, dp, dp, dp]
        L.orc_point_zone_shift.argtypes = [dp, dp, dp]
        L.orc_point_zone_shift.restype = C.c_double
        L.orc_site_draws.argtypes = [i, i, i, i, i, C.c_uint64, C.c_uint32, C.c_uint32, i, u32p]
        L.orc_point_strain_shift.argtypes = [dp, dp, dp, dp]
        L.orc_point_strain_shift.restype = C.c_double
        L.orc_accept_threshold.argtypes = [i, C.c_double, C.c_double]
        L.orc_accept_threshold.restype = C.c_double
        L.orc_site_trial.argtypes = [i, i, i, u16p, i, i, i, C.c_uint64, C.c_uint32, C.c_uint32,
                                     C.c_double, C.c_double, i, i, i, C.c_double, dp, dp, dp,
                                     u16p, dp, dp]
        L.orc_site_trial.restype = C.c_int
        L.orc_site_trial_at.argtypes = L.orc_site_trial.argtypes
        L.orc_site_trial_at.restype = C.c_int
        L.orc_half_sweep.argtypes = [i, i, i, u16p, i, C.c_uint64, C.c_uint32, C.c_uint32,
                                     C.c_double, C.c_double, i, i, i, C.c_double, dp, dp, dp,
                                     u8p, dp, dp]
        L.orc_half_sweep.restype = C.c_int64
        L.orc_unlike_bonds.argtypes = [i, i, i, u16p]
        L.orc_unlike_bonds.restype = C.c_int64
        L.orc_orientation_counts.argtypes = [C.c_int64, u16p, i, i64p]
        L.orc_gs_sweep.argtypes = [i, i, i, u16p, C.c_uint64, C.c_uint32, C.c_uint32, C.c_double, C.c_double,
                                   i, i, i64p]
        L.orc_gs_sweep.restype = C.c_int64
        L.orc_grain_count.argtypes = [i, i, i, u16p, i64p]
        L.orc_grain_count.restype = C.c_int64
        _lib = L
    return _lib


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


# ---------------------------------------------------------------------------
# Random numbers
# ---------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11): 4 counter words, 2 key words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


# ---------------------------------------------------------------------------
# Orientation tables (Sec. "Elastic Deformation", Eqs. 16-18)
# ---------------------------------------------------------------------------

def euler_to_A(phi, theta, psi):
    A = np.zeros(9)
    lib().orc_euler_zyz_to_A(float(phi), float(theta), float(psi), _p(A, C.c_double))
    return A.reshape(3, 3)


def rotated_stiffness(c11, c12, c44, A):
    A = _f64(A).reshape(9)
    Cv = np.zeros(36)
    lib().orc_rotated_stiffness(float(c11), float(c12), float(c44), _p(A, C.c_double), _p(Cv, C.c_double))
    return Cv.reshape(6, 6)


def invert6(Cv):
    Cv = _f64(Cv).reshape(36)
    S = np.zeros(36)
    if lib().orc_invert6(_p(Cv, C.c_double), _p(S, C.c_double)) != 0:
        raise ValueError("singular stiffness")
    return S.reshape(6, 6)


def tables(euler, c11, c12, c44):
    """Per-orientation rotation A (Q,3,3), stiffness C' (Q,6,6) and compliance S' (Q,6,6)."""
    euler = np.asarray(euler, dtype=np.float64).reshape(-1, 3)
    Q = euler.shape[0]
    A = np.zeros((Q, 3, 3))
    Ct = np.zeros((Q, 6, 6))
    St = np.zeros((Q, 6, 6))
    for q in range(Q):
        A[q] = euler_to_A(*euler[q])
        Ct[q] = rotated_stiffness(c11, c12, c44, A[q])
        St[q] = invert6(Ct[q])
    return A, Ct, St


# ---------------------------------------------------------------------------
# Calibration (Sec. "Time, Length and Energy Scales", Eqs. 11-13, Table 1)
# ---------------------------------------------------------------------------

TABLE1 = dict(m_star=0.27, gamma_star=2.4, m_s=1.0e-13, gamma_s=0.45, l0=1.0e-3)


def characteristic_energy(K, gamma_s=TABLE1["gamma_s"], l0=TABLE1["l0"], gamma_star=TABLE1["gamma_star"]):
    """E0 = gamma_s l0^2 Delta^2 / gamma*  (Eq. 12), Delta = 1/K."""
    d = 1.0 / K
    return gamma_s * l0 ** 2 * d ** 2 / gamma_star


def characteristic_time(K, m_star=TABLE1["m_star"], m_s=TABLE1["m_s"], gamma_s=TABLE1["gamma_s"], l0=TABLE1["l0"]):
    """t0 = l0^2 m* Delta^2 / (m_s gamma_s)  (Eq. 11), Delta = 1/K."""
    d = 1.0 / K
    return l0 ** 2 * m_star * d ** 2 / (m_s * gamma_s)


def elastic_scale(K, **kw):
    """MC energy per GPa of elastic energy density: Delta^3 l0^3 / (2 E0) (Eq. 13) x 1e9 J/m^3."""
    l0 = kw.get("l0", TABLE1["l0"])
    d = 1.0 / K
    return 1.0e9 * d ** 3 * l0 ** 3 / (2.0 * characteristic_energy(K, **kw))


def default_dt(c11, c12, c44, h=2.0, rho=1.0):
    """Explicit step 0.5 h / c with c^2 = (largest stiffness eigenvalue of the cubic crystal) / rho."""
    lam = max(c11 + 2.0 * c12, c11 - c12, 2.0 * c44)
    return 0.5 * h / math.sqrt(lam / rho)


DEFAULT_DAMPING = 0.05


# ---------------------------------------------------------------------------
# Loading control (uniaxial strain along n with traction-free sides)
# ---------------------------------------------------------------------------

def axis_vectors(n):
    """N: n(x)n as Voigt tensor components; Ns: weights giving n.sigma.n from a Voigt stress."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    N = np.array([n[0] ** 2, n[1] ** 2, n[2] ** 2, n[1] * n[2], n[0] * n[2], n[0] * n[1]])
    Ns = np.array([n[0] ** 2, n[1] ** 2, n[2] ** 2, 2 * n[1] * n[2], 2 * n[0] * n[2], 2 * n[0] * n[1]])
    return n, N, Ns


def reuss_compliance(St, counts):
    f = np.asarray(counts, dtype=np.float64)
    f = f / f.sum()
    return np.einsum("q,qij->ij", f, St)


def initial_uniaxial_strain(S_R, n, eps0):
    _, N, _ = axis_vectors(n)
    b = S_R @ N
    return eps0 / (N @ b) * b


def initial_traction_strain(S_R, n, s0):
    """Mean strain whose Reuss stress is the uniaxial stress s0 n(x)n."""
    _, N, _ = axis_vectors(n)
    return S_R @ (s0 * N)


def update_traction_strain(E, mean_sig, S_R, n, s0):
    """Stress control: move the mean strain by the Reuss compliance times the gap
    between the prescribed uniaxial stress s0 n(x)n and the mean stress."""
    _, N, _ = axis_vectors(n)
    return E + S_R @ (s0 * N - mean_sig)


def update_uniaxial_strain(E, mean_sig, S_R, n, eps0):
    """Remove the lateral part of the mean stress with the Reuss compliance, then
    put the axial strain n.E.n back to eps0 along the uniaxial-stress direction."""
    _, N, Ns = axis_vectors(n)
    r = mean_sig - (Ns @ mean_sig) * N
    E = E - S_R @ r
    b = S_R @ N
    return E + (eps0 - N @ E) / (N @ b) * b


# ---------------------------------------------------------------------------
# MPM (Sec. "Elastic Deformation")
# ---------------------------------------------------------------------------

def point_strain(shape, u, Ebar, x, y, z):
    nz, ny, nx = shape
    eps = np.zeros(6)
    u = _f64(u)
    E = _f64(Ebar)
    lib().orc_point_strain(nx, ny, nz, _p(u, C.c_double), _p(E, C.c_double), x, y, z, _p(eps, C.c_double))
    return eps


def point_stress(spins, Ct, u, Ebar, x, y, z):
    nz, ny, nx = spins.shape
    sig = np.zeros(6)
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    Cf = _f64(Ct)
    u = _f64(u)
    E = _f64(Ebar)
    lib().orc_point_stress(nx, ny, nz, _p(s, C.c_uint16), _p(Cf, C.c_double), _p(u, C.c_double),
                           _p(E, C.c_double), x, y, z, _p(sig, C.c_double))
    return sig


def internal_force(spins, Ct, u, Ebar):
    nz, ny, nx = spins.shape
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    Cf, u, E = _f64(Ct), _f64(u), _f64(Ebar)
    f = np.zeros_like(u)
    lib().orc_internal_force(nx, ny, nz, _p(s, C.c_uint16), _p(Cf, C.c_double), _p(u, C.c_double),
                             _p(E, C.c_double), _p(f, C.c_double))
    return f


def node_force(spins, Ct, u, Ebar, i, j, k):
    """Internal force of node (i,j,k), gathered over its 64 points."""
    nz, ny, nx = spins.shape
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    Cf, u, E = _f64(Ct), _f64(u), _f64(Ebar)
    f = np.zeros(3)
    lib().orc_node_force(nx, ny, nz, _p(s, C.c_uint16), _p(Cf, C.c_double), _p(u, C.c_double),
                         _p(E, C.c_double), int(i), int(j), int(k), _p(f, C.c_double))
    return f


def strain_field(shape, u, Ebar):
    """(N,6) strain of every point."""
    nz, ny, nx = shape
    u, E = _f64(u), _f64(Ebar)
    eps = np.zeros((nx * ny * nz, 6))
    lib().orc_strain_field(nx, ny, nz, _p(u, C.c_double), _p(E, C.c_double), _p(eps, C.c_double))
    return eps


def lumped_mass(shape):
    nz, ny, nx = shape
    m = np.zeros((nz // 2) * (ny // 2) * (nx // 2))
    lib().orc_lumped_mass(nx, ny, nz, _p(m, C.c_double))
    return m


def mpm_steps(spins, Ct, Ebar, u, v, nsteps, dt, damping):
    """nsteps explicit steps, in place on the (nnodes,3) arrays u and v."""
    nz, ny, nx = spins.shape
    assert u.dtype == np.float64 and u.flags.c_contiguous and v.dtype == np.float64 and v.flags.c_contiguous
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    Cf, E = _f64(Ct), _f64(Ebar)
    f = np.zeros_like(u)
    m = np.zeros(u.shape[0])
    L = lib()
    for _ in range(int(nsteps)):
        L.orc_mpm_step(nx, ny, nz, _p(s, C.c_uint16), _p(Cf, C.c_double), _p(E, C.c_double),
                       _p(u, C.c_double), _p(v, C.c_double), float(dt), float(damping),
                       _p(f, C.c_double), _p(m, C.c_double))


def stress_field(spins, Ct, u, Ebar):
    """(N,6) stress, mean stress (6) and elastic energy (Eq. 1 summed)."""
    nz, ny, nx = spins.shape
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    Cf, u, E = _f64(Ct), _f64(u), _f64(Ebar)
    sig = np.zeros((nx * ny * nz, 6))
    mean = np.zeros(6)
    W = np.zeros(1)
    lib().orc_stress_field(nx, ny, nz, _p(s, C.c_uint16), _p(Cf, C.c_double), _p(u, C.c_double),
                           _p(E, C.c_double), _p(sig, C.c_double), _p(mean, C.c_double), _p(W, C.c_double))
    return sig, mean, float(W[0])


# ---------------------------------------------------------------------------
# Monte Carlo (Sec. "Hybrid Monte Carlo Methodology", "Microstructural Evolution")
# ---------------------------------------------------------------------------

TRIAL_NEIGHBOR, TRIAL_UNIFORM_Q = 0, 1


ELASTIC_OFF, ELASTIC_TRACTION, ELASTIC_ZONE1, ELASTIC_STRAIN = 0, 1, 2, 3


def site_draws(nx, ny, x, y, z, seed, mcs, replica, trial=0):
    """(r0, r1) of the trial at (x, y, z): r0 picks the trial state, r1 decides.  The
    colour's four sites of a 2x2x2 block share the Philox block with counter (block
    origin index, mcs, replica, 2 + colour); the site with the j-th smallest local corner
    index takes word j.  Neighbour trials (trial 0): r1 = low 32 bits of 6 r0; trials over
    all orientations: r1 = word j of the block with counter word 3 = 4 + colour."""
    out = np.zeros(2, dtype=np.uint32)
    lib().orc_site_draws(int(nx), int(ny), int(x), int(y), int(z), int(seed), int(mcs), int(replica),
                         int(trial), _p(out, C.c_uint32))
    return int(out[0]), int(out[1])


def point_zone_shift(S_old, S_new, sig):
    a, b, s = _f64(S_old), _f64(S_new), _f64(sig)
    return lib().orc_point_zone_shift(_p(a, C.c_double), _p(b, C.c_double), _p(s, C.c_double))


def point_strain_shift(S_old, C_old, C_new, sig):
    """Constant-strain one-point shift 1/2 e.(C_new - C_old).e with e = S_old sig."""
    a, b, c, s = _f64(S_old), _f64(C_old), _f64(C_new), _f64(sig)
    return lib().orc_point_strain_shift(_p(a, C.c_double), _p(b, C.c_double), _p(c, C.c_double),
                                        _p(s, C.c_double))


def accept_threshold(k, J, kT):
    return lib().orc_accept_threshold(int(k), float(J), float(kT))


def site_trial(spins, x, y, z, seed, mcs, replica, J, kT, trial, Q, elastic, lam, St, sig, Ct=None):
    nz, ny, nx = spins.shape
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    Sf = _f64(St) if St is not None else np.zeros(36)
    Cf = _f64(Ct) if Ct is not None else np.zeros_like(Sf)
    sg = _f64(sig) if sig is not None else np.zeros(6 * nx * ny * nz)
    qn = np.zeros(1, dtype=np.uint16)
    dH = np.zeros(1)
    t = np.zeros(1)
    acc = lib().orc_site_trial(nx, ny, nz, _p(s, C.c_uint16), x, y, z, int(seed), int(mcs), int(replica),
                               float(J), float(kT), int(trial), int(Q), int(elastic), float(lam),
                               _p(Sf, C.c_double), _p(Cf, C.c_double), _p(sg, C.c_double), _p(qn, C.c_uint16),
                               _p(dH, C.c_double), _p(t, C.c_double))
    return bool(acc), int(qn[0]), float(dH[0]), float(t[0])


def site_trial_at(spins, x, y, z, seed, mcs, replica, J, kT, trial, Q, elastic, lam, St, sig_p, Ct=None):
    """One trial with the site's own stress sig_p (6 values) instead of a whole field."""
    nz, ny, nx = spins.shape
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    Sf = _f64(St) if St is not None else np.zeros(36)
    Cf = _f64(Ct) if Ct is not None else np.zeros_like(Sf)
    sg = _f64(sig_p) if sig_p is not None else np.zeros(6)
    qn = np.zeros(1, dtype=np.uint16)
    dH = np.zeros(1)
    t = np.zeros(1)
    acc = lib().orc_site_trial_at(nx, ny, nz, _p(s, C.c_uint16), x, y, z, int(seed), int(mcs), int(replica),
                                  float(J), float(kT), int(trial), int(Q), int(elastic), float(lam),
                                  _p(Sf, C.c_double), _p(Cf, C.c_double), _p(sg, C.c_double), _p(qn, C.c_uint16),
                                  _p(dH, C.c_double), _p(t, C.c_double))
    return bool(acc), int(qn[0]), float(dH[0]), float(t[0])


def half_sweep(spins, colour, seed, mcs, replica, J, kT, trial, Q, elastic, lam, St, sig, Ct=None):
    """In-place red/black half sweep; returns (accepted, changed[N] u8, dH[N], thresh[N]).
    elastic: 0 off, 1 constant-traction point zone (St), 3 constant-strain point zone (St, Ct)."""
    nz, ny, nx = spins.shape
    assert spins.dtype == np.uint16 and spins.flags.c_contiguous
    N = nx * ny * nz
    Sf = _f64(St) if St is not None else np.zeros(36)
    Cf = _f64(Ct) if Ct is not None else np.zeros_like(Sf)
    sg = _f64(sig) if sig is not None else np.zeros(1)
    changed = np.zeros(N, dtype=np.uint8)
    dH = np.zeros(N)
    t = np.zeros(N)
    acc = lib().orc_half_sweep(nx, ny, nz, _p(spins, C.c_uint16), int(colour), int(seed), int(mcs), int(replica),
                               float(J), float(kT), int(trial), int(Q), int(elastic), float(lam),
                               _p(Sf, C.c_double), _p(Cf, C.c_double), _p(sg, C.c_double), _p(changed, C.c_uint8),
                               _p(dH, C.c_double), _p(t, C.c_double))
    return int(acc), changed, dH, t


def gs_sweep(spins, seed, mcs, replica, J, kT, trial, Q):
    """In-place Gauss-Seidel Monte Carlo step (sequential random sites, each
    accepted trial applied at once); returns (accepted, summed bond-count change)."""
    nz, ny, nx = spins.shape
    assert spins.dtype == np.uint16 and spins.flags.c_contiguous
    de = np.zeros(1, dtype=np.int64)
    acc = lib().orc_gs_sweep(nx, ny, nz, _p(spins, C.c_uint16), int(seed), int(mcs), int(replica), float(J),
                             float(kT), int(trial), int(Q), _p(de, C.c_int64))
    return int(acc), int(de[0])


def grain_count(spins, want_labels=False):
    """Grains = face-connected sets of one orientation on the periodic lattice."""
    nz, ny, nx = spins.shape
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    lab = np.zeros(s.size, dtype=np.int64) if want_labels else None
    n = lib().orc_grain_count(nx, ny, nz, _p(s, C.c_uint16), _p(lab, C.c_int64) if want_labels else None)
    if n < 0:
        raise MemoryError("grain count")
    return (int(n), lab.reshape(s.shape)) if want_labels else int(n)


def unlike_bonds(spins):
    nz, ny, nx = spins.shape
    s = np.ascontiguousarray(spins, dtype=np.uint16)
    return int(lib().orc_unlike_bonds(nx, ny, nz, _p(s, C.c_uint16)))


def orientation_counts(spins, Q):
    s = np.ascontiguousarray(spins, dtype=np.uint16).reshape(-1)
    out = np.zeros(Q, dtype=np.int64)
    lib().orc_orientation_counts(s.size, _p(s, C.c_uint16), int(Q), _p(out, C.c_int64))
    return out


# ---------------------------------------------------------------------------
# Texture measures (Sec. "Results": orientation angle and Young's modulus)
# ---------------------------------------------------------------------------

def young_modulus_along(St, n):
    """E(n) = 1 / (n.S'.n) for every orientation (uniaxial stress along n)."""
    _, N, _ = axis_vectors(n)
    return 1.0 / np.einsum("i,qij,j->q", N, St, N)


def angle_to_nearest_100(A, n):
    """Angle (degrees) between n and the closest crystal <100> axis (columns of A)."""
    n, _, _ = axis_vectors(n)
    c = np.abs(np.einsum("qij,i->qj", A, n)).max(axis=1)
    return np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))


def texture_histogram(kind, nbins, counts, A, St, n, c11, c12, c44):
    """Volume fractions per bin.  kind 0: per orientation; 1: angle to nearest
    <100> in bins of 90/nbins degrees; 2: E(n)/C11 in nbins equal bins over
    [E<100>, E<111>]/C11 (cubic closed form bounds)."""
    counts = np.asarray(counts, dtype=np.int64)
    Ntot = counts.sum()
    if kind == 0:
        return counts / Ntot
    if kind == 1:
        ang = angle_to_nearest_100(A, n)
        b = np.minimum((ang / (90.0 / nbins)).astype(np.int64), nbins - 1)
    else:
        d = (c11 - c12) * (c11 + 2 * c12)
        S11, S12, S44 = (c11 + c12) / d, -c12 / d, 1.0 / c44
        e_lo, e_hi = 1.0 / S11, 1.0 / (S11 - 2.0 * (S11 - S12 - 0.5 * S44) / 3.0)
        lo, hi = min(e_lo, e_hi) / c11, max(e_lo, e_hi) / c11
        x = young_modulus_along(St, n) / c11
        b = np.clip(((x - lo) / (hi - lo) * nbins).astype(np.int64), 0, nbins - 1)
    out = np.zeros(nbins, dtype=np.int64)
    np.add.at(out, b, counts)
    return out / Ntot


# ---------------------------------------------------------------------------
# The Monte Carlo step schedule (Sec. "Results": equilibrate, then one MC step)
# ---------------------------------------------------------------------------

BC_UNIAXIAL, BC_STRAIN6, BC_TRACTION = 0, 1, 2
# ELASTIC_* and TRIAL_* are defined with the Monte Carlo functions above


class OracleHMC:
    """State and schedule of one replica.  One Monte Carlo step (MCS) is:
    ``mpm_steps_per_mcs`` explicit steps, the stress of every point from the
    resulting displacement, the red then the black half sweep with that stress
    frozen, and (uniaxial control) one update of the mean strain."""

    def __init__(self, shape, Q, *, J=1.0, kT=0.7, c11=246.5, c12=147.3, c44=124.7,
                 bc=BC_UNIAXIAL, load_axis=(0, 0, 1), strain=1e-3, strain6=None, stress=0.0,
                 elastic_scale_=None, elastic=ELASTIC_TRACTION, trial=TRIAL_NEIGHBOR,
                 mpm_steps_per_mcs=50, dt=None, damping=None, seed=0, replica=0):
        self.shape = tuple(shape)  # (nz, ny, nx)
        nz, ny, nx = self.shape
        assert nx % 2 == 0 and ny % 2 == 0 and nz % 2 == 0
        self.Q, self.J, self.kT = Q, J, kT
        self.c = (c11, c12, c44)
        self.bc, self.axis, self.eps0 = bc, np.asarray(load_axis, dtype=np.float64), strain
        self.sig0 = stress
        self.strain6 = np.zeros(6) if strain6 is None else np.asarray(strain6, dtype=np.float64)
        self.lam = elastic_scale(max(nx, ny, nz)) if elastic_scale_ is None or elastic_scale_ < 0 else elastic_scale_
        self.elastic, self.trial = elastic, trial
        self.n_mpm = mpm_steps_per_mcs
        self.dt = default_dt(c11, c12, c44) if dt is None or dt <= 0 else dt
        self.damping = DEFAULT_DAMPING if damping is None or damping < 0 else damping
        self.seed, self.replica = seed, replica
        self.mcs = 0
        self.nnodes = (nx // 2) * (ny // 2) * (nz // 2)

    def set_orientations(self, euler, spins):
        self.A, self.Ct, self.St = tables(euler, *self.c)
        self.spins = np.ascontiguousarray(np.asarray(spins, dtype=np.uint16).reshape(self.shape))
        self.S_R = reuss_compliance(self.St, orientation_counts(self.spins, self.Q))
        if self.bc == BC_UNIAXIAL:
            self.Ebar = initial_uniaxial_strain(self.S_R, self.axis, self.eps0)
        elif self.bc == BC_TRACTION:
            self.Ebar = initial_traction_strain(self.S_R, self.axis, self.sig0)
        else:
            self.Ebar = self.strain6.copy()
        self.u = np.zeros((self.nnodes, 3))
        self.v = np.zeros((self.nnodes, 3))
        self.mcs = 0

    def mpm_steps(self, n):
        mpm_steps(self.spins, self.Ct, self.Ebar, self.u, self.v, n, self.dt, self.damping)

    def stress(self):
        self.sig, self.mean_sig, self.W = stress_field(self.spins, self.Ct, self.u, self.Ebar)
        return self.sig

    def half_sweep(self, colour):
        return half_sweep(self.spins, colour, self.seed, self.mcs, self.replica, self.J, self.kT,
                          self.trial, self.Q, self.elastic, self.lam, self.St,
                          self.sig if self.elastic else None, self.Ct)

    def end_mcs(self):
        if self.bc == BC_UNIAXIAL:
            self.Ebar = update_uniaxial_strain(self.Ebar, self.mean_sig, self.S_R, self.axis, self.eps0)
        elif self.bc == BC_TRACTION:
            self.Ebar = update_traction_strain(self.Ebar, self.mean_sig, self.S_R, self.axis, self.sig0)
        self.mcs += 1

    def set_load(self, value):
        """New uniaxial strain (UNIAXIAL) or stress (TRACTION); the mean strain
        moves at once by the Reuss response to the change."""
        _, N, _ = axis_vectors(self.axis)
        if self.bc == BC_UNIAXIAL:
            b = self.S_R @ N
            self.Ebar = self.Ebar + (value - self.eps0) / (N @ b) * b
            self.eps0 = value
        elif self.bc == BC_TRACTION:
            self.Ebar = self.Ebar + self.S_R @ ((value - self.sig0) * N)
            self.sig0 = value
        else:
            raise ValueError("STRAIN6 has no scalar load")

    def mc_sweeps(self, n):
        total = 0
        for _ in range(int(n)):
            self.mpm_steps(self.n_mpm)
            self.stress()
            total += self.half_sweep(0)[0]
            total += self.half_sweep(1)[0]
            self.end_mcs()
        return total
