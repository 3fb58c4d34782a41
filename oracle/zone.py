"""Constant-traction zone energy and brute-force re-solve (test infrastructure).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Dense FP64 linear
algebra on tiny periodic grids.

* ``strain_matrix`` writes the strain-displacement map B_p of one material point
  (6 x 3*nnodes, trilinear shape functions, two points per cell edge), so that
  eps_p = Ebar + B_p u.
* ``equilibrium`` minimises the total elastic energy
  Pi(u) = sum_p 1/2 V (Ebar + B_p u) . C_p (Ebar + B_p u) over the periodic
  displacement (the quasi-static state the explicit solver of Sec. "Elastic
  Deformation" seeks), by a dense least-squares solve.
* ``brute_force_shift`` re-solves the whole domain before and after a trial
  reorientation and returns the change of Pi: the exact elastic part of
  [[H]]* that Sec. "Hybrid Monte Carlo Methodology" calls intractable.
* ``zone_shift`` is the approximation of Eq. 6: a zone Omega_1 (a cube of
  points around the site, or the whole domain) is re-equilibrated with the
  forces that the reservoir Omega_2 exerts on its nodes held at their current
  values (constant traction), and the shift is the change of the zone's energy
  minus the work of those fixed forces.  For the single-point zone this is
  Eq. 8 in the constant-traction reading; for the whole domain it is the
  brute-force shift.
* ``zone_shift_local`` is the same shift for the 27-point zone (half-width 1)
  written on the zone's own 27 nodes, so that it serves grids of any size
  (pinned to ``zone_shift`` on small grids).
"""
from __future__ import annotations

import numpy as np

H = 2.0   # cell edge, voxels
VP = 1.0  # particle volume


def strain_matrix(shape, x, y, z):
    nz, ny, nx = shape
    nbx, nby, nbz = nx // 2, ny // 2, nz // 2
    nn = nbx * nby * nbz
    B = np.zeros((6, 3 * nn))
    cx, cy, cz = x // 2, y // 2, z // 2
    xi = np.array([((x & 1) + 0.5) / H, ((y & 1) + 0.5) / H, ((z & 1) + 0.5) / H])
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                n = [xi[0] if di else 1 - xi[0], xi[1] if dj else 1 - xi[1], xi[2] if dk else 1 - xi[2]]
                s = [(1 if di else -1) / H, (1 if dj else -1) / H, (1 if dk else -1) / H]
                g = (s[0] * n[1] * n[2], n[0] * s[1] * n[2], n[0] * n[1] * s[2])
                I = ((cx + di) % nbx) + nbx * (((cy + dj) % nby) + nby * ((cz + dk) % nbz))
                B[:, 3 * I + 0] += (g[0], 0, 0, 0, g[2], g[1])
                B[:, 3 * I + 1] += (0, g[1], 0, g[2], 0, g[0])
                B[:, 3 * I + 2] += (0, 0, g[2], g[1], g[0], 0)
    return B


def all_strain_matrices(shape):
    nz, ny, nx = shape
    out = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                out.append(strain_matrix(shape, x, y, z))
    return np.stack(out)  # (N, 6, 3nn), natural point order


def assemble(Bs, Cp, Ebar, points=None):
    """K = sum V B^T C B, F = sum V B^T C Ebar over the chosen points."""
    idx = range(Bs.shape[0]) if points is None else points
    n = Bs.shape[2]
    K = np.zeros((n, n))
    F = np.zeros(n)
    for p in idx:
        BC = Bs[p].T @ Cp[p]
        K += VP * BC @ Bs[p]
        F += VP * BC @ Ebar
    return K, F


def energy(Bs, Cp, Ebar, u, points=None):
    idx = range(Bs.shape[0]) if points is None else points
    W = 0.0
    for p in idx:
        e = Ebar + Bs[p] @ u
        W += 0.5 * VP * e @ Cp[p] @ e
    return W


def equilibrium(Bs, Cp, Ebar):
    K, F = assemble(Bs, Cp, Ebar)
    u, *_ = np.linalg.lstsq(K, -F, rcond=None)
    return u, energy(Bs, Cp, Ebar, u)


def point_stiffness(spins, Ct):
    return Ct[np.asarray(spins).reshape(-1)]


def brute_force_shift(spins, Ct, Ebar, p, q_new, Bs=None):
    shape = spins.shape
    Bs = all_strain_matrices(shape) if Bs is None else Bs
    Cp = point_stiffness(spins, Ct)
    _, W0 = equilibrium(Bs, Cp, Ebar)
    Cp2 = Cp.copy()
    Cp2[p] = Ct[q_new]
    _, W1 = equilibrium(Bs, Cp2, Ebar)
    return W1 - W0


def zone_points(shape, p, r):
    """Points of the periodic cube of half-width r around point p (r < 0: all)."""
    nz, ny, nx = shape
    if r < 0:
        return list(range(nx * ny * nz))
    x, y, z = p % nx, (p // nx) % ny, p // (nx * ny)
    assert 2 * r + 1 <= min(nx, ny, nz)
    pts = []
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                pts.append(((x + dx) % nx) + nx * (((y + dy) % ny) + ny * ((z + dz) % nz)))
    return pts


def zone_shift(spins, Ct, Ebar, u0, p, q_new, r, Bs=None):
    """Eq. 6 for a zone of half-width r around point p (r < 0: whole domain),
    about the current displacement u0."""
    shape = spins.shape
    Bs = all_strain_matrices(shape) if Bs is None else Bs
    Cp = point_stiffness(spins, Ct)
    pts = zone_points(shape, p, r)
    dofs = np.nonzero(np.abs(Bs[pts]).sum(axis=(0, 1)) > 0)[0]
    # dead forces of the reservoir on the zone's nodes, frozen at the current state
    g = np.zeros(Bs.shape[2])
    for s in pts:
        g += VP * Bs[s].T @ (Cp[s] @ (Ebar + Bs[s] @ u0))
    W_old = energy(Bs, Cp, Ebar, u0, pts) - g @ u0
    Cp2 = Cp.copy()
    Cp2[p] = Ct[q_new]
    K, F = assemble(Bs, Cp2, Ebar, pts)
    Kd = K[np.ix_(dofs, dofs)]
    rhs = (g - F)[dofs]
    du, *_ = np.linalg.lstsq(Kd, rhs, rcond=None)
    u1 = u0.copy()
    u1[dofs] = du
    W_new = energy(Bs, Cp2, Ebar, u1, pts) - g @ u1
    return W_new - W_old


def zone_shift_local(spins, Ct, Ebar, u0, x, y, z, q_new):
    """zone_shift for the zone of half-width 1 around voxel (x, y, z), on the zone's
    own nodes: the 27 points span 2 x 2 x 2 cells and their 3 x 3 x 3 nodes (grid
    edges >= 6, so the nodes are distinct), and every point's strain-displacement
    map touches only those, so restricting B_p to the 81 zone DOFs changes nothing.
    u0: (nnodes, 3) current displacement."""
    nz, ny, nx = spins.shape
    nbx, nby, nbz = nx // 2, ny // 2, nz // 2
    u0 = np.asarray(u0).reshape(-1, 3)
    lo = ((x - 1) // 2, (y - 1) // 2, (z - 1) // 2)          # the zone's lowest node (unwrapped)
    nodes = [((lo[0] + i) % nbx) + nbx * (((lo[1] + j) % nby) + nby * ((lo[2] + k) % nbz))
             for k in range(3) for j in range(3) for i in range(3)]
    u = u0[nodes].reshape(-1)                                   # local DOF 3 (i + 3 j + 9 k) + alpha
    pts, Bs, Cp = [], [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                px, py, pz = x + dx, y + dy, z + dz                 # unwrapped voxel coordinates
                xi = np.array([((px & 1) + 0.5) / H, ((py & 1) + 0.5) / H, ((pz & 1) + 0.5) / H])
                B = np.zeros((6, 81))
                for dk in (0, 1):
                    for dj in (0, 1):
                        for di in (0, 1):
                            n = [xi[0] if di else 1 - xi[0], xi[1] if dj else 1 - xi[1], xi[2] if dk else 1 - xi[2]]
                            sg = [(1 if di else -1) / H, (1 if dj else -1) / H, (1 if dk else -1) / H]
                            g = (sg[0] * n[1] * n[2], n[0] * sg[1] * n[2], n[0] * n[1] * sg[2])
                            li = (px // 2 + di - lo[0]) + 3 * ((py // 2 + dj - lo[1]) + 3 * (pz // 2 + dk - lo[2]))
                            B[:, 3 * li + 0] += (g[0], 0, 0, 0, g[2], g[1])
                            B[:, 3 * li + 1] += (0, g[1], 0, g[2], 0, g[0])
                            B[:, 3 * li + 2] += (0, 0, g[2], g[1], g[0], 0)
                Bs.append(B)
                Cp.append(Ct[int(spins[pz % nz, py % ny, px % nx])])
                pts.append((dx, dy, dz))
    Bs = np.stack(Bs)
    Cp = np.stack(Cp)
    # dead forces of the reservoir on the zone's nodes, frozen at the current state
    g = np.zeros(81)
    for s in range(27):
        g += VP * Bs[s].T @ (Cp[s] @ (Ebar + Bs[s] @ u))
    W_old = energy(Bs, Cp, Ebar, u) - g @ u
    Cp2 = Cp.copy()
    Cp2[13] = Ct[q_new]                                          # the site: offset (0, 0, 0)
    K, F = assemble(Bs, Cp2, Ebar)
    du, *_ = np.linalg.lstsq(K, g - F, rcond=None)
    W_new = energy(Bs, Cp2, Ebar, du) - g @ du
    return W_new - W_old


def site_trial_zone_local(spins, x, y, z, seed, mcs, replica, J, kT, trial, Q, lam, Ct, Ebar, u0):
    """site_trial_zone for the zone of half-width 1 with zone_shift_local (any grid size)."""
    from . import TRIAL_NEIGHBOR, accept_threshold, site_draws
    nz, ny, nx = spins.shape
    w = site_draws(nx, ny, x, y, z, seed, mcs, replica, trial)
    nb = [int(spins[z, y, (x - 1) % nx]), int(spins[z, y, (x + 1) % nx]),
          int(spins[z, (y - 1) % ny, x]), int(spins[z, (y + 1) % ny, x]),
          int(spins[(z - 1) % nz, y, x]), int(spins[(z + 1) % nz, y, x])]
    q = int(spins[z, y, x])
    if trial == TRIAL_NEIGHBOR:
        qn = nb[(int(w[0]) * 6) >> 32]
    else:
        qn = (int(w[0]) * int(Q)) >> 32
    if qn == q:
        return False, qn, 0.0, -1.0
    dE = sum(1 for v in nb if v == q) - sum(1 for v in nb if v == qn)
    dHe = lam * zone_shift_local(spins, Ct, Ebar, u0, x, y, z, qn)
    if dHe == 0.0:
        return (dE <= 0 or float(w[1]) < accept_threshold(dE, J, kT)), qn, J * dE, -1.0
    Ht = J * dE + dHe
    t = -kT * np.log((float(w[1]) + 0.5) / 4294967296.0) if kT > 0 else 0.0
    return bool(Ht <= t), qn, Ht, t


# ---------------------------------------------------------------------------
# Red/black half sweep with the zone energy of Eq. 6 (zone half-width r)
# ---------------------------------------------------------------------------

def site_trial_zone(spins, x, y, z, seed, mcs, replica, J, kT, trial, Q, lam, Ct, Ebar, u0, r, Bs):
    """One Metropolis trial (Eq. 5) at voxel (x, y, z): the trial orientation
    and the bond-energy change as in the one-point sweep (the site's Philox
    draws, neighbour order -x,+x,-y,+y,-z,+z), the elastic
    term lam * zone_shift over the zone of half-width r about the current
    displacement u0.  Returns (accepted, q_new, dH, threshold)."""
    from . import TRIAL_NEIGHBOR, accept_threshold, site_draws
    nz, ny, nx = spins.shape
    p = x + nx * (y + ny * z)
    w = site_draws(nx, ny, x, y, z, seed, mcs, replica, trial)
    nb = [int(spins[z, y, (x - 1) % nx]), int(spins[z, y, (x + 1) % nx]),
          int(spins[z, (y - 1) % ny, x]), int(spins[z, (y + 1) % ny, x]),
          int(spins[(z - 1) % nz, y, x]), int(spins[(z + 1) % nz, y, x])]
    q = int(spins[z, y, x])
    if trial == TRIAL_NEIGHBOR:
        qn = nb[(int(w[0]) * 6) >> 32]
    else:
        qn = (int(w[0]) * int(Q)) >> 32
    if qn == q:
        return False, qn, 0.0, -1.0
    dE = sum(1 for v in nb if v == q) - sum(1 for v in nb if v == qn)
    dHe = lam * zone_shift(spins, Ct, Ebar, u0, p, qn, r, Bs)
    if dHe == 0.0:
        return (dE <= 0 or float(w[1]) < accept_threshold(dE, J, kT)), qn, J * dE, -1.0
    H = J * dE + dHe
    t = -kT * np.log((float(w[1]) + 0.5) / 4294967296.0) if kT > 0 else 0.0
    return bool(H <= t), qn, H, t


def half_sweep_zone(spins, colour, seed, mcs, replica, J, kT, trial, Q, lam, Ct, Ebar, u0, r, Bs=None):
    """Red/black half step (Sec. "Microstructural Evolution") with the zone
    energy: every site of one colour ((x+y+z) even = red = 0) is tried against
    the orientations at the start of the half step, then the accepted trials
    are applied together.  A zone of half-width r >= 1 contains sites of the
    same colour, so the trials read the start-of-step copy.  In place; returns
    (accepted, changed[N] u8, dH[N], thresh[N]) in natural site order."""
    nz, ny, nx = spins.shape
    Bs = all_strain_matrices(spins.shape) if Bs is None else Bs
    start = spins.copy()
    N = nx * ny * nz
    changed = np.zeros(N, dtype=np.uint8)
    dH = np.zeros(N)
    thr = np.zeros(N)
    flips = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if ((x + y + z) & 1) != colour:
                    continue
                p = x + nx * (y + ny * z)
                acc, qn, h, t = site_trial_zone(start, x, y, z, seed, mcs, replica, J, kT, trial, Q, lam,
                                                Ct, Ebar, u0, r, Bs)
                dH[p], thr[p] = h, t
                if acc:
                    changed[p] = 1
                    flips.append((z, y, x, qn))
    for z, y, x, qn in flips:
        spins[z, y, x] = qn
    return len(flips), changed, dH, thr
