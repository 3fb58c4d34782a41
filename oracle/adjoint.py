"""Forward-mode (tangent-linear) gradient of the explicit MPM stress solve
(test infrastructure; see ``oracle/__init__.py``).

The map: T explicit steps (Sec. "Elastic Deformation") from a given nodal
state with the spins frozen, parameters theta = (C11, C12, C44, Ebar_1..6);
outputs the elastic energy W = sum_p 1/2 eps_p.C'_p.eps_p (one voxel per point)
and the per-point field w_p = 1/2 eps_p.C'_p.eps_p = 1/2 sigma_p.S'_p.sigma_p
(the one-point zone energy of Eq. 8 in the constant-traction reading).  For a
cotangent (gW, g) this computes dL/dtheta of L = gW W + sum_p g_p w_p by
carrying, for each parameter, the derivative of (u, v) along with (u, v):

  f  = F(u; C, Ebar),                 df = F(du; C, 0) + dF/dtheta
  v' = (1 - damping) v + dt f / m,    dv' = (1 - damping) dv + dt df / m
  u' = u + dt v',                     du' = du + dt dv'

F is linear in C' and in Ebar, so dF/dC11 is F evaluated with the stiffness
table replaced by the rotated basis tensor of C11 (the rotation of the cubic
tensor with (C11, C12, C44) = (1, 0, 0)), and dF/dEbar_k is F(0; C, e_k).  No
reverse sweep is involved: this is independent of any adjoint.
"""
from __future__ import annotations

import numpy as np

from . import euler_to_A, internal_force, rotated_stiffness, strain_field, tables

N_PARAMS = 9


def basis_tables(euler):
    """Rotated basis tensors R1, R2, R3 (Q,6,6) with C' = C11 R1 + C12 R2 + C44 R3
    (the rotation of Eq. 17 is linear in the tensor; the basis tensors are singular,
    so no compliance is formed)."""
    euler = np.asarray(euler, dtype=np.float64).reshape(-1, 3)
    A = [euler_to_A(*e) for e in euler]
    return [np.stack([rotated_stiffness(*c, a) for a in A]) for c in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0))]


def forward(spins, Ct, Ebar, u0, v0, nsteps, dt, damping):
    """Final (u, v) of nsteps explicit steps (same update as ``oracle.mpm_steps``)."""
    u, v = u0.copy(), v0.copy()
    for _ in range(nsteps):
        f = internal_force(spins, Ct, u, Ebar)
        v = (1.0 - damping) * v + dt * f / 8.0
        u = u + dt * v
    return u, v


def outputs(spins, Ct, Ebar, u):
    """W and the field w_p at displacement u."""
    eps = strain_field(spins.shape, u, Ebar)
    Cp = Ct[spins.reshape(-1)]
    sig = np.einsum("pij,pj->pi", Cp, eps)
    w = 0.5 * np.einsum("pi,pi->p", sig, eps)
    return w.sum(), w


def tangent_linear_gradient(spins, euler, c, Ebar, u0, v0, nsteps, dt, damping, gW, g=None):
    """dL/d(C11, C12, C44, Ebar_1..6) for L = gW W + sum_p g_p w_p at the final state."""
    shape = spins.shape
    _, Ct, _ = tables(euler, *c)
    R = basis_tables(euler)
    N = spins.size
    alpha = gW + (np.zeros(N) if g is None else np.asarray(g, dtype=np.float64).reshape(-1))
    sp = spins.reshape(-1)
    grad = np.zeros(N_PARAMS)
    for k in range(N_PARAMS):
        u, v = u0.copy(), v0.copy()
        du, dv = np.zeros_like(u), np.zeros_like(v)
        Ek = np.zeros(6)
        if k >= 3:
            Ek[k - 3] = 1.0
        for _ in range(nsteps):
            f = internal_force(spins, Ct, u, Ebar)
            df = internal_force(spins, Ct, du, np.zeros(6))
            if k < 3:
                df += internal_force(spins, R[k], u, Ebar)
            else:
                df += internal_force(spins, Ct, np.zeros_like(u), Ek)
            v = (1.0 - damping) * v + dt * f / 8.0
            dv = (1.0 - damping) * dv + dt * df / 8.0
            u = u + dt * v
            du = du + dt * dv
        eps = strain_field(shape, u, Ebar)
        deps = strain_field(shape, du, Ek if k >= 3 else np.zeros(6))
        sig = np.einsum("pij,pj->pi", Ct[sp], eps)
        dw = np.einsum("pi,pi->p", sig, deps)
        if k < 3:
            dw += 0.5 * np.einsum("pi,pij,pj->p", eps, R[k][sp], eps)
        grad[k] = alpha @ dw
    return grad
