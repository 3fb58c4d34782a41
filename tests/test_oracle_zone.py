"""Oracle pins of the zone half sweep (Eq. 6 with a zone of half-width r)."""
import numpy as np
import pytest

import hmc_synth as S
import oracle as O
import oracle.zone as Z

C3 = (246.5, 147.3, 124.7)


@pytest.fixture(scope="module")
def poly():
    shape = (6, 6, 8)
    eul = S.euler_uniform_so3(5, 21)
    sp = S.voronoi_spins(shape, 6, 5, 22)
    A, Ct, St = O.tables(eul, *C3)
    Bs = Z.all_strain_matrices(shape)
    rng = np.random.default_rng(7)
    u0 = rng.normal(size=Bs.shape[2]) * 2e-4
    E = np.array([1e-3, -3e-4, -4e-4, 2e-4, -1e-4, 1e-4])
    return dict(shape=shape, sp=sp, Ct=Ct, St=St, Bs=Bs, u0=u0, E=E)


def test_radius_zero_sweep_is_the_point_zone_sweep(poly):
    """r = 0 reproduces the one-point half sweep of the C oracle (stress from the
    same displacement), decision for decision away from the threshold."""
    sp0 = poly["sp"].copy()
    sig, _, _ = O.stress_field(sp0, poly["Ct"], poly["u0"].reshape(-1, 3), poly["E"])
    lam = 3e3
    for colour in (0, 1):
        a = sp0.copy()
        b = sp0.copy()
        na, ca, da, ta = O.half_sweep(a, colour, 5, 3, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 5, 1, lam, poly["St"], sig)
        nb, cb, db, tb = Z.half_sweep_zone(b, colour, 5, 3, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 5, lam, poly["Ct"],
                                           poly["E"], poly["u0"], 0, poly["Bs"])
        assert np.abs(da - db).max() < 1e-9 * max(1.0, np.abs(da).max())
        near = np.abs(da - ta) < 1e-9 * np.maximum(1.0, np.abs(ta))
        assert np.all((ca == cb) | near)
        if not near.any():
            assert na == nb and np.array_equal(a, b)


def test_zero_elastic_scale_is_pure_potts(poly):
    sp0 = poly["sp"].copy()
    for colour in (0, 1):
        a = sp0.copy()
        b = sp0.copy()
        na, ca, _, _ = O.half_sweep(a, colour, 9, 1, 2, 1.0, 0.7, O.TRIAL_NEIGHBOR, 5, 0, 0.0, None, None)
        nb, cb, _, _ = Z.half_sweep_zone(b, colour, 9, 1, 2, 1.0, 0.7, O.TRIAL_NEIGHBOR, 5, 0.0, poly["Ct"],
                                         poly["E"], poly["u0"], 1, poly["Bs"])
        assert na == nb and np.array_equal(ca, cb) and np.array_equal(a, b)


def test_radius_one_shift_is_the_rank_six_update(poly):
    """Eq. 6 over the 27-point zone equals the rank-6 form
    1/2 e0.dC (I + G dC)^-1 e0, G = B_p K^+ B_p^T (K: zone stiffness, old
    orientations; e0: strain of the point at u0): only the point's stiffness
    changes and the old zone energy is stationary at u0."""
    sp, Ct, Bs, E, u0 = poly["sp"], poly["Ct"], poly["Bs"], poly["E"], poly["u0"]
    Cp = Z.point_stiffness(sp, Ct)
    for p in (0, 29, 131, 287):
        pts = Z.zone_points(sp.shape, p, 1)
        K, _ = Z.assemble(Bs, Cp, E, pts)
        G = Bs[p] @ np.linalg.pinv(K, rcond=1e-12) @ Bs[p].T
        q_old = int(sp.reshape(-1)[p])
        q_new = (q_old + 3) % 5
        dC = Ct[q_new] - Ct[q_old]
        e0 = E + Bs[p] @ u0
        ref = 0.5 * e0 @ dC @ np.linalg.solve(np.eye(6) + G @ dC, e0)
        got = Z.zone_shift(sp, Ct, E, u0, p, q_new, 1, Bs)
        assert abs(got - ref) < 1e-8 * abs(ref)


def test_radius_one_shift_is_the_relaxed_misfit_energy(poly):
    """The same change in the form the GPU kernel evaluates: with K' the zone
    stiffness with the point's new orientation and f = B_p^T dC e0,
    1/2 e0.dC (I + G dC)^-1 e0 = 1/2 e0.dC e0 - 1/2 f.K'^+ f (Sherman-Morrison-Woodbury:
    dC (I + G dC)^-1 = dC - dC B_p K'^+ B_p^T dC), checked against the oracle's zone
    re-solve with K' from the oracle's own assembly."""
    sp, Ct, Bs, E, u0 = poly["sp"], poly["Ct"], poly["Bs"], poly["E"], poly["u0"]
    for p in (0, 29, 131, 287):
        pts = Z.zone_points(sp.shape, p, 1)
        q_old = int(sp.reshape(-1)[p])
        q_new = (q_old + 2) % 5
        Cp2 = Z.point_stiffness(sp, Ct).copy()
        Cp2[p] = Ct[q_new]
        K2, _ = Z.assemble(Bs, Cp2, E, pts)
        dC = Ct[q_new] - Ct[q_old]
        e0 = E + Bs[p] @ u0
        f = Bs[p].T @ (dC @ e0)
        ref = 0.5 * e0 @ dC @ e0 - 0.5 * f @ np.linalg.pinv(K2, rcond=1e-12) @ f
        got = Z.zone_shift(sp, Ct, E, u0, p, q_new, 1, Bs)
        assert abs(got - ref) < 1e-8 * abs(ref)
        # the relaxation term is a real share of the change, not a rounding-level correction
        assert 0.0 < f @ np.linalg.pinv(K2, rcond=1e-12) @ f


def test_radius_one_sweep_reads_the_start_of_step(poly):
    sp0 = poly["sp"].copy()
    b = sp0.copy()
    n, ch, dH, t = Z.half_sweep_zone(b, 1, 4, 2, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 5, 3e3, poly["Ct"],
                                     poly["E"], poly["u0"], 1, poly["Bs"])
    nz, ny, nx = sp0.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    colour = ((x + y + z) & 1).reshape(-1)
    assert n == int(ch.sum()) and n > 0
    assert not ch[colour == 0].any()
    diff = (b != sp0).reshape(-1)
    assert np.array_equal(diff, ch.astype(bool))
    # each accepted trial equals the decision taken against the unchanged field
    for p in np.nonzero(ch)[0][:5]:
        xx, yy, zz = p % nx, (p // nx) % ny, p // (nx * ny)
        acc, qn, h, tt = Z.site_trial_zone(sp0, xx, yy, zz, 4, 2, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 5, 3e3,
                                           poly["Ct"], poly["E"], poly["u0"], 1, poly["Bs"])
        assert acc and b.reshape(-1)[p] == qn and h == dH[p] and tt == t[p]


def test_uniform_field_has_no_moves(poly):
    sp = np.zeros(poly["shape"], dtype=np.uint16)
    n, ch, _, _ = Z.half_sweep_zone(sp, 0, 4, 2, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 5, 3e3, poly["Ct"],
                                    poly["E"], poly["u0"], 1, poly["Bs"])
    assert n == 0 and not sp.any()


@pytest.mark.parametrize("shape", [(6, 6, 8), (8, 10, 6)])
def test_local_radius_one_shift_equals_the_global_one(shape):
    """zone_shift_local (the 27 nodes of the zone only) equals zone_shift with r = 1 on
    the whole grid's strain matrices, for sites at every parity and at the periodic wrap,
    and the local trial equals the global one decision for decision."""
    eul = S.euler_uniform_so3(5, 31)
    sp = S.voronoi_spins(shape, 6, 5, 32)
    A, Ct, St = O.tables(eul, *C3)
    Bs = Z.all_strain_matrices(shape)
    rng = np.random.default_rng(33)
    u0 = rng.normal(size=Bs.shape[2]) * 2e-4
    E = np.array([1e-3, -3e-4, -4e-4, 2e-4, -1e-4, 1e-4])
    nz, ny, nx = shape
    sites = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (1, 2, 3), (2, 1, 0), (3, 3, 3), (nx - 2, 0, nz - 1)]
    sites += [tuple(int(v) for v in rng.integers(0, [nx, ny, nz])) for _ in range(6)]
    for (x, y, z) in sites:
        p = x + nx * (y + ny * z)
        for qn in (0, 3):
            g = Z.zone_shift(sp, Ct, E, u0, p, qn, 1, Bs)
            l = Z.zone_shift_local(sp, Ct, E, u0.reshape(-1, 3), x, y, z, qn)
            assert abs(g - l) <= 1e-10 * abs(g) + 1e-15, (x, y, z, qn, g, l)
        a = Z.site_trial_zone(sp, x, y, z, 7, 2, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 5, 3e3, Ct, E, u0, 1, Bs)
        b = Z.site_trial_zone_local(sp, x, y, z, 7, 2, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 5, 3e3, Ct, E, u0)
        assert a[0] == b[0] and a[1] == b[1]
        assert abs(a[2] - b[2]) <= 1e-9 * max(1.0, abs(a[2]))
