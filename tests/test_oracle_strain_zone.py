"""Oracle pins of the constant-strain one-point zone (Eq. 8 with the point's
strain held fixed): 1/2 e.(C'(q') - C'(q)).e with e = S'(q) sigma."""
import math

import numpy as np

import hmc_synth as S
import oracle as O

C3 = dict(c11=246.5, c12=147.3, c44=124.7)


def test_closed_form_100_to_45_degrees_about_z():
    """Uniaxial sigma along x on a <100> crystal, trial rotated 45 degrees about
    z: C'11 - C11 = -(C'12 - C12) = C44 - (C11 - C12)/2 and the other changed
    entries vanish, so the shift is 1/2 (C44 - (C11 - C12)/2) sigma^2 (S11 - S12)^2."""
    eul = np.array([[0.0, 0.0, 0.0], [math.pi / 4, 0.0, 0.0]])
    _, Ct, St = O.tables(eul, *C3.values())
    sig = np.array([0.3, 0, 0, 0, 0, 0])
    c11, c12, c44 = C3["c11"], C3["c12"], C3["c44"]
    d = (c11 - c12) * (c11 + 2 * c12)
    S11, S12 = (c11 + c12) / d, -c12 / d
    ref = 0.5 * (c44 - 0.5 * (c11 - c12)) * 0.3 ** 2 * (S11 - S12) ** 2
    got = O.point_strain_shift(St[0], Ct[0], Ct[1], sig)
    assert ref > 0 and abs(got - ref) < 1e-12 * ref   # the stiffer orientation along x costs energy


def test_first_order_agrees_with_the_traction_zone():
    """Both zones are 1/2 e.dC.e to first order in dC: for a small rotation of a
    generic orientation under a generic stress the two shifts agree to O(dC)."""
    rng = np.random.default_rng(3)
    base = S.euler_uniform_so3(1, 5)[0]
    sig = rng.normal(size=6) * 0.2
    for eps in (1e-3, 1e-4):
        eul = np.array([base, base + np.array([eps, 0.7 * eps, -0.4 * eps])])
        _, Ct, St = O.tables(eul, *C3.values())
        a = O.point_strain_shift(St[0], Ct[0], Ct[1], sig)
        b = O.point_zone_shift(St[0], St[1], sig)
        assert abs(a - b) < 20 * eps * abs(b), (eps, a, b)


def test_strain_sweep_with_zero_stress_is_pure_potts():
    shape = (6, 8, 10)
    Q = 6
    eul = S.euler_uniform_so3(Q, 3)
    _, Ct, St = O.tables(eul, *C3.values())
    sp = S.voronoi_spins(shape, 8, Q, 4)
    a, b = sp.copy(), sp.copy()
    na, ca, _, _ = O.half_sweep(a, 0, 5, 1, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, Q, 0, 0.0, None, None)
    nb, cb, _, _ = O.half_sweep(b, 0, 5, 1, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, Q, O.ELASTIC_STRAIN, 3e3, St,
                                np.zeros((sp.size, 6)), Ct)
    assert na == nb and np.array_equal(ca, cb) and np.array_equal(a, b)


def test_strain_sweep_uses_the_strain_shift():
    shape = (6, 8, 10)
    Q = 6
    eul = S.euler_uniform_so3(Q, 3)
    _, Ct, St = O.tables(eul, *C3.values())
    sp = S.voronoi_spins(shape, 8, Q, 4)
    rng = np.random.default_rng(1)
    sig = rng.normal(size=(sp.size, 6)) * 0.05
    lam = 2e3
    a = sp.copy()
    n, ch, dH, t = O.half_sweep(a, 1, 5, 2, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, Q, O.ELASTIC_STRAIN, lam, St, sig, Ct)
    checked = 0
    for p in range(sp.size):
        x, y, z = p % 10, (p // 10) % 8, p // 80
        if (x + y + z) % 2 != 1:
            continue
        acc, qn, h, tt = O.site_trial_at(sp, x, y, z, 5, 2, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, Q, O.ELASTIC_STRAIN,
                                         lam, St, sig[p], Ct)
        if qn == sp.reshape(-1)[p]:
            continue
        q = int(sp.reshape(-1)[p])
        nb = [sp[z, y, (x - 1) % 10], sp[z, y, (x + 1) % 10], sp[z, (y - 1) % 8, x], sp[z, (y + 1) % 8, x],
              sp[(z - 1) % 6, y, x], sp[(z + 1) % 6, y, x]]
        dE = sum(v == q for v in nb) - sum(v == qn for v in nb)
        shift = lam * O.point_strain_shift(St[q], Ct[q], Ct[qn], sig[p])
        assert abs(h - (dE + shift)) < 1e-12 * max(1.0, abs(h))
        assert h == dH[p] and acc == bool(ch[p])
        checked += 1
    assert checked > 20
