"""Oracle pins for the Potts / Metropolis sweep and the elastic shift (CPU only)."""
from fractions import Fraction
import math

import numpy as np
import pytest

import hmc_synth as S
import oracle as O
import oracle.zone as Z

C3 = (246.5, 147.3, 124.7)


def _unlike_bonds_numpy(s):
    return int(sum((s != np.roll(s, -1, axis=a)).sum() for a in range(3)))


def test_unlike_bonds_brute_force():
    for seed in range(3):
        s = S.random_spins((6, 8, 10), 4, seed)
        assert O.unlike_bonds(s) == _unlike_bonds_numpy(s)


def test_integer_threshold_equals_float_rule():
    """r1 < T(k) exactly when (r1 + 1/2) 2^-32 < exp(-k J / kT), in exact rational arithmetic."""
    for kT in (0.7, 1.0, 2.6, 0.05):
        for k in range(1, 7):
            T = O.accept_threshold(k, 1.0, kT)
            p = Fraction(math.exp(-k / kT))
            assert T == int(T)
            T = int(T)
            if T > 0:
                assert (Fraction(T - 1) + Fraction(1, 2)) / 2 ** 32 < p
            assert not ((Fraction(T) + Fraction(1, 2)) / 2 ** 32 < p)
    assert O.accept_threshold(3, 1.0, 0.0) == 0.0
    assert O.accept_threshold(0, 1.0, 0.7) == 2 ** 32
    # acceptance probabilities e^(-k / 0.7) for k = 1..5, to four digits
    for k, pk in zip(range(1, 6), (0.2397, 0.0574, 0.0138, 0.0033, 0.00079)):
        assert abs(O.accept_threshold(k, 1.0, 0.7) / 2 ** 32 - pk) < 0.0005 * max(1, pk * 100)


def test_local_energy_change_equals_global_recount():
    rng = np.random.default_rng(2)
    s = S.voronoi_spins((8, 8, 8), 12, 5, 4)
    for _ in range(200):
        x, y, z = rng.integers(0, 8, size=3)
        acc, qn, dH, t = O.site_trial(s, x, y, z, 9, int(rng.integers(1000)), 0, 1.0, 0.7,
                                      O.TRIAL_NEIGHBOR, 5, 0, 0.0, None, None)
        s2 = s.copy()
        s2[z, y, x] = qn
        assert dH == O.unlike_bonds(s2) - O.unlike_bonds(s)
        nbrs = {s[z, y, (x - 1) % 8], s[z, y, (x + 1) % 8], s[z, (y - 1) % 8, x], s[z, (y + 1) % 8, x],
                s[(z - 1) % 8, y, x], s[(z + 1) % 8, y, x]}
        assert qn in nbrs


def test_metropolis_acceptance_frequency():
    """Site spin a with neighbours (a,a,a,a,b,b): trial b with probability 1/3 and
    Delta E = 2, accepted with probability exp(-2/0.7)."""
    s = np.zeros((4, 4, 4), dtype=np.uint16)
    s[1, 1, 0] = 1  # -x neighbour of (1,1,1)
    s[1, 0, 1] = 1  # -y neighbour
    n = 40000
    acc = sum(O.site_trial(s, 1, 1, 1, 123, m, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 2, 0, 0.0, None, None)[0]
              for m in range(n))
    p = math.exp(-2 / 0.7) / 3
    assert abs(acc / n - p) < 5 * math.sqrt(p * (1 - p) / n)


def test_uniform_trial_draw():
    s = np.zeros((4, 4, 4), dtype=np.uint16)
    qs = [O.site_trial(s, 0, 0, 0, 5, m, 0, 1.0, 1e9, O.TRIAL_UNIFORM_Q, 7, 0, 0.0, None, None)[1]
          for m in range(7000)]
    cnt = np.bincount(qs, minlength=7)
    assert cnt.min() > 850 and cnt.max() < 1150


def test_half_sweep_colour_and_volume_conservation():
    s = S.voronoi_spins((8, 10, 12), 20, 9, 6)
    z, y, x = np.meshgrid(range(8), range(10), range(12), indexing="ij")
    colour = (x + y + z) & 1
    total = s.size
    for c in (0, 1, 0, 1):
        before = s.copy()
        cnt0 = O.orientation_counts(before, 9)
        acc, changed, _, _ = O.half_sweep(s, c, 77, 3, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 9, 0, 0.0, None, None)
        diff = (s != before)
        assert not diff[colour != c].any()
        assert diff.sum() == acc == changed.sum()
        cnt1 = O.orientation_counts(s, 9)
        assert cnt1.sum() == total
        delta = np.zeros(9, dtype=np.int64)
        np.add.at(delta, before[diff], -1)
        np.add.at(delta, s[diff], 1)
        assert (cnt1 - cnt0 == delta).all()


def test_flat_bicrystal_is_frozen_at_zero_temperature():
    s = np.zeros((8, 8, 8), dtype=np.uint16)
    s[:, :, 4:] = 1  # two flat periodic boundaries normal to x
    for m in range(20):
        for c in (0, 1):
            O.half_sweep(s, c, 5, m, 0, 1.0, 0.0, O.TRIAL_NEIGHBOR, 2, 0, 0.0, None, None)
    assert (s[:, :, :4] == 0).all() and (s[:, :, 4:] == 1).all()


def test_point_zone_shift_reduces_to_bar_formula():
    """Uniaxial stress s along x, orientations with moduli E1, E2 along x:
    shift = 1/2 s^2 (1/E1 - 1/E2) (Eq. 21, magnitude), positive when going soft -> stiff."""
    eul = np.array([[0.0, 0, 0], [np.radians(45.0), 0, 0]])  # soft <100> and stiff <110> along x
    A, Ct, St = O.tables(eul, 250.8, 150.0, 123.5)
    E = O.young_modulus_along(St, [1, 0, 0])
    assert E[0] < E[1]
    s = 0.03  # 30 MPa
    sig = np.array([s, 0, 0, 0, 0, 0])
    d = O.point_zone_shift(St[0], St[1], sig)
    assert abs(d - 0.5 * s * s * (1 / E[0] - 1 / E[1])) < 1e-15
    assert d > 0  # soft -> stiff costs energy: the softer grain grows


def test_elastic_sweep_with_zero_stress_is_pure_potts():
    s = S.voronoi_spins((8, 8, 8), 10, 6, 2)
    _, Ct, St = O.tables(S.euler_uniform_so3(6, 3), *C3)
    a, b = s.copy(), s.copy()
    zero = np.zeros((s.size, 6))
    for m in range(4):
        for c in (0, 1):
            O.half_sweep(a, c, 3, m, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 6, 0, 0.0, None, None)
            O.half_sweep(b, c, 3, m, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 6, 1, 1e4, St, zero)
    assert (a == b).all()


def test_elastic_threshold_rule():
    """With the elastic term on, accept iff dH <= -kT ln u, u = (r1 + 1/2) 2^-32."""
    rng = np.random.default_rng(3)
    s = S.voronoi_spins((8, 8, 8), 10, 6, 2)
    _, Ct, St = O.tables(S.euler_uniform_so3(6, 3), *C3)
    sig = rng.normal(size=(s.size, 6)) * 0.2
    for _ in range(100):
        x, y, z = rng.integers(0, 8, size=3)
        m = int(rng.integers(100))
        acc, qn, dH, t = O.site_trial(s, x, y, z, 9, m, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 6, 1, 5e3, St, sig)
        if qn == s[z, y, x]:
            continue
        p = x + 8 * (y + 8 * z)
        r = O.site_draws(8, 8, x, y, z, 9, m, 0, O.TRIAL_NEIGHBOR)
        u = (float(r[1]) + 0.5) / 2 ** 32
        assert abs(t + 0.7 * math.log(u)) < 1e-15
        assert acc == (dH <= t)


@pytest.fixture(scope="module")
def small_poly():
    shape = (6, 6, 6)
    eul = S.euler_uniform_so3(5, 11)
    sp = S.voronoi_spins(shape, 5, 5, 12)
    A, Ct, St = O.tables(eul, *C3)
    Bs = Z.all_strain_matrices(shape)
    return dict(shape=shape, sp=sp, A=A, Ct=Ct, St=St, Bs=Bs)


def test_zone_radius_zero_is_point_zone_closed_form(small_poly):
    """Eq. 6 with Omega_1 = one point equals w(q_old) - w(q_new) at any state."""
    rng = np.random.default_rng(4)
    E = np.array([-4e-4, -4e-4, 1.2e-3, 0, 1e-4, 0])
    u0 = rng.normal(size=small_poly["Bs"].shape[2]) * 1e-4
    for p in (0, 17, 100, 215):
        q_old = int(small_poly["sp"].reshape(-1)[p])
        q_new = (q_old + 2) % 5
        x, y, z = p % 6, (p // 6) % 6, p // 36
        sig = O.point_stress(small_poly["sp"], small_poly["Ct"], u0.reshape(-1, 3), E, x, y, z)
        ref = O.point_zone_shift(small_poly["St"][q_old], small_poly["St"][q_new], sig)
        got = Z.zone_shift(small_poly["sp"], small_poly["Ct"], E, u0, p, q_new, 0, small_poly["Bs"])
        assert abs(got - ref) < 1e-10 * abs(ref)


def test_whole_domain_zone_is_brute_force_resolve(small_poly):
    E = np.array([-4e-4, -4e-4, 1.2e-3, 0, 1e-4, 0])
    Cp = Z.point_stiffness(small_poly["sp"], small_poly["Ct"])
    u0, _ = Z.equilibrium(small_poly["Bs"], Cp, E)
    for p in (3, 90):
        q_old = int(small_poly["sp"].reshape(-1)[p])
        q_new = (q_old + 1) % 5
        bf = Z.brute_force_shift(small_poly["sp"], small_poly["Ct"], E, p, q_new, small_poly["Bs"])
        zs = Z.zone_shift(small_poly["sp"], small_poly["Ct"], E, u0, p, q_new, -1, small_poly["Bs"])
        assert abs(zs - bf) < 1e-10 * abs(bf)


def test_brute_force_favours_the_softer_orientation():
    """Fixed mean strain along z: replacing a stiff point by a soft one lowers the energy."""
    shape = (6, 6, 6)
    eul = np.array([[0.0, 0, 0], [0.0, np.arccos(1 / np.sqrt(3)), np.pi / 4]])  # <100> and <111> along z
    _, Ct, St = O.tables(eul, *C3)
    E_axis = O.young_modulus_along(St, [0, 0, 1])
    assert E_axis[0] < E_axis[1]
    sp = np.ones(shape, dtype=np.uint16)
    sp[:, :, :3] = 0
    E = np.array([0, 0, 1e-3, 0, 0, 0.0])
    p = 4 + 6 * (2 + 6 * 2)  # a stiff point
    assert Z.brute_force_shift(sp, Ct, E, p, 0) < 0
