"""Synthetic inputs and the oracle's texture measures (CPU only)."""
import numpy as np

import hmc_synth as S
import oracle as O


def test_voronoi_tree_matches_brute_force():
    for shape, ns, seed in (((10, 12, 14), 40, 1), ((16, 16, 16), 300, 2), ((6, 8, 4), 3, 3)):
        pos, _ = S.voronoi_seeds(shape, ns, 8, seed)
        assert (S.voronoi_owner(shape, pos) == S.voronoi_owner_brute(shape, pos)).all()


def test_voronoi_tie_goes_to_lowest_index():
    shape = (2, 2, 4)
    pos = np.array([[0.5, 0.5, 0.5], [2.5, 0.5, 0.5], [0.5, 0.5, 0.5]])  # duplicate of seed 0
    own = S.voronoi_owner_brute(shape, pos)
    assert 2 not in own.tolist()


def test_euler_uniform_on_so3():
    e = S.euler_uniform_so3(20000, 5)
    A = np.stack([O.euler_to_A(*t) for t in e[:4000]])
    # uniform rotations: E[A] = 0 and E[A_ij^2] = 1/3
    assert np.abs(A.mean(axis=0)).max() < 0.03
    assert np.abs((A ** 2).mean(axis=0) - 1 / 3).max() < 0.03


def test_texture_histograms():
    eul = S.euler_uniform_so3(50, 2)
    A, Ct, St = O.tables(eul, 246.5, 147.3, 124.7)
    sp = S.voronoi_spins((16, 16, 16), 60, 50, 3)
    counts = O.orientation_counts(sp, 50)
    assert counts.sum() == sp.size
    assert (counts == np.bincount(sp.ravel(), minlength=50)).all()
    n = (1, 1, 1)
    ang = O.angle_to_nearest_100(A, n)
    assert ang.max() <= np.degrees(np.arccos(1 / np.sqrt(3))) + 1e-9
    for kind, nb in ((0, 50), (1, 9), (2, 10)):
        f = O.texture_histogram(kind, nb, counts, A, St, n, 246.5, 147.3, 124.7)
        assert abs(f.sum() - 1) < 1e-15
    f1 = O.texture_histogram(1, 9, counts, A, St, n, 246.5, 147.3, 124.7)
    assert (f1[6:] == 0).all()
    E = O.young_modulus_along(St, n)
    d = (246.5 - 147.3) * (246.5 + 2 * 147.3)
    S11 = (246.5 + 147.3) / d
    assert E.min() >= 1 / S11 - 1e-9


def _rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _ry(b):
    c, s = np.cos(b), np.sin(b)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def test_angle_to_nearest_100_rotation_about_z():
    """Sec. "Results" (single-angle orientation set, load along x): a crystal turned by phi
    about z has its [100] axis at phi and its [010] axis at 90 - phi from x, so the angle
    to the nearest <100> is min(phi, 90 - phi)."""
    phi = np.radians(np.arange(0, 90, 3) + 0.25)
    A = np.stack([O.euler_to_A(p, 0.0, 0.0) for p in phi])
    want = np.minimum(np.degrees(phi), 90.0 - np.degrees(phi))
    assert np.allclose(O.angle_to_nearest_100(A, (1, 0, 0)), want, rtol=0, atol=1e-9)
    assert np.allclose(O.angle_to_nearest_100(A, (0, 1, 0)), want, rtol=0, atol=1e-9)
    # the z axis is a crystal <100> axis for every rotation about z
    assert np.allclose(O.angle_to_nearest_100(A, (0, 0, 1)), 0.0, rtol=0, atol=1e-6)


def test_angle_to_nearest_100_uses_crystal_axes_as_columns():
    """A maps crystal-frame vectors to the sample frame (Eq. 18, z-y-z), so the crystal
    axes in the sample frame are the columns of A: the cosine of the angle between the
    load axis x and crystal axis j is A[0, j], the first ROW of A.  For Euler angles
    (0.3, 0.7, 1.1) the first row and the first column give different angles (38.3
    against 17.5 degrees), so taking rows for columns fails here."""
    f, t, p = 0.3, 0.7, 1.1
    cf, sf, ct, st, cp, sp = np.cos(f), np.sin(f), np.cos(t), np.sin(t), np.cos(p), np.sin(p)
    # Rz(f) Ry(t) Rz(p) multiplied out by hand: first row and first column
    row0 = np.array([cf * ct * cp - sf * sp, -cf * ct * sp - sf * cp, cf * st])
    col0 = np.array([cf * ct * cp - sf * sp, sf * ct * cp + cf * sp, -st * cp])
    A = _rz(f) @ _ry(t) @ _rz(p)
    assert np.allclose(A[0], row0) and np.allclose(A[:, 0], col0)
    want = np.degrees(np.arccos(np.abs(row0).max()))
    wrong = np.degrees(np.arccos(np.abs(col0).max()))
    assert abs(want - 38.2575) < 1e-3 and abs(wrong - 17.4598) < 1e-3
    got = O.angle_to_nearest_100(O.euler_to_A(f, t, p)[None], (1, 0, 0))[0]
    assert abs(got - want) < 1e-9
    # the same angle from the crystal-frame direction cosines of the load axis, A^T x
    l = A.T @ np.array([1.0, 0.0, 0.0])
    assert abs(np.degrees(np.arccos(np.abs(l).max())) - got) < 1e-9


def test_angle_histogram_of_the_z_rotation_set():
    """ANGLE_100 fractions of 90 equal-volume orientations at phi = k + 1/2 degrees about
    z, load along x: the angles are min(k + 1/2, 89.5 - k), so each 10-degree bin below
    40 degrees holds 20 of them, the 40-50 bin 10, and the bins above 45 degrees none."""
    eul = np.stack([np.radians(np.arange(90) + 0.5), np.zeros(90), np.zeros(90)], axis=1)
    A, Ct, St = O.tables(eul, 246.5, 147.3, 124.7)
    counts = np.full(90, 7, dtype=np.int64)
    f = O.texture_histogram(1, 9, counts, A, St, (1, 0, 0), 246.5, 147.3, 124.7)
    want = np.array([20, 20, 20, 20, 10, 0, 0, 0, 0]) / 90.0
    assert np.array_equal(f, want)


def test_box_grain_spins_match_their_definition():
    """Box grains: voxel (x, y, z) takes (a[x // e] ^ b[y // e] ^ c[z // e]) mod Q, here
    evaluated voxel by voxel, with a grid whose edges are not multiples of e."""
    shape, e, Q, seed = (13, 10, 22), 4, 37, 5
    got = S.box_grain_spins(shape, e, Q, seed)
    nz, ny, nx = shape
    rng = np.random.default_rng([0x5EED, 5, seed])
    a = rng.integers(0, 1 << 16, size=nx // e + 1, dtype=np.uint32)
    b = rng.integers(0, 1 << 16, size=ny // e + 1, dtype=np.uint32)
    c = rng.integers(0, 1 << 16, size=nz // e + 1, dtype=np.uint32)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                assert got[z, y, x] == (int(a[x // e]) ^ int(b[y // e]) ^ int(c[z // e])) % Q
    assert got.dtype == np.uint16 and got.max() < Q
