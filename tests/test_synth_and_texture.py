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
