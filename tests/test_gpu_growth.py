"""Grain count on the GPU against the oracle, and the grain-growth validation of
Sec. "Microstructural Evolution" on the GPU path: 60^3 lattice, 99 random
orientations, kT/J = 1, pure Potts red/black steps; V^(3/2) = c2 t after the
transient, and the red/black mobility above that of the Gauss-Seidel update."""
import numpy as np
import pytest

import hmc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def _fields(shape):
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    nx = shape[2]
    yield np.zeros(shape, dtype=np.uint16)
    yield ((x + y + z) & 1).astype(np.uint16)
    yield ((x == 0) | (x == nx - 1)).astype(np.uint16)
    yield S.random_spins(shape, 3, 4)
    yield S.voronoi_spins(shape, 40, 7, 5)


@pytest.mark.parametrize("shape", [(4, 6, 8), (12, 10, 34), (64, 64, 64)])
def test_grain_count_matches_oracle(G, shape):
    g = G.HMC(shape, 7, elastic=0, mpm_steps_per_mcs=0)
    for f in _fields(shape):
        g.set_orientations(S.euler_uniform_so3(7, 1), f)
        assert g.grain_count() == O.grain_count(f)
    g.close()


def test_grain_growth_validation(G):
    shape, Q, kT = (60, 60, 60), 99, 1.0
    sp0 = S.random_spins(shape, Q, 1)
    g = G.HMC(shape, Q, J=1.0, kT=kT, elastic=0, mpm_steps_per_mcs=0, seed=7)
    g.set_orientations(S.euler_uniform_so3(Q, 1), sp0)
    o = sp0.copy()
    t, V = [], []
    for m in range(1, 301):
        g.mc_sweeps(1)
        if m % 25 == 0:
            t.append(m)
            V.append(o.size / g.grain_count())
    # the pure Potts path is bit-exact with the oracle's red/black step
    for m in range(300):
        O.half_sweep(o, 0, 7, m, 0, 1.0, kT, O.TRIAL_NEIGHBOR, Q, 0, 0.0, None, None)
        O.half_sweep(o, 1, 7, m, 0, 1.0, kT, O.TRIAL_NEIGHBOR, Q, 0, 0.0, None, None)
    assert (g.spins() == o).all()
    assert abs(V[-1] - o.size / O.grain_count(o)) == 0
    t = np.array(t, dtype=float)
    V = np.array(V)
    sel = t >= 100
    c2_rb, _ = np.polyfit(t[sel], V[sel] ** 1.5, 1)
    assert np.corrcoef(t[sel], V[sel] ** 1.5)[0, 1] > 0.99
    assert np.all(np.diff(V) > 0)
    # Gauss-Seidel steps from the same start on the oracle
    gs = sp0.copy()
    tg, Vg = [], []
    for m in range(1, 301):
        O.gs_sweep(gs, 7, m, 0, 1.0, kT, O.TRIAL_NEIGHBOR, Q)
        if m % 25 == 0:
            tg.append(m)
            Vg.append(gs.size / O.grain_count(gs))
    tg = np.array(tg, dtype=float)
    Vg = np.array(Vg)
    c2_gs, _ = np.polyfit(tg[tg >= 100], Vg[tg >= 100] ** 1.5, 1)
    assert np.corrcoef(tg[tg >= 100], Vg[tg >= 100] ** 1.5)[0, 1] > 0.99
    assert c2_rb > 1.5 * c2_gs, (c2_rb, c2_gs)
    g.close()
