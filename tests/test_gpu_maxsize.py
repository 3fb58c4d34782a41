"""Parity at the largest sizes the library accepts, on sampled outputs the oracle
computes one by one (box-grain fields, FP32, one-point traction zone):

* 640 x 768 x 768 (3.8e8 sites, 4.7e7 cells): the colour-packed stress holds 48 x 4.7e7 =
  2.3e9 elements, past 2^31, so every stress offset must be 64-bit; a stress pass and a
  half sweep from rest, then one explicit step on sampled nodes;
* 1026 x 1024 x 2048 (2.15e9 sites, the grid limit is 2^32 - 1): site indices past 2^31
  (the Philox counter and the natural-order spin field); a stress pass and a half sweep on
  sampled sites, the other colour untouched, and the orientation volumes exact.

At rest (u = 0) a site's stress is C'(q) Ebar, which the oracle forms on a one-orientation
4^3 grid; no oracle input comes from the CUDA path.  The autotuner is off (its scratch
copies would double the device memory at these sizes)."""
import numpy as np
import pytest

import hmc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu

C3 = dict(c11=246.5, c12=147.3, c44=124.7)
AXIS, STRAIN, SEED, Q = (1.0, 1.0, 1.0), 2e-3, 99, 64


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def _handle(G, shape, spins, euler):
    g = G.HMC(shape, Q, precision=G.HMC_FP32, J=1.0, kT=0.7, load_axis=AXIS, strain=STRAIN,
              mpm_steps_per_mcs=50, seed=SEED, **C3)
    g.set_orientations(euler, spins)
    A, Ct, St = O.tables(euler, C3["c11"], C3["c12"], C3["c44"])
    counts = np.zeros(Q, dtype=np.int64)
    for z in range(spins.shape[0]):
        counts += np.bincount(spins[z].ravel(), minlength=Q)
    E = O.initial_uniaxial_strain(O.reuss_compliance(St, counts), AXIS, STRAIN)
    assert np.abs(g.strain() - E).max() < 1e-12 * np.abs(E).max()
    return g, Ct, St, E


def _check_half_sweep(after, spins, colour, Ct, St, E, extra, n_random=1500):
    """Sampled decisions against the oracle's own, each with the oracle's stress at rest."""
    nz, ny, nx = spins.shape
    lam = O.elastic_scale(max(spins.shape))
    zeros = np.zeros((8, 3))
    sig = {}

    def sigma(q):
        if q not in sig:
            sig[q] = O.point_stress(np.full((4, 4, 4), q, dtype=np.uint16), Ct, zeros, E, 0, 0, 0)
        return sig[q]

    rng = np.random.default_rng(31)
    sites = [tuple(int(v) for v in rng.integers(0, [nx, ny, nz])) for _ in range(n_random)] + list(extra)
    n = mis = changed = 0
    for (x, y, z) in sites:
        if (x + y + z) & 1 != colour:
            x = (x + 1) % nx
        q = int(spins[z, y, x])
        acc, qn, dH, t = O.site_trial_at(spins, x, y, z, SEED, 0, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, Q, 1, lam, St,
                                         sigma(q))
        want = qn if acc else q
        n += 1
        changed += int(want != q)
        if after[z, y, x] != want:
            mis += 1
            assert t >= 0 and abs(dH - t) <= 1e-4 * max(1.0, abs(t)), (x, y, z, dH, t)
    assert mis <= max(2, 1e-3 * n)
    assert changed > 0
    # the other colour untouched, one plane at a time
    par = (np.arange(ny)[:, None] + np.arange(nx)[None, :]) & 1
    for z in range(nz):
        other = par != ((colour + z) & 1)
        assert (after[z][other] == spins[z][other]).all(), z


def test_stress_offsets_past_2e31_elements(G, monkeypatch):
    monkeypatch.setenv("HMC_AUTOTUNE", "0")
    shape = (640, 768, 768)
    nz, ny, nx = shape
    assert 48 * (nx // 2) * (ny // 2) * (nz // 2) > 2 ** 31
    spins = S.box_grain_spins(shape, 8, Q, 11)
    euler = S.euler_uniform_so3(Q, 12)
    g, Ct, St, E = _handle(G, shape, spins, euler)
    g.compute_stress()
    g.sweep_half(1)
    after = g.spins()
    last = [(nx - 1, ny - 1, nz - 1), (nx - 2, ny - 1, nz - 1), (0, 0, nz - 1), (nx - 1, 0, nz // 2)]
    _check_half_sweep(after, spins, 1, Ct, St, E, last)
    del after
    # one explicit step from rest on the original spins: v = dt f / m, u = dt v (m = 8)
    g.set_spins(spins)
    g.mpm_steps(1)
    ug, vg = g.nodal()
    nbx, nby, nbz = nx // 2, ny // 2, nz // 2
    u0 = np.zeros((nbx * nby * nbz, 3))
    dt = O.default_dt(**C3)
    rng = np.random.default_rng(32)
    nodes = [tuple(int(v) for v in rng.integers(0, [nbx, nby, nbz])) for _ in range(300)]
    nodes += [(nbx - 1, nby - 1, nbz - 1), (0, nby - 1, nbz - 1), (nbx - 1, 0, nbz - 2), (3, 4, nbz - 1)]
    du, dv, ru, rv = [], [], [], []
    for (i, j, k) in nodes:
        I = i + nbx * (j + nby * k)
        f = O.node_force(spins, Ct, u0, E, i, j, k)
        v = dt * f / 8.0
        u = dt * v
        du.append(ug[I] - u)
        dv.append(vg[I] - v)
        ru.append(u)
        rv.append(v)
    assert np.linalg.norm(rv) > 0
    assert np.linalg.norm(np.array(dv)) < 1e-5 * np.linalg.norm(rv)
    assert np.linalg.norm(np.array(du)) < 1e-5 * np.linalg.norm(ru) + 1e-12
    g.close()


def test_site_indices_past_2e31(G, monkeypatch):
    monkeypatch.setenv("HMC_AUTOTUNE", "0")
    shape = (1026, 1024, 2048)
    nz, ny, nx = shape
    assert 2 ** 31 < nx * ny * nz < 2 ** 32
    spins = S.box_grain_spins(shape, 8, Q, 13)
    euler = S.euler_uniform_so3(Q, 14)
    g, Ct, St, E = _handle(G, shape, spins, euler)
    g.compute_stress()
    g.sweep_half(0)
    after = g.spins()
    # sites whose linear index is 2^31 or more (z >= 1024), the last site, and a few before 2^31
    rng = np.random.default_rng(33)
    past = [(int(rng.integers(0, nx)), int(rng.integers(0, ny)), 1024 + int(rng.integers(0, 2))) for _ in range(500)]
    past += [(nx - 1, ny - 1, nz - 1), (0, 0, 1024), (nx - 2, ny - 1, 1023)]
    _check_half_sweep(after, spins, 0, Ct, St, E, past, n_random=500)
    _, counts = g.texture_histogram(G.HMC_HIST_ANGLE_100, 9)
    want = np.zeros(Q, dtype=np.int64)
    for z in range(nz):
        want += np.bincount(after[z].ravel(), minlength=Q)
    assert (counts == want).all() and counts.sum() == nx * ny * nz
    g.close()
