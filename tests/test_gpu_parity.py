"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle."""
import numpy as np
import pytest

import hmc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu

C3 = dict(c11=246.5, c12=147.3, c44=124.7)


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def make_pair(G, shape, Q, precision, *, seed=11, n_seeds=30, axis=(0, 0, 1.0), strain=2e-3, elastic=1,
              trial=0, n_mpm=5, kT=0.7, bc=0, strain6=None, lam=None):
    eul = S.euler_uniform_so3(Q, seed)
    spins = S.voronoi_spins(shape, n_seeds, Q, seed)
    nz, ny, nx = shape
    dt = O.default_dt(**C3)
    lam = O.elastic_scale(max(shape)) if lam is None else lam
    kw = dict(J=1.0, kT=kT, bc=bc, load_axis=tuple(axis), strain=strain, elastic=elastic, trial=trial,
              mpm_steps_per_mcs=n_mpm, dt=dt, damping=0.05, elastic_scale=lam, seed=seed * 7919 + 3)
    if strain6 is not None:
        kw["strain6"] = tuple(strain6)
    g = G.HMC(shape, Q, precision=precision, **kw, **C3)
    g.set_orientations(eul, spins)
    o = O.OracleHMC(shape, Q, J=1.0, kT=kT, bc=bc, load_axis=axis, strain=strain, strain6=strain6,
                    elastic_scale_=lam, elastic=elastic, trial=trial, mpm_steps_per_mcs=n_mpm, dt=dt,
                    damping=0.05, seed=seed * 7919 + 3, **C3)
    o.set_orientations(eul, spins)
    return g, o


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("shape,trial", [((20, 36, 70), 0), ((4, 6, 34), 0), ((10, 10, 12), 1), ((6, 34, 8), 1)])
def test_pure_potts_bit_exact(G, shape, trial):
    g, o = make_pair(G, shape, 7, G.HMC_FP32, elastic=0, trial=trial, n_mpm=0, n_seeds=12)
    for m in range(4):
        a_g = g.mc_sweeps(1)
        a_o = o.mc_sweeps(1)
        assert a_g == a_o
        assert (g.spins() == o.spins).all(), f"MCS {m}"
    assert g.info().mcs == 4


@pytest.mark.parametrize("trial", [0, 1])
def test_pure_potts_bit_exact_16bit_orientations(G, trial):
    """Orientation indices over the whole 16-bit range (Q = 65535, grains on both sides of
    32768): the bond counts compare orientations as 16-bit halves of packed pairs, so no
    high bit may leak between halves."""
    shape = (8, 12, 34)
    g, o = make_pair(G, shape, 65535, G.HMC_FP32, elastic=0, trial=trial, n_mpm=0, n_seeds=16)
    assert (o.spins >= 32768).any() and (o.spins < 32768).any()
    for m in range(3):
        assert g.mc_sweeps(1) == o.mc_sweeps(1)
        assert (g.spins() == o.spins).all(), f"MCS {m}"


def test_defaults_agree_with_oracle(G):
    g = G.HMC((32, 32, 32), 4)
    i = g.info()
    assert abs(i.dt - O.default_dt(**C3)) < 1e-15
    assert abs(i.damping - O.DEFAULT_DAMPING) < 1e-15
    assert abs(i.elastic_scale - O.elastic_scale(32)) < 1e-9 * i.elastic_scale


def test_zero_load_hybrid_is_pure_potts(G):
    shape = (12, 18, 36)
    g0, o = make_pair(G, shape, 9, G.HMC_FP32, elastic=0, n_mpm=3, strain=0.0)
    g1, _ = make_pair(G, shape, 9, G.HMC_FP32, elastic=1, n_mpm=3, strain=0.0)
    for m in range(3):
        g0.mc_sweeps(1)
        g1.mc_sweeps(1)
        o.mc_sweeps(1)
        s = o.spins
        assert (g0.spins() == s).all() and (g1.spins() == s).all()
    assert np.abs(g1.stress()).max() == 0.0


def _random_state(o, rng, scale=2e-4):
    u = rng.normal(size=(o.nnodes, 3)) * scale
    v = rng.normal(size=(o.nnodes, 3)) * scale
    return u, v


@pytest.mark.parametrize("precision,steps,tol", [(0, 20, 1e-12), (1, 200, 1e-4)])
def test_mpm_parity(G, precision, steps, tol):
    shape = (18, 38, 70)
    E6 = [-4e-4, -3e-4, 1e-3, 1e-4, -2e-4, 5e-5]
    g, o = make_pair(G, shape, 16, precision, bc=1, strain6=E6, n_mpm=0)
    rng = np.random.default_rng(5)
    u, v = _random_state(o, rng)
    g.set_nodal(u, v)
    o.u, o.v = u.copy(), v.copy()
    g.mpm_steps(steps)
    o.mpm_steps(steps)
    ug, vg = g.nodal()
    assert rel(ug, o.u) < tol and rel(vg, o.v) < tol
    mean_g, W_g = g.compute_stress()
    sig_o = o.stress()
    assert rel(g.stress(), sig_o) < tol
    assert rel(mean_g, o.mean_sig) < tol
    assert abs(W_g - o.W) < tol * abs(o.W)


@pytest.mark.parametrize("Q", [1024, 1100])
def test_mpm_parity_large_orientation_sets(G, Q):
    """The FP32 step holds the orientation table of its cubic form in shared memory up to
    1024 orientations and reads it from global memory beyond: both paths against the
    FP64 oracle after 200 steps, with orientation indices drawn over the whole table."""
    shape = (10, 18, 34)
    E6 = [-4e-4, -3e-4, 1e-3, 1e-4, -2e-4, 5e-5]
    g, o = make_pair(G, shape, Q, 1, bc=1, strain6=E6, n_mpm=0, n_seeds=40, seed=13)
    assert int(o.spins.max()) > 700
    rng = np.random.default_rng(6)
    u, v = _random_state(o, rng)
    g.set_nodal(u, v)
    o.u, o.v = u.copy(), v.copy()
    g.mpm_steps(200)
    o.mpm_steps(200)
    ug, vg = g.nodal()
    assert rel(ug, o.u) < 1e-4 and rel(vg, o.v) < 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_stress_parity_ragged_tiles(G, precision):
    shape = (6, 34, 66)  # 17 x 33 cells in y, x: partial 16x16 tiles
    g, o = make_pair(G, shape, 5, precision, axis=(1, 2, 3.0), n_mpm=0)
    rng = np.random.default_rng(9)
    u, v = _random_state(o, rng)
    g.set_nodal(u, v)
    o.u, o.v = u.copy(), v.copy()
    g.compute_stress()
    tol = 1e-13 if precision == 0 else 2e-6
    assert rel(g.stress(), o.stress()) < tol
    g.mpm_steps(3)
    o.mpm_steps(3)
    assert rel(g.nodal()[0], o.u) < (1e-12 if precision == 0 else 1e-5)


@pytest.mark.parametrize("precision,elastic", [(0, 1), (1, 1), (0, 3), (1, 3)])
def test_hybrid_lockstep_decisions(G, precision, elastic):
    """Both sides sweep the same spins with the same stress (the oracle's, pushed
    to the device); decisions may differ only where |dH - t| is within 1e-6.
    elastic 1: constant-traction point zone; 3: constant-strain point zone."""
    shape = (16, 34, 36)
    g, o = make_pair(G, shape, 16, precision, axis=(1, 1, 1.0), n_mpm=10, n_seeds=20, elastic=elastic)
    o.mpm_steps(10)
    sig = o.stress()
    n_site = n_mis = 0
    for m in range(3):
        for colour in (0, 1):
            g.set_spins(o.spins)
            g.set_stress(sig)
            pre = o.spins.copy()
            g.sweep_half(colour)
            _, changed, dH, t = o.half_sweep(colour)
            gs = g.spins()
            z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
            mask = ((x + y + z) & 1) == colour
            diff = (gs != o.spins) & mask
            n_site += int(mask.sum())
            n_mis += int(diff.sum())
            for p in np.flatnonzero(diff.ravel()):
                assert t.ravel()[p] >= 0 and abs(dH.ravel()[p] - t.ravel()[p]) <= 1e-6 * max(1.0, abs(t.ravel()[p]))
            assert (gs[~mask] == pre[~mask]).all()
        o.end_mcs()
        g.end_mcs()
    assert n_mis <= max(1, 1e-4 * n_site)


def test_mcs_fp64_end_to_end(G):
    shape = (12, 20, 36)
    g, o = make_pair(G, shape, 12, G.HMC_FP64, axis=(0.3, 0.5, 1.0), n_mpm=8, n_seeds=15)
    for m in range(3):
        a_g = g.mc_sweeps(1)
        a_o = o.mc_sweeps(1)
        assert a_g == a_o
        assert (g.spins() == o.spins).all()
        assert rel(g.nodal()[0], o.u) < 1e-11
        assert rel(g.strain(), o.Ebar) < 1e-12


def test_mcs_fp32_mismatch_is_small(G):
    shape = (16, 34, 36)
    g, o = make_pair(G, shape, 12, G.HMC_FP32, axis=(1, 1, 1.0), n_mpm=20, n_seeds=15)
    g.mc_sweeps(2)
    o.mc_sweeps(2)
    frac = float((g.spins() != o.spins).mean())
    assert frac < 0.01  # FP32 stress vs FP64; reported as the end-to-end mismatch fraction
    assert rel(g.nodal()[0], o.u) < 1e-3


def test_statistics(G):
    shape = (14, 22, 34)
    g, o = make_pair(G, shape, 20, G.HMC_FP32, axis=(1, 1, 1.0), n_mpm=2, n_seeds=25)
    g.mc_sweeps(2)
    sp = g.spins()
    unlike, W, mean = g.energy()
    assert unlike == O.unlike_bonds(sp)
    counts = O.orientation_counts(sp, 20)
    f, c = g.texture_histogram(G.HMC_HIST_PER_Q, 20)
    assert (c == counts).all() and c.sum() == sp.size
    assert np.allclose(f, counts / sp.size, rtol=0, atol=1e-15)
    for kind, nb in ((G.HMC_HIST_ANGLE_100, 9), (G.HMC_HIST_YOUNG, 12)):
        f, _ = g.texture_histogram(kind, nb)
        ref = O.texture_histogram(kind, nb, counts, o.A, o.St, (1, 1, 1.0), **C3)
        assert np.allclose(f, ref, rtol=0, atol=1e-15)


def test_checkpoint_resume_is_bit_identical(G):
    shape = (8, 18, 34)
    g, _ = make_pair(G, shape, 8, G.HMC_FP32, n_mpm=4)
    g.mc_sweeps(2)
    blob = g.state()
    g.mc_sweeps(3)
    a = g.spins().copy()
    u_a = g.nodal()[0]
    g.set_state(blob)
    g.mc_sweeps(3)
    assert (g.spins() == a).all()
    assert np.array_equal(g.nodal()[0], u_a)


@pytest.mark.parametrize("precision", [0, 1])
def test_homogeneous_block(G, precision):
    shape = (8, 8, 36)
    rng = np.random.default_rng(2)
    eul = rng.random((1, 3)) * 6
    n = np.array([0.2, -0.5, 0.8])
    g = G.HMC(shape, 1, precision=precision, load_axis=tuple(n), strain=1.3e-3, mpm_steps_per_mcs=5, **C3)
    g.set_orientations(eul, np.zeros(shape, dtype=np.uint16))
    g.mpm_steps(10)
    g.compute_stress()
    _, _, St = O.tables(eul, **C3)
    _, N, _ = O.axis_vectors(n)
    s = 1.3e-3 / (N @ St[0] @ N)
    tol = 1e-12 if precision == 0 else 1e-5
    assert np.abs(g.stress() - s * N[None, :]).max() < tol * abs(s)
    # FP32 rounding leaves a uniform net force: at most a rigid drift, far below strain x edge
    u = g.nodal()[0]
    assert np.abs(u - u.mean(axis=0)).max() < (1e-14 if precision == 0 else 1e-9)
    assert np.abs(u).max() < (1e-14 if precision == 0 else 1e-6 * 1.3e-3 * 36)


def test_errors_leave_handle_usable(G):
    g = G.HMC((4, 4, 4), 2)
    with pytest.raises(G.HMCError) as e:
        g.mc_sweeps(1)
    assert e.value.status == G.HMC_ERR_STATE
    with pytest.raises(G.HMCError):
        g.set_orientations(np.zeros((2, 3)), np.full(64, 5, dtype=np.uint16))
    g.set_orientations(np.zeros((2, 3)), np.zeros(64, dtype=np.uint16))
    g.mc_sweeps(1)


@pytest.mark.parametrize("precision", [0, 1])
def test_recomputed_stress_sweeps_are_bit_identical(G, precision):
    """store_stress = 0: the sweeps form each trial site's stress from the nodal
    displacement with the stress pass's arithmetic, so whole Monte Carlo steps give
    the same bits as with the stored field."""
    shape = (12, 18, 34)
    out = []
    for store in (1, 0):
        eul = S.euler_uniform_so3(12, 4)
        sp = S.voronoi_spins(shape, 15, 12, 4)
        g = G.HMC(shape, 12, precision=precision, load_axis=(1, 1, 1.0), strain=2e-3, mpm_steps_per_mcs=8,
                  elastic_scale=2e3, store_stress=store, seed=77, **C3)
        g.set_orientations(eul, sp)
        acc = g.mc_sweeps(3)
        out.append((acc, g.spins().copy(), g.nodal()[0], g.strain()))
        g.close()
    assert out[0][0] == out[1][0] and out[0][0] > 0
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2]) and np.array_equal(out[0][3], out[1][3])


def test_recomputed_strain_zone_matches_stored(G):
    """Constant-strain zone: the recomputed strain is the point strain itself, the
    stored form S'(q) sigma rounds through the stress; decisions agree but for
    trials within rounding of their threshold."""
    shape = (12, 18, 34)
    res = []
    for store in (1, 0):
        eul = S.euler_uniform_so3(12, 4)
        sp = S.voronoi_spins(shape, 15, 12, 4)
        g = G.HMC(shape, 12, precision=0, load_axis=(1, 1, 1.0), strain=2e-3, mpm_steps_per_mcs=8,
                  elastic=G.HMC_ELASTIC_STRAIN, elastic_scale=2e3, store_stress=store, seed=78, **C3)
        g.set_orientations(eul, sp)
        g.mc_sweeps(1)
        res.append(g.spins().copy())
        g.close()
    assert (res[0] != res[1]).mean() <= 1e-4


@pytest.mark.parametrize("elastic", [1, 3])
def test_sweep_margins_match_the_oracle(G, elastic):
    """hmc_sweep_half_margins (FP64): the same decisions as the plain half sweep, and for
    every trial evaluated with the elastic term its (H - t) / max(1, |t|) equals the
    oracle's to rounding; a trial is accepted exactly when that margin is <= 0."""
    shape = (10, 18, 34)
    g, o = make_pair(G, shape, 16, G.HMC_FP64, axis=(1, 1, 1.0), n_mpm=6, n_seeds=20, elastic=elastic)
    o.mpm_steps(6)
    sig = o.stress()
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    for colour in (0, 1):
        g.set_spins(o.spins)
        g.set_stress(sig)
        pre = o.spins.copy()
        acc, m = g.sweep_half_margins(colour)
        acc_o, changed, dH, t = o.half_sweep(colour)
        assert acc == acc_o and (g.spins() == o.spins).all()
        mask = ((x + y + z) & 1) == colour
        ev = ~np.isnan(m)
        assert ev.sum() > 0 and not (ev & ~mask).any()
        dH, t = dH.reshape(shape), t.reshape(shape)
        want = (dH - t) / np.maximum(1.0, np.abs(t))
        assert np.abs(m[ev] - want[ev]).max() < 1e-12
        moved = o.spins != pre
        assert (moved <= ev).all()                 # every change came from an evaluated trial
        assert ((m[ev] <= 0) == moved[ev]).all()   # accepted exactly when the margin is <= 0


def test_plain_fp64_step_matches_fused_and_oracle(G):
    """The plain unfused incremental FP64 step (the baseline form) advances u and v as the
    fused total-form step does, to FP64 rounding, on a ragged polycrystal; both match the
    oracle.  FP32 and batch handles are refused."""
    shape = (10, 18, 34)
    g, o = make_pair(G, shape, 9, G.HMC_FP64, axis=(0.4, 1.0, 0.7), n_mpm=0, n_seeds=14)
    rng = np.random.default_rng(4)
    u0 = rng.normal(size=(np.prod(shape) // 8, 3)) * 1e-3
    v0 = rng.normal(size=u0.shape) * 1e-4
    g.set_nodal(u0, v0)
    g.mpm_steps_plain(25)
    up, vp = g.nodal()
    g.set_nodal(u0, v0)
    g.mpm_steps(25)
    uf, vf = g.nodal()
    o.u, o.v = u0.copy(), v0.copy()
    o.mpm_steps(25)
    assert rel(up, uf) < 1e-12 and rel(vp, vf) < 1e-12
    assert rel(up, o.u) < 1e-12 and rel(vp, o.v) < 1e-12
    g32, _ = make_pair(G, shape, 9, G.HMC_FP32, n_mpm=0, n_seeds=14)
    with pytest.raises(G.HMCError) as e:
        g32.mpm_steps_plain(1)
    assert e.value.status == G.HMC_ERR_ARG
