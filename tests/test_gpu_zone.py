"""Parity of the 27-point zone sweep (HMC_ELASTIC_ZONE1, Eq. 6 over a zone of
half-width one point) with the oracle's zone half sweep (dense least-squares
re-solve of the zone for every trial)."""
import numpy as np
import pytest

import hmc_synth as S
import oracle as O
import oracle.zone as Z

pytestmark = pytest.mark.gpu

C3 = dict(c11=246.5, c12=147.3, c44=124.7)
E6 = np.array([1e-3, -3e-4, -4e-4, 2e-4, -1e-4, 1e-4])


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def zone_handle(G, shape, Q, precision, seed, lam, *, n_seeds=6, kT=0.7, trial=0, bc=1, n_mpm=0, axis=(0, 0, 1.0)):
    eul = S.euler_uniform_so3(Q, seed)
    sp = S.voronoi_spins(shape, n_seeds, Q, seed + 1)
    g = G.HMC(shape, Q, precision=precision, J=1.0, kT=kT, bc=bc, strain6=tuple(E6), load_axis=axis, strain=2e-3,
              elastic=G.HMC_ELASTIC_ZONE1, trial=trial, mpm_steps_per_mcs=n_mpm, dt=O.default_dt(**C3),
              damping=0.05, elastic_scale=lam, seed=seed * 7919 + 3, **C3)
    g.set_orientations(eul, sp)
    return g, eul, sp


def _mask(shape, colour):
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    return ((x + y + z) & 1) == colour


@pytest.mark.parametrize("shape,precision,trial", [((6, 6, 8), 0, 0), ((8, 6, 10), 0, 1), ((6, 8, 6), 1, 0)])
def test_zone_half_sweeps_match_oracle(G, shape, precision, trial):
    """Both sides start every half step from the same spins and nodal state; a
    decision may differ only where |dH - t| is within the arithmetic's bound
    (FP64: 1e-9, FP32: 1e-4 relative to max(1, |t|))."""
    Q, seed, lam = 5, 3, 3.0e3
    g, eul, sp = zone_handle(G, shape, Q, precision, seed, lam, trial=trial)
    _, Ct, _ = O.tables(eul, **C3)
    Bs = Z.all_strain_matrices(shape)
    rng = np.random.default_rng(seed)
    nn = int(np.prod(shape)) // 8
    u0 = rng.normal(size=(nn, 3)) * 2e-4
    g.set_nodal(u0, np.zeros((nn, 3)))
    tol = 1e-9 if precision == 0 else 1e-4
    spo = sp.copy()
    n_site = n_mis = n_acc = 0
    for colour in (0, 1):
        g.set_spins(spo)
        pre = spo.copy()
        acc_g = g.sweep_half(colour)
        acc_o, changed, dH, t = Z.half_sweep_zone(spo, colour, seed * 7919 + 3, 0, 0, 1.0, 0.7, trial, Q, lam, Ct,
                                                  E6, u0.reshape(-1), 1, Bs)
        gs = g.spins()
        mask = _mask(shape, colour)
        assert (gs[~mask] == pre[~mask]).all()
        diff = (gs != spo).ravel()
        for p in np.flatnonzero(diff):
            assert t[p] >= 0 and abs(dH[p] - t[p]) <= tol * max(1.0, abs(t[p])), (p, dH[p], t[p])
        n_site += int(mask.sum())
        n_mis += int(diff.sum())
        n_acc += acc_o
        if not diff.any():
            assert acc_g == acc_o
    assert n_acc > 0
    if precision == 0:
        assert n_mis == 0
    else:
        assert n_mis <= max(1, 1e-3 * n_site)
    g.close()


def test_zone_mcs_fp64_matches_oracle(G):
    """Whole Monte Carlo steps (MPM steps, stress, both half sweeps with the zone,
    uniaxial control) through the captured graph against the oracle's schedule."""
    shape, Q, seed, lam = (6, 8, 10), 6, 5, 2.0e3
    g, eul, sp = zone_handle(G, shape, Q, 0, seed, lam, bc=0, n_mpm=6, axis=(0.3, 0.5, 1.0), n_seeds=8)
    o = O.OracleHMC(shape, Q, J=1.0, kT=0.7, bc=0, load_axis=(0.3, 0.5, 1.0), strain=2e-3, elastic_scale_=lam,
                    mpm_steps_per_mcs=6, dt=O.default_dt(**C3), damping=0.05, seed=seed * 7919 + 3, **C3)
    o.set_orientations(eul, sp)
    Bs = Z.all_strain_matrices(shape)
    total = 0
    for m in range(3):
        a_g = g.mc_sweeps(1)
        o.mpm_steps(o.n_mpm)
        o.stress()
        a_o = 0
        for colour in (0, 1):
            a_o += Z.half_sweep_zone(o.spins, colour, o.seed, o.mcs, 0, 1.0, 0.7, 0, Q, lam, o.Ct, o.Ebar,
                                     o.u.reshape(-1), 1, Bs)[0]
        o.end_mcs()
        assert a_g == a_o, m
        assert (g.spins() == o.spins).all(), m
        assert np.linalg.norm(g.nodal()[0] - o.u) < 1e-11 * np.linalg.norm(o.u)
        total += a_o
    assert total > 0
    g.close()


def test_zone_batch_replicas_equal_solo_runs(G):
    """Trials of all replicas share one list and one zone launch; each replica's
    spins equal its own single-replica run bit for bit."""
    shapes = [(6, 6, 8), (8, 10, 6)]
    Q, lam = 5, 3.0e3
    eul = S.euler_uniform_so3(Q, 9)
    fields = [S.voronoi_spins(s, 5, Q, 20 + i) for i, s in enumerate(shapes)]
    per = [dict(seed=101, strain6=tuple(E6)), dict(seed=202, strain6=tuple(-E6))]
    common = dict(J=1.0, kT=0.7, bc=1, elastic=G.HMC_ELASTIC_ZONE1, mpm_steps_per_mcs=4, elastic_scale=lam,
                  precision=G.HMC_FP32, **C3)
    b = G.HMCBatch(shapes, Q, per, **common)
    b.set_orientations(eul, fields)
    b.mc_sweeps(3)
    for r, s in enumerate(shapes):
        kw = dict(common)
        kw.update(per[r])
        g = G.HMC(s, Q, **kw)
        g.set_orientations(eul, fields[r])
        g.mc_sweeps(3)
        assert (b.spins(r) == g.spins()).all(), r
        assert np.array_equal(b.nodal(r)[0], g.nodal()[0])
        g.close()
    b.close()


def test_zone_needs_edges_of_six(G):
    with pytest.raises(G.HMCError) as e:
        G.HMC((4, 6, 6), 3, elastic=G.HMC_ELASTIC_ZONE1)
    assert e.value.status == G.HMC_ERR_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_zone_at_128_cubed_sampled(G, precision):
    """The 27-point zone sweep on the 128^3 workload (Q = 256, 5 000 grains, 2e-3 along
    [001]) in the launch configuration the bench times, against the oracle's zone solve on
    the zone's own nodes (zone_shift_local) for sampled sites of one half sweep from a
    synthetic displacement.  FP64: every sampled decision equal unless within 1e-9 of its
    threshold; FP32: within 1e-4."""
    spec, euler, spins = S.workload_inputs("ni128")
    shape, Q = spec["shape"], spec["Q"]
    nz, ny, nx = shape
    seed = 0x5EED1280
    g = G.HMC(shape, Q, precision=precision, J=spec["J"], kT=spec["kT"], load_axis=tuple(spec["axis"]),
              strain=spec["strain"], elastic=G.HMC_ELASTIC_ZONE1, mpm_steps_per_mcs=spec["mpm_steps"], seed=seed,
              **C3)
    g.set_orientations(euler, spins)
    A, Ct, St = O.tables(euler, C3["c11"], C3["c12"], C3["c44"])
    E = O.initial_uniaxial_strain(O.reuss_compliance(St, O.orientation_counts(spins, Q)), tuple(spec["axis"]),
                                  spec["strain"])
    assert np.abs(g.strain() - E).max() < 1e-12 * np.abs(E).max()
    nn = (nx // 2) * (ny // 2) * (nz // 2)
    rng = np.random.default_rng(41)
    u0 = rng.normal(size=(nn, 3)) * 2e-4
    g.set_nodal(u0, np.zeros((nn, 3)))
    u_o = u0.astype(np.float32).astype(np.float64) if precision == 1 else u0   # the device holds FP32
    g.sweep_half(0)
    after = g.spins()
    lam = O.elastic_scale(max(shape))
    tol = 1e-9 if precision == 0 else 1e-4
    n = zoned = mis = 0
    while zoned < 60:
        x, y, z = (int(v) for v in rng.integers(0, [nx, ny, nz]))
        if (x + y + z) & 1:
            x = (x + 1) % nx
        acc, qn, dH, t = Z.site_trial_zone_local(spins, x, y, z, seed, 0, 0, spec["J"], spec["kT"],
                                                 O.TRIAL_NEIGHBOR, Q, lam, Ct, E, u_o)
        q = int(spins[z, y, x])
        zoned += int(qn != q)
        n += 1
        want = qn if acc else q
        if after[z, y, x] != want:
            mis += 1
            assert t >= 0 and abs(dH - t) <= tol * max(1.0, abs(t)), (x, y, z, dH, t)
    assert mis <= (0 if precision == 0 else 2)
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_zone_trials_between_equal_stiffnesses(G, precision):
    """Orientations 0, 1 and 2, 3 are the same rotation twice, so a trial between them changes
    no stiffness: dC = 0, the border f = B_p^T dC e0 is zero, the elimination leaves exactly
    zero and the trial is decided on the bond energy alone (the pure Potts rule), as in the
    oracle's re-solve, which finds no energy change."""
    shape, Q, seed, lam = (6, 8, 8), 4, 11, 3.0e3
    eul = S.euler_uniform_so3(Q, seed)
    eul[1] = eul[0]
    eul[3] = eul[2]
    sp = S.voronoi_spins(shape, 6, Q, seed + 1)
    g = G.HMC(shape, Q, precision=precision, J=1.0, kT=0.7, bc=1, strain6=tuple(E6), load_axis=(0, 0, 1.0),
              strain=2e-3, elastic=G.HMC_ELASTIC_ZONE1, trial=1, mpm_steps_per_mcs=0, dt=O.default_dt(**C3),
              damping=0.05, elastic_scale=lam, seed=seed * 7919 + 3, **C3)
    g.set_orientations(eul, sp)
    _, Ct, _ = O.tables(eul, **C3)
    assert np.array_equal(Ct[0], Ct[1]) and np.array_equal(Ct[2], Ct[3])
    Bs = Z.all_strain_matrices(shape)
    rng = np.random.default_rng(seed)
    nn = int(np.prod(shape)) // 8
    u0 = rng.normal(size=(nn, 3)) * 2e-4
    g.set_nodal(u0, np.zeros((nn, 3)))
    tol = 1e-9 if precision == 0 else 1e-4
    spo = sp.copy()
    equal_flips = 0
    for colour in (0, 1):
        g.set_spins(spo)
        pre = spo.copy()
        g.sweep_half(colour)
        _, _, dH, t = Z.half_sweep_zone(spo, colour, seed * 7919 + 3, 0, 0, 1.0, 0.7, 1, Q, lam, Ct, E6,
                                        u0.reshape(-1), 1, Bs)
        gs = g.spins()
        moved = pre != spo
        equal_flips += int(np.sum(moved & ((pre // 2) == (spo // 2))))
        for p in np.flatnonzero((gs != spo).ravel()):
            assert abs(dH[p] - t[p]) <= tol * max(1.0, abs(t[p])), (p, dH[p], t[p])
        if precision == 0:
            assert (gs == spo).all()
    assert equal_flips > 0   # trials between equal stiffnesses were taken
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_zone_with_zero_elastic_scale_is_pure_potts(G, precision):
    """lambda = 0: every listed trial gets dH_e = 0 and the integer Metropolis threshold, so
    three MCS of the 27-point zone mode equal three MCS with the elastic term off, bit for bit
    (same draws, same decisions)."""
    shape, Q, seed = (8, 6, 10), 6, 13
    eul = S.euler_uniform_so3(Q, seed)
    sp = S.voronoi_spins(shape, 7, Q, seed + 1)
    out = []
    for elastic in (G.HMC_ELASTIC_ZONE1, G.HMC_ELASTIC_OFF):
        g = G.HMC(shape, Q, precision=precision, J=1.0, kT=0.7, elastic=elastic, elastic_scale=0.0,
                  mpm_steps_per_mcs=3, seed=seed * 31 + 1, **C3)
        g.set_orientations(eul, sp)
        acc = g.mc_sweeps(3)
        out.append((acc, g.spins().copy()))
        g.close()
    assert out[0][0] == out[1][0] and out[0][0] > 0
    assert np.array_equal(out[0][1], out[1][1])
