"""Full-size parity on the 256^3 bench workload (Q = 1024, 40 000 Voronoi grains,
2e-3 along [111], FP32), in the launch configuration bench.py times, on sampled
outputs the oracle computes one by one.  Every oracle input comes from the
synthetic generators, never from the CUDA path."""
import numpy as np
import pytest

import hmc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    spec, euler, spins = S.workload_inputs("ni256")
    nz, ny, nx = spec["shape"]
    nn = (nx // 2) * (ny // 2) * (nz // 2)
    rng = np.random.default_rng(77)
    u0 = rng.normal(size=(nn, 3)) * 1e-3   # a synthetic displacement state
    v0 = rng.normal(size=(nn, 3)) * 1e-4
    kw = dict(J=spec["J"], kT=spec["kT"], c11=spec["c11"], c12=spec["c12"], c44=spec["c44"],
              load_axis=spec["axis"], strain=spec["strain"], mpm_steps_per_mcs=spec["mpm_steps"], seed=99)
    g = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP32, **kw)
    g.set_orientations(euler, spins)
    A, Ct, St = O.tables(euler, spec["c11"], spec["c12"], spec["c44"])
    S_R = O.reuss_compliance(St, O.orientation_counts(spins, spec["Q"]))
    E = O.initial_uniaxial_strain(S_R, spec["axis"], spec["strain"])
    yield dict(G=G, g=g, spec=spec, spins=spins, u0=u0, v0=v0, Ct=Ct, St=St, E=E, rng=rng)
    g.close()


def _sample_nodes(rng, nbx, nby, nbz, n=400):
    pts = [rng.integers(0, [nbx, nby, nbz]) for _ in range(n)]
    # tile edges (15-node patches), chunk edges and the periodic wrap
    for i in (0, 14, 15, 29, 30, nbx - 1):
        for k in (0, 1, nbz // 2, nbz - 1):
            pts.append(np.array([i, (7 * i + 3) % nby, k]))
            pts.append(np.array([(5 * i + 1) % nbx, i % nby, k]))
    return pts


def test_fullsize_strain_bar_matches(big):
    Eg = big["g"].strain()
    assert np.abs(Eg - big["E"]).max() < 1e-12 * np.abs(big["E"]).max()


def test_fullsize_mpm_step_sampled(big):
    g, spins = big["g"], big["spins"]
    nz, ny, nx = spins.shape
    g.set_nodal(big["u0"], big["v0"])
    g.mpm_steps(1)
    ug, vg = g.nodal()
    dt, zeta = O.default_dt(246.5, 147.3, 124.7), O.DEFAULT_DAMPING
    u0 = big["u0"].astype(np.float32).astype(np.float64)  # the device holds the state in FP32
    v0 = big["v0"].astype(np.float32).astype(np.float64)
    du, ref_u, dv, ref_v = [], [], [], []
    for (i, j, k) in _sample_nodes(big["rng"], nx // 2, ny // 2, nz // 2):
        I = i + (nx // 2) * (j + (ny // 2) * k)
        f = O.node_force(spins, big["Ct"], u0, big["E"], i, j, k)
        v = (1 - zeta) * v0[I] + dt * f / 8.0
        u = u0[I] + dt * v
        du.append(ug[I] - u)
        ref_u.append(u - u0[I])
        dv.append(vg[I] - v)
        ref_v.append(v)
    du, dv = np.array(du), np.array(dv)
    assert np.linalg.norm(dv) < 1e-5 * np.linalg.norm(ref_v)
    assert np.linalg.norm(du) < 1e-5 * np.linalg.norm(ref_u) + 1e-9


def test_fullsize_stress_sampled_and_reduced(big):
    g, spins = big["g"], big["spins"]
    g.set_nodal(big["u0"], big["v0"])
    mean_g, W_g = g.compute_stress()
    sig_g = g.stress()
    u0 = big["u0"].astype(np.float32).astype(np.float64)
    nz, ny, nx = spins.shape
    rng = big["rng"]
    d, r = [], []
    for _ in range(3000):
        x, y, z = (int(v) for v in rng.integers(0, [nx, ny, nz]))
        s = O.point_stress(spins, big["Ct"], u0, big["E"], x, y, z)
        d.append(sig_g[x + nx * (y + ny * z)] - s)
        r.append(s)
    assert np.linalg.norm(np.array(d)) < 2e-6 * np.linalg.norm(np.array(r))
    # the FP64 domain reductions against the oracle's whole-field pass
    _, mean_o, W_o = O.stress_field(spins, big["Ct"], u0, big["E"])
    assert np.linalg.norm(mean_g - mean_o) < 1e-6 * np.linalg.norm(mean_o)
    assert abs(W_g - W_o) < 1e-6 * abs(W_o)


@pytest.mark.parametrize("colour", [0, 1])
def test_fullsize_half_sweep_sampled(big, colour):
    """The device sweeps with its own FP32 stress; the oracle decides sampled
    sites with its own FP64 stress.  A decision may differ only where
    |dH - t| is within the FP32 stress margin 1e-4 max(1, |t|)."""
    G, g, spins = big["G"], big["g"], big["spins"]
    nz, ny, nx = spins.shape
    g.set_spins(spins)
    g.set_nodal(big["u0"], big["v0"])
    g.compute_stress()
    mcs = 0  # no Monte Carlo step has completed on this handle yet
    assert g.info().mcs == mcs
    g.sweep_half(colour)
    after = g.spins()
    u0 = big["u0"].astype(np.float32).astype(np.float64)
    lam = O.elastic_scale(256)
    rng = big["rng"]
    n = mis = 0
    for _ in range(20000):
        x, y, z = (int(v) for v in rng.integers(0, [nx, ny, nz]))
        if (x + y + z) & 1 != colour:
            x = (x + 1) % nx
        sig = O.point_stress(spins, big["Ct"], u0, big["E"], x, y, z)
        acc, qn, dH, t = O.site_trial_at(spins, x, y, z, 99, mcs, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 1024, 1, lam,
                                         big["St"], sig)
        want = qn if acc else spins[z, y, x]
        n += 1
        if after[z, y, x] != want:
            mis += 1
            assert t >= 0 and abs(dH - t) <= 1e-4 * max(1.0, abs(t))
    assert mis <= max(2, 1e-3 * n)
    # sites of the other colour are untouched
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    other = ((x + y + z) & 1) != colour
    assert (after[other] == spins[other]).all()


def test_fullsize_graph_mcs_conserves_volume(big):
    G, g, spins = big["G"], big["g"], big["spins"]
    g.set_spins(spins)
    acc = g.mc_sweeps(2)
    after = g.spins()
    f, counts = g.texture_histogram(G.HMC_HIST_ANGLE_100, 9)
    assert counts.sum() == spins.size and abs(f.sum() - 1) < 1e-12
    assert (counts == np.bincount(after.ravel(), minlength=1024)).all()
    assert 0 < int((after != spins).sum()) <= acc


def test_configured_500_mcs_run(big):
    """The 256^3 workload run as configured: 500 Monte Carlo steps (50 MPM steps each, FP32
    stress, FP64 reductions) with the ANGLE_100 histogram logged every 10 steps.  Every log
    sums to one over all sites, the volumes recounted from the spins every 100 steps equal the
    library's, every step accepts trials, and the mean strain and energy stay finite."""
    G, spec, spins = big["G"], big["spec"], big["spins"]
    kw = dict(J=spec["J"], kT=spec["kT"], c11=spec["c11"], c12=spec["c12"], c44=spec["c44"],
              load_axis=spec["axis"], strain=spec["strain"], mpm_steps_per_mcs=spec["mpm_steps"], seed=3)
    g = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP32, **kw)
    try:
        g.set_orientations(spins=spins, euler=S.workload_inputs("ni256")[1])
        first = None
        for m in range(50):
            acc = g.mc_sweeps(10)
            assert acc > 0, m
            f, counts = g.texture_histogram(G.HMC_HIST_ANGLE_100, 9)
            assert counts.sum() == spins.size and abs(f.sum() - 1) < 1e-12, m
            first = f.copy() if first is None else first
            if m % 10 == 9:
                assert (counts == np.bincount(g.spins().ravel(), minlength=spec["Q"])).all(), m
        unlike, w, sig = g.energy()
        assert np.all(np.isfinite(g.strain())) and np.isfinite(w) and np.all(np.isfinite(sig)) and unlike > 0
        assert g.info().mcs == 500
        assert np.abs(f - first).sum() > 0   # the texture evolves
    finally:
        g.close()
