"""Degenerate and boundary cases of the method against the FP64 oracle, through the C ABI:
the smallest grid (4^3: every block's neighbours wrap), zero temperature (only trials
that do not raise H are accepted), J = 0 (the elastic term alone decides), a single
orientation (no trial can change anything), trials over all orientations with a
two-orientation set, and the elastic scale at zero (the hybrid reduces to pure Potts)."""
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


def pair(G, shape, Q, *, J=1.0, kT=0.7, trial=0, lam=None, n_mpm=6, seed=3, axis=(1, 1, 1.0), strain=2e-3,
         elastic=1, n_seeds=6):
    eul = S.euler_uniform_so3(Q, seed)
    sp = S.voronoi_spins(shape, n_seeds, Q, seed) if Q > 1 else np.zeros(shape, dtype=np.uint16)
    lam = O.elastic_scale(max(shape)) if lam is None else lam
    kw = dict(J=J, kT=kT, load_axis=tuple(axis), strain=strain, elastic=elastic, trial=trial,
              mpm_steps_per_mcs=n_mpm, seed=seed * 131 + 7, **C3)
    g = G.HMC(shape, Q, precision=G.HMC_FP64, elastic_scale=lam, **kw)
    g.set_orientations(eul, sp)
    o = O.OracleHMC(shape, Q, elastic_scale_=lam, **kw)
    o.set_orientations(eul, sp.copy())
    return g, o


def run_both(g, o, n_mcs):
    for m in range(n_mcs):
        ag, ao = g.mc_sweeps(1), o.mc_sweeps(1)
        assert ag == ao, f"MCS {m}: accepted {ag} vs {ao}"
        assert (g.spins() == o.spins).all(), f"MCS {m}: spins differ"
        u = g.nodal()[0]
        # relative, with an absolute floor far below the load's displacement scale (strain x
        # edge ~ 1e-2) for the homogeneous cases, where u is rounding noise around zero
        assert np.linalg.norm(u - o.u) <= 1e-11 * np.linalg.norm(o.u) + 1e-14


def test_smallest_grid(G):
    g, o = pair(G, (4, 4, 4), 5, n_seeds=4)
    run_both(g, o, 4)


def test_zero_temperature(G):
    g, o = pair(G, (8, 10, 12), 6, kT=0.0)
    run_both(g, o, 3)


def test_no_bond_energy(G):
    g, o = pair(G, (8, 10, 12), 6, J=0.0, lam=5e3)
    run_both(g, o, 3)


def test_single_orientation_never_changes(G):
    g, o = pair(G, (6, 8, 10), 1, trial=1)
    before = g.spins().copy()
    assert g.mc_sweeps(3) == 0
    assert (g.spins() == before).all()
    run_both(g, o, 1)


def test_uniform_trials_two_orientations(G):
    g, o = pair(G, (6, 8, 14), 2, trial=1, n_seeds=5)
    run_both(g, o, 3)


def test_zero_elastic_scale_is_pure_potts(G):
    g, o = pair(G, (8, 8, 16), 6, lam=0.0)
    gp, _ = pair(G, (8, 8, 16), 6, elastic=0)
    for m in range(3):
        ag, ao, ap = g.mc_sweeps(1), o.mc_sweeps(1), gp.mc_sweeps(1)
        assert ag == ao == ap, f"MCS {m}"
        assert (g.spins() == o.spins).all() and (gp.spins() == g.spins()).all(), f"MCS {m}"


def test_empty_calls_and_refused_inputs_leave_the_state_alone(G):
    """Zero counts do nothing; negative counts, a bad colour and an orientation index >= Q are
    refused with HMC_ERR_ARG before anything is launched, and the handle then continues in
    lock-step with the oracle."""
    g, o = pair(G, (6, 8, 10), 5)
    run_both(g, o, 1)
    s0, (u0, v0), e0 = g.spins().copy(), g.nodal(), g.strain()
    mcs0 = g.info().mcs
    assert g.mc_sweeps(0) == 0
    g.mpm_steps(0)
    assert (g.spins() == s0).all() and g.info().mcs == mcs0
    u1, v1 = g.nodal()
    assert np.array_equal(u1, u0) and np.array_equal(v1, v0) and np.array_equal(g.strain(), e0)
    for call in (lambda: g.mc_sweeps(-1), lambda: g.mpm_steps(-2), lambda: g.sweep_half(2),
                 lambda: g.set_spins(np.where(np.arange(s0.size) == 17, 5, s0.ravel()).astype(np.uint16))):
        with pytest.raises(G.HMCError) as e:
            call()
        assert e.value.status == G.HMC_ERR_ARG
    assert (g.spins() == s0).all()
    run_both(g, o, 2)
