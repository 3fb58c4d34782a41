"""Stress-controlled (traction) loading and load ramps on the GPU path against the
oracle, and the texture response of Sec. "Results" (91 orientations rotated
about z, uniaxial tension along x: the soft orientations near 0 and 90 degrees
grow at the expense of the stiff ones near 45 degrees)."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("bc,load,ramp", [(2, 0.02, 0.01), (0, 1e-3, 5e-4)])
def test_loading_ramp_fp64_matches_oracle(G, bc, load, ramp):
    shape, Q, seed, lam = (12, 10, 18), 10, 7, 3.0e3
    eul = S.euler_uniform_so3(Q, seed)
    sp = S.voronoi_spins(shape, 12, Q, seed)
    axis = (1.0, 0.3, 0.2)
    kw = dict(J=1.0, kT=0.7, bc=bc, load_axis=axis, elastic=1, mpm_steps_per_mcs=8, dt=O.default_dt(**C3),
              damping=0.05, elastic_scale=lam, seed=seed * 7919 + 3)
    g = G.HMC(shape, Q, precision=G.HMC_FP64, strain=load, stress=load, **kw, **C3)
    g.set_orientations(eul, sp)
    o = O.OracleHMC(shape, Q, J=1.0, kT=0.7, bc=bc, load_axis=axis, strain=load, stress=load, elastic_scale_=lam,
                    mpm_steps_per_mcs=8, dt=O.default_dt(**C3), damping=0.05, seed=seed * 7919 + 3, **C3)
    o.set_orientations(eul, sp)
    assert rel(g.strain(), o.Ebar) < 1e-14
    for m in range(4):
        g.set_load(load + m * ramp)
        o.set_load(load + m * ramp)
        assert rel(g.strain(), o.Ebar) < 1e-12
        a_g = g.mc_sweeps(1)
        a_o = o.mc_sweeps(1)
        assert a_g == a_o
        assert (g.spins() == o.spins).all()
        assert rel(g.strain(), o.Ebar) < 1e-11
        assert rel(g.nodal()[0], o.u) < 1e-11
    g.close()


def test_set_load_rejected_for_strain6(G):
    g = G.HMC((4, 4, 4), 2, bc=G.HMC_BC_STRAIN6)
    g.set_orientations(S.euler_uniform_so3(2, 1), np.zeros((4, 4, 4), dtype=np.uint16))
    with pytest.raises(G.HMCError) as e:
        g.set_load(1e-3)
    assert e.value.status == G.HMC_ERR_ARG
    g.close()


def _texture_run(G, lam, stress):
    """1M sites (100^3), 91 orientations rotated about z by 0..90 degrees, random
    start coarsened 100 MCS at kT/J = 2.6 (pure Potts), then 75 loading substeps
    up to `stress` GPa along x, each one MCS with 50 MPM steps."""
    shape, Q = (100, 100, 100), 91
    eul = S.euler_z_rotations(Q)
    sp = S.random_spins(shape, Q, 8)
    g = G.HMC(shape, Q, precision=G.HMC_FP32, J=1.0, kT=2.6, bc=G.HMC_BC_TRACTION, load_axis=(1.0, 0, 0),
              stress=0.0, elastic=0, mpm_steps_per_mcs=0, seed=91, **C3)
    g.set_orientations(eul, sp)
    g.mc_sweeps(100)
    coarse = g.spins().copy()
    h = G.HMC(shape, Q, precision=G.HMC_FP32, J=1.0, kT=1.0, bc=G.HMC_BC_TRACTION, load_axis=(1.0, 0, 0),
              stress=0.0, elastic=1, elastic_scale=lam, mpm_steps_per_mcs=50, seed=92, **C3)
    h.set_orientations(eul, coarse)
    for k in range(1, 76):
        h.set_load(stress * k / 75)
        h.mc_sweeps(1)
    _, counts = h.texture_histogram(G.HMC_HIST_PER_Q, Q)
    f0 = np.bincount(coarse.ravel(), minlength=Q) / coarse.size
    f1 = counts / counts.sum()
    g.close()
    h.close()
    return f0, f1


def test_texture_softer_orientations_grow(G):
    ang = np.arange(91)
    soft = (ang <= 15) | (ang >= 75)
    stiff = (ang >= 30) & (ang <= 60)
    lam = 3.7e5   # the driving force at 30 MPa is then about J / 2 between 0 and 45 degrees
    f0, f_load = _texture_run(G, lam, 0.03)
    _, f_ctrl = _texture_run(G, lam, 0.0)
    d_soft = f_load[soft].sum() - f_ctrl[soft].sum()
    d_stiff = f_load[stiff].sum() - f_ctrl[stiff].sum()
    print("soft", f0[soft].sum(), f_ctrl[soft].sum(), f_load[soft].sum(), "stiff", f0[stiff].sum(),
          f_ctrl[stiff].sum(), f_load[stiff].sum())
    assert d_soft > 0.01 and d_stiff < -0.01
