"""Oracle pins of the stress-controlled (traction) loading and the load ramp."""
import numpy as np

import hmc_synth as S
import oracle as O

C3 = dict(c11=246.5, c12=147.3, c44=124.7)


def test_traction_single_crystal_closed_form():
    """One orientation and no displacement: the Reuss strain of the prescribed
    stress is the exact strain, so the mean stress equals s0 n(x)n at once."""
    shape = (4, 6, 8)
    eul = np.array([[0.3, 0.7, 1.1]])
    o = O.OracleHMC(shape, 1, bc=O.BC_TRACTION, load_axis=(1.0, 0.2, 0.1), stress=0.03, mpm_steps_per_mcs=0, **C3)
    o.set_orientations(eul, np.zeros(shape, dtype=np.uint16))
    o.stress()
    _, N, _ = O.axis_vectors((1.0, 0.2, 0.1))
    assert np.allclose(o.mean_sig, 0.03 * N, rtol=0, atol=1e-14)
    o.end_mcs()   # at the target: no change
    assert np.allclose(O.update_traction_strain(o.Ebar, o.mean_sig, o.S_R, o.axis, 0.03), o.Ebar, rtol=0,
                       atol=1e-18)


def test_traction_control_drives_the_mean_stress_to_the_target():
    """With the spins held fixed the control contracts the mean-stress gap
    geometrically; with the Monte Carlo steps running, the gap left after each
    step is set by that step's flips and stays a small fraction of s0."""
    shape = (8, 8, 8)
    Q = 6
    eul = S.euler_uniform_so3(Q, 3)
    sp = S.voronoi_spins(shape, 8, Q, 4)
    _, N, _ = O.axis_vectors((1.0, 0, 0))
    for sweeps in (False, True):
        o = O.OracleHMC(shape, Q, bc=O.BC_TRACTION, load_axis=(1.0, 0, 0), stress=0.05, elastic=O.ELASTIC_OFF,
                        mpm_steps_per_mcs=60, kT=0.0, **C3)
        o.set_orientations(eul, sp)
        gaps = []
        for m in range(8):
            if sweeps:
                o.mc_sweeps(1)
            else:
                o.mpm_steps(60)
                o.stress()
                o.end_mcs()
            gaps.append(np.abs(o.mean_sig - 0.05 * N).max())
        if sweeps:
            assert gaps[-1] < 0.1 * gaps[0] and gaps[-1] < 5e-3 * 0.05
        else:
            assert (o.spins == sp).all()
            assert gaps[-1] < 1e-6 * 0.05 and all(b < 0.5 * a for a, b in zip(gaps, gaps[1:]))


def test_set_load_moves_the_mean_strain_by_the_reuss_response():
    shape = (6, 6, 6)
    Q = 4
    eul = S.euler_uniform_so3(Q, 5)
    sp = S.random_spins(shape, Q, 6)
    axis = (0.2, 0.5, 1.0)
    _, N, _ = O.axis_vectors(axis)
    u = O.OracleHMC(shape, Q, bc=O.BC_UNIAXIAL, load_axis=axis, strain=1e-3, **C3)
    u.set_orientations(eul, sp)
    E0 = u.Ebar.copy()
    u.set_load(2.5e-3)
    assert abs(N @ u.Ebar - 2.5e-3) < 1e-18
    assert np.allclose(u.Ebar - E0, 1.5e-3 / (N @ (u.S_R @ N)) * (u.S_R @ N), rtol=1e-12, atol=0)
    t = O.OracleHMC(shape, Q, bc=O.BC_TRACTION, load_axis=axis, stress=0.01, **C3)
    t.set_orientations(eul, sp)
    E0 = t.Ebar.copy()
    t.set_load(0.04)
    assert np.allclose(t.Ebar - E0, t.S_R @ (0.03 * N), rtol=1e-12, atol=0)
    assert np.allclose(t.Ebar, O.initial_traction_strain(t.S_R, axis, 0.04), rtol=1e-12, atol=0)
