"""Failure detection through host-side fault injection (no GPU fault is produced)."""
import os

import numpy as np
import pytest


@pytest.fixture
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def _with_fault(value):
    class F:
        def __enter__(self):
            self.old = os.environ.get("HMC_FAULT")
            os.environ["HMC_FAULT"] = value

        def __exit__(self, *a):
            if self.old is None:
                os.environ.pop("HMC_FAULT", None)
            else:
                os.environ["HMC_FAULT"] = self.old
    return F()


def test_injected_allocation_failure_on_host(G):
    with _with_fault("alloc"):
        with pytest.raises(G.HMCError) as e:
            G.hmc_create(G.hmc_default_params())
    assert e.value.status == G.HMC_ERR_OOM
    assert "injected" in G.hmc_last_error(None)


@pytest.mark.gpu
def test_injected_launch_failure_leaves_handle_usable(G):
    g = G.HMC((8, 8, 8), 2, mpm_steps_per_mcs=2)
    g.set_orientations(np.zeros((2, 3)), np.zeros(512, dtype=np.uint16))
    with _with_fault("launch"):
        with pytest.raises(G.HMCError) as e:
            g.mc_sweeps(1)
        assert e.value.status == G.HMC_ERR_CUDA
        with pytest.raises(G.HMCError):
            g.mpm_steps(3)
    assert g.info().mcs == 0
    g.mc_sweeps(1)
    assert g.info().mcs == 1


@pytest.mark.gpu
def test_injected_nan_is_detected_and_cleared(G):
    g = G.HMC((8, 8, 8), 2, mpm_steps_per_mcs=2)
    g.set_orientations(np.zeros((2, 3)), np.zeros(512, dtype=np.uint16))
    with _with_fault("nan"):
        with pytest.raises(G.HMCError) as e:
            g.compute_stress()
    assert e.value.status == G.HMC_ERR_NONFINITE
    with pytest.raises(G.HMCError) as e:
        g.mc_sweeps(1)
    assert e.value.status == G.HMC_ERR_NONFINITE
    g.set_nodal(np.zeros((64, 3)), np.zeros((64, 3)))
    mean, W = g.compute_stress()
    assert np.isfinite(W) and np.isfinite(mean).all()


@pytest.mark.gpu
def test_injected_copy_wait_runs_out_and_is_reported(G):
    """HMC_FAULT=sweep_wait: the stored-stress sweep never starts its stress copy,
    so the CTA's bounded wait (1 s) runs out; the CTA changes nothing, the call
    reports HMC_ERR_TIMEOUT once, and the handle sweeps normally afterwards."""
    from hmc_synth import voronoi_spins, euler_uniform_so3
    g = G.HMC((8, 8, 8), 4, mpm_steps_per_mcs=2, elastic_scale=3e3)
    sp = voronoi_spins((8, 8, 8), 6, 4, 1)
    g.set_orientations(euler_uniform_so3(4, 1), sp)
    g.compute_stress()
    with _with_fault("sweep_wait"):
        with pytest.raises(G.HMCError) as e:
            g.sweep_half(0)
    assert e.value.status == G.HMC_ERR_TIMEOUT
    assert (g.spins() == sp).all()
    assert g.sweep_half(0) > 0


@pytest.mark.gpu
def test_injected_lost_copy_makes_the_handle_refuse_further_calls(G):
    """HMC_FAULT=copy_lost records, on the host, what a sweep CTA records when its stress
    copy never lands: the call reports HMC_ERR_TIMEOUT and every later call on the handle
    is refused with HMC_ERR_STATE (its shared memory can no longer be trusted); other
    handles are not affected and the handle can still be destroyed."""
    from hmc_synth import voronoi_spins, euler_uniform_so3
    g = G.HMC((8, 8, 8), 4, mpm_steps_per_mcs=2, elastic_scale=3e3)
    sp = voronoi_spins((8, 8, 8), 6, 4, 1)
    g.set_orientations(euler_uniform_so3(4, 1), sp)
    g.compute_stress()
    with _with_fault("copy_lost"):
        with pytest.raises(G.HMCError) as e:
            g.sweep_half(0)
    assert e.value.status == G.HMC_ERR_TIMEOUT
    for call in (lambda: g.sweep_half(1), lambda: g.mc_sweeps(1), lambda: g.mpm_steps(1)):
        with pytest.raises(G.HMCError) as e:
            call()
        assert e.value.status == G.HMC_ERR_STATE
    other = G.HMC((8, 8, 8), 4, mpm_steps_per_mcs=2)
    other.set_orientations(euler_uniform_so3(4, 1), sp)
    assert other.mc_sweeps(1) >= 0
    other.close()
    g.close()
