"""hmc_stress_noalloc: the allocation-free stress pass.

Callers that cannot allocate device memory where they need the stress (code
running inside another framework's memory pool or a fixed-budget arena, or
code that must not call cudaMalloc/cudaFree because those calls synchronise
the device) use this entry point on their own device buffers.  Its scratch is a
fixed static device array shared by every call, so this test runs it twice in a
row on two different states and checks each result against the handle's own
stress pass (hmc_compute_stress + hmc_get_stress) on the same state.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C3 = dict(c11=246.5, c12=147.3, c44=124.7)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_noalloc_stress_matches_handle_on_two_calls():
    from conftest import build_libhmc
    build_libhmc()
    torch = pytest.importorskip("torch")
    import hmc_synth as S
    import oracle as O
    import paper_1009_0457_gb300 as G

    shape, Q = (20, 34, 66), 12
    nz, ny, nx = shape
    eul = S.euler_uniform_so3(Q, 3)
    spins = S.voronoi_spins(shape, 25, Q, 3)
    g = G.HMC(shape, Q, precision=G.HMC_FP32, load_axis=(1, 1, 1.0), strain=2e-3, mpm_steps_per_mcs=4, **C3)
    g.set_orientations(eul, spins)
    _, Ct, _ = O.tables(eul, **C3)  # FP64 stiffness table of the inputs, rounded to FP32 for the device
    dev = torch.device("cuda", 0)
    N = spins.size
    d_spins = torch.from_numpy(spins.reshape(-1).view(np.int16).copy()).to(dev)
    d_ctab = torch.from_numpy(Ct.reshape(-1).astype(np.float32)).to(dev)
    d_sigma = torch.empty(N * 6, dtype=torch.float32, device=dev)
    d_mean = torch.empty(6, dtype=torch.float64, device=dev)
    d_energy = torch.empty(1, dtype=torch.float64, device=dev)
    for call in range(2):
        g.mpm_steps(5)  # a different displacement state for each call
        mean_ref, W_ref = g.compute_stress()
        sig_ref = g.stress()
        u, _ = g.nodal()
        d_u = torch.from_numpy(u.reshape(-1).astype(np.float32)).to(dev)
        E = g.strain()
        d_sigma.fill_(float("nan"))
        d_mean.fill_(float("nan"))
        d_energy.fill_(float("nan"))
        torch.cuda.synchronize()
        G.hmc_stress_noalloc(d_spins.data_ptr(), d_u.data_ptr(), d_ctab.data_ptr(), E, nx, ny, nz,
                             d_sigma.data_ptr(), d_mean.data_ptr(), d_energy.data_ptr(), None)
        torch.cuda.synchronize()
        sig = d_sigma.cpu().numpy().astype(np.float64).reshape(N, 6)
        assert rel(sig, sig_ref) < 2e-6, f"call {call}"
        assert rel(d_mean.cpu().numpy(), mean_ref) < 2e-6, f"call {call}"
        assert abs(d_energy.item() - W_ref) < 2e-6 * abs(W_ref), f"call {call}"

    # sizes beyond the fixed scratch array are refused before any launch
    with pytest.raises(G.HMCError) as e:
        G.hmc_stress_noalloc(d_spins.data_ptr(), d_u.data_ptr(), d_ctab.data_ptr(), E, 258, 258, 258,
                             d_sigma.data_ptr(), d_mean.data_ptr(), d_energy.data_ptr(), None)
    assert e.value.status == G.HMC_ERR_ARG
    assert "limit" in G.hmc_last_error(None)
    g.close()


def test_noalloc_stress_at_its_largest_grid():
    """256^3 points fill every one of the 8 192 partial-sum slots of the fixed scratch
    array: the call is accepted and equals the handle's stress pass on the same state."""
    from conftest import build_libhmc
    build_libhmc()
    torch = pytest.importorskip("torch")
    import hmc_synth as S
    import oracle as O
    import paper_1009_0457_gb300 as G

    shape, Q = (256, 256, 256), 12
    nz, ny, nx = shape
    eul = S.euler_uniform_so3(Q, 5)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    spins = ((x // 12 + 3 * (y // 20) + 5 * (z // 28)) % Q).astype(np.uint16)
    g = G.HMC(shape, Q, precision=G.HMC_FP32, load_axis=(0.3, 0.4, 1.0), strain=2e-3, mpm_steps_per_mcs=0, **C3)
    g.set_orientations(eul, spins)
    rng = np.random.default_rng(8)
    nn = (nx // 2) * (ny // 2) * (nz // 2)
    u = (rng.standard_normal((nn, 3)) * 1e-3).astype(np.float32).astype(np.float64)
    g.set_nodal(u, np.zeros_like(u))
    mean_ref, W_ref = g.compute_stress()
    sig_ref = g.stress()
    E = g.strain()
    _, Ct, _ = O.tables(eul, **C3)
    dev = torch.device("cuda", 0)
    N = spins.size
    d_spins = torch.from_numpy(spins.reshape(-1).view(np.int16).copy()).to(dev)
    d_ctab = torch.from_numpy(Ct.reshape(-1).astype(np.float32)).to(dev)
    d_u = torch.from_numpy(u.reshape(-1).astype(np.float32)).to(dev)
    d_sigma = torch.full((N * 6,), float("nan"), dtype=torch.float32, device=dev)
    d_mean = torch.full((6,), float("nan"), dtype=torch.float64, device=dev)
    d_energy = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    G.hmc_stress_noalloc(d_spins.data_ptr(), d_u.data_ptr(), d_ctab.data_ptr(), E, nx, ny, nz,
                         d_sigma.data_ptr(), d_mean.data_ptr(), d_energy.data_ptr(), None)
    torch.cuda.synchronize()
    sig = d_sigma.cpu().numpy().astype(np.float64).reshape(N, 6)
    assert rel(sig, sig_ref) < 2e-6
    assert rel(d_mean.cpu().numpy(), mean_ref) < 2e-6
    assert abs(d_energy.item() - W_ref) < 2e-6 * abs(W_ref)
    g.close()
