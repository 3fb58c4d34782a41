"""Device-pointer spin exchange (zero-copy with tensors) through the C ABI."""
import numpy as np
import pytest

import hmc_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def test_device_pointer_spins(G):
    torch = pytest.importorskip("torch")
    shape, Q = (8, 10, 12), 5
    sp = S.voronoi_spins(shape, 6, Q, 3)
    eul = S.euler_uniform_so3(Q, 2)
    g = G.HMC(shape, Q, elastic=0, mpm_steps_per_mcs=0)
    d = torch.from_numpy(sp.reshape(-1).view(np.int16).copy()).cuda()
    G.hmc_set_orientations_dev(g.h, eul, d.data_ptr())
    assert (g.spins() == sp).all()
    g.mc_sweeps(2)
    out = torch.zeros(sp.size, dtype=torch.int16, device="cuda")
    G.hmc_get_spins_dev(g.h, out.data_ptr())
    assert (out.cpu().numpy().view(np.uint16).reshape(shape) == g.spins()).all()
    sp2 = S.random_spins(shape, Q, 4)
    d2 = torch.from_numpy(sp2.reshape(-1).view(np.int16).copy()).cuda()
    G.hmc_set_spins_dev(g.h, d2.data_ptr())
    assert (g.spins() == sp2).all()
    # rejected before anything is launched or changed
    bad = sp.copy()
    bad[1, 2, 3] = Q
    d3 = torch.from_numpy(bad.reshape(-1).view(np.int16).copy()).cuda()
    with pytest.raises(G.HMCError) as e:
        G.hmc_set_spins_dev(g.h, d3.data_ptr())
    assert e.value.status == G.HMC_ERR_ARG
    assert (g.spins() == sp2).all()
    for ptr in (d2.data_ptr() + 2, sp2.ctypes.data, 0):
        with pytest.raises(G.HMCError) as e:
            G.hmc_set_spins_dev(g.h, ptr)
        assert e.value.status == G.HMC_ERR_ARG
    assert (g.spins() == sp2).all()
    g.close()
