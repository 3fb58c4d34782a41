"""Adjoint of the explicit MPM stress solve against the FP64 oracle's
tangent-linear gradient (small grid), central finite differences of the FP64
forward map (the 128^3 workload: 5 000 Voronoi grains, Q = 256, 200 steps,
checkpoint every 20), and the torch.autograd wrapper."""
import numpy as np
import pytest

import hmc_synth as S
import oracle as O
import oracle.adjoint as AD

pytestmark = pytest.mark.gpu

C3 = (246.5, 147.3, 124.7)


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def _handle(G, shape, eul, sp, c, E, precision, u0=None):
    g = G.HMC(shape, eul.shape[0], c11=c[0], c12=c[1], c44=c[2], bc=G.HMC_BC_STRAIN6, strain6=tuple(E),
              mpm_steps_per_mcs=0, precision=precision)
    g.set_orientations(eul, sp)
    if u0 is not None:
        g.set_nodal(u0, None)
    return g


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-3)])
def test_adjoint_matches_oracle_tangent_linear(G, precision, tol):
    shape = (8, 12, 34)
    eul = S.euler_uniform_so3(6, 7)
    sp = S.voronoi_spins(shape, 9, 6, 8)
    E = np.array([1e-3, -3e-4, -4e-4, 2e-4, -1e-4, 1e-4])
    rng = np.random.default_rng(1)
    nn = int(np.prod(shape)) // 8
    u0 = rng.normal(size=(nn, 3)) * 1e-4
    g_field = rng.normal(size=int(np.prod(shape)))
    T, ck = 23, 5
    ref = AD.tangent_linear_gradient(sp, eul, C3, E, u0, np.zeros((nn, 3)), T, O.default_dt(*C3), O.DEFAULT_DAMPING,
                                     0.7, g_field)
    g = _handle(G, shape, eul, sp, C3, E, precision, u0)
    W, w = g.adjoint_forward(T, ck)
    grad = g.adjoint_backward(0.7, g_field)
    _, Ct, _ = O.tables(eul, *C3)
    uT, _ = AD.forward(sp, Ct, E, u0, np.zeros((nn, 3)), T, O.default_dt(*C3), O.DEFAULT_DAMPING)
    W_o, w_o = AD.outputs(sp, Ct, E, uT)
    assert abs(W - W_o) < max(tol, 1e-6 if precision else 0) * abs(W_o)
    assert np.linalg.norm(w - w_o) < max(tol, 1e-5 if precision else 0) * np.linalg.norm(w_o)
    scale = np.abs(ref).max()
    assert np.abs(grad[:3] - ref[:3]).max() < tol * max(np.abs(ref[:3]).max(), 1e-30) + 1e-14 * scale
    assert np.abs(grad[3:] - ref[3:]).max() < tol * np.abs(ref[3:]).max()
    # a second backward with another cotangent reuses the checkpoints
    grad_w = g.adjoint_backward(1.0, None)
    ref_w = AD.tangent_linear_gradient(sp, eul, C3, E, u0, np.zeros((nn, 3)), T, O.default_dt(*C3),
                                       O.DEFAULT_DAMPING, 1.0, None)
    assert np.abs(grad_w - ref_w).max() < tol * np.abs(ref_w).max()
    # anything that moves the state invalidates the reverse sweep
    g.mpm_steps(1)
    with pytest.raises(G.HMCError) as e:
        g.adjoint_backward(1.0, None)
    assert e.value.status == G.HMC_ERR_STATE
    g.close()


def test_adjoint_workload_against_central_differences(G):
    """128^3, 5 000 grains, Q = 256, Ebar = the initial mixed-control strain for
    2e-3 along [001]; FP32 adjoint (200 steps, checkpoint every 20) against
    central differences (h = 1e-4 relative) of the FP64 forward map."""
    spec, euler, spins = S.workload_inputs("ni128")
    shape = spec["shape"]
    _, _, St = O.tables(euler, *C3)
    E = O.initial_uniaxial_strain(O.reuss_compliance(St, O.orientation_counts(spins, spec["Q"])), (0, 0, 1), 2e-3)
    rng = np.random.default_rng(5)
    g_field = rng.random(int(np.prod(shape)))
    T, ck, gW = 200, 20, 0.5

    g32 = _handle(G, shape, euler, spins, C3, E, 1)
    g32.adjoint_forward(T, ck, want_field=False)
    grad32 = g32.adjoint_backward(gW, g_field)
    g32.close()
    g64 = _handle(G, shape, euler, spins, C3, E, 0)
    g64.adjoint_forward(T, ck, want_field=False)
    grad64 = g64.adjoint_backward(gW, g_field)
    g64.close()

    def L(c, Eb):
        h = _handle(G, shape, euler, spins, c, Eb, 0)
        W, w = h.adjoint_forward(T, ck)
        h.close()
        return gW * W + g_field @ w

    fd = np.zeros(9)
    for k in range(9):
        step = 1e-4 * (C3[k] if k < 3 else abs(E[k - 3]) if abs(E[k - 3]) > 1e-6 else 1e-3 * 2e-3)
        cp, cm, Ep, Em = list(C3), list(C3), E.copy(), E.copy()
        if k < 3:
            cp[k] += step
            cm[k] -= step
        else:
            Ep[k - 3] += step
            Em[k - 3] -= step
        fd[k] = (L(cp, Ep) - L(cm, Em)) / (2 * step)
    scale = np.abs(fd).max()
    assert np.abs(grad64 - fd).max() < 1e-6 * scale
    assert np.abs(grad32 - fd).max() < 2e-3 * scale


def test_autograd_function(G):
    torch = pytest.importorskip("torch")
    from paper_1009_0457_gb300.autograd import HMCElastic
    shape = (6, 8, 10)
    eul = S.euler_uniform_so3(4, 3)
    sp = S.voronoi_spins(shape, 5, 4, 2)
    theta = torch.tensor([*C3, 1e-3, -3e-4, -4e-4, 2e-4, 0.0, 1e-4], dtype=torch.float64, requires_grad=True)
    W, w = HMCElastic.apply(theta, sp, eul, 12, 5, 0)
    loss = 0.3 * W + (w * torch.linspace(0, 1, w.numel(), dtype=torch.float64)).sum()
    loss.backward()
    nn = int(np.prod(shape)) // 8
    ref = AD.tangent_linear_gradient(sp, eul, C3, theta.detach().numpy()[3:], np.zeros((nn, 3)), np.zeros((nn, 3)),
                                     12, O.default_dt(*C3), O.DEFAULT_DAMPING, 0.3, np.linspace(0, 1, w.numel()))
    assert np.abs(theta.grad.numpy() - ref).max() < 1e-9 * np.abs(ref).max()
