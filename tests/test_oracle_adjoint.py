"""Oracle pins for the tangent-linear gradient of the explicit MPM solve (CPU only)."""
import numpy as np

import hmc_synth as S
import oracle as O
import oracle.adjoint as AD

C3 = (246.5, 147.3, 124.7)


def test_tangent_linear_matches_central_differences():
    shape = (6, 8, 10)
    eul = S.euler_uniform_so3(4, 3)
    sp = S.voronoi_spins(shape, 5, 4, 2)
    E = np.array([1e-3, -3e-4, -4e-4, 2e-4, 0, 1e-4])
    nn = int(np.prod(shape)) // 8
    rng = np.random.default_rng(0)
    u0, v0 = rng.normal(size=(nn, 3)) * 1e-4, np.zeros((nn, 3))
    dt, T = O.default_dt(*C3), 15
    g = rng.normal(size=int(np.prod(shape)))
    grad = AD.tangent_linear_gradient(sp, eul, C3, E, u0, v0, T, dt, 0.05, 0.7, g)

    def L(c, Eb):
        _, Ct, _ = O.tables(eul, *c)
        u, _ = AD.forward(sp, Ct, Eb, u0, v0, T, dt, 0.05)
        W, w = AD.outputs(sp, Ct, Eb, u)
        return 0.7 * W + g @ w

    for k in range(9):
        h = 1e-4 * (C3[k] if k < 3 else 1e-3)
        cp, cm, Ep, Em = list(C3), list(C3), E.copy(), E.copy()
        if k < 3:
            cp[k] += h
            cm[k] -= h
        else:
            Ep[k - 3] += h
            Em[k - 3] -= h
        fd = (L(cp, Ep) - L(cm, Em)) / (2 * h)
        assert abs(grad[k] - fd) < 1e-7 * abs(fd), k


def test_homogeneous_gradient_closed_form():
    """One orientation, no displacement: W = N/2 E.C'.E, dW/dC_i = N/2 E.R_i.E, dW/dE = N C'E."""
    shape = (4, 6, 8)
    N = int(np.prod(shape))
    eul = np.array([[0.4, 1.1, -0.3]])
    sp = np.zeros(shape, dtype=np.uint16)
    E = np.array([1e-3, -2e-4, -5e-4, 3e-4, -1e-4, 2e-4])
    z = np.zeros((N // 8, 3))
    grad = AD.tangent_linear_gradient(sp, eul, C3, E, z, z, 7, O.default_dt(*C3), 0.05, 1.0)
    _, Ct, _ = O.tables(eul, *C3)
    R = AD.basis_tables(eul)
    ref = [N / 2 * E @ R[i][0] @ E for i in range(3)] + list(N * Ct[0] @ E)
    assert np.allclose(grad, ref, rtol=1e-12, atol=0)
    assert np.allclose(C3[0] * R[0][0] + C3[1] * R[1][0] + C3[2] * R[2][0], Ct[0], atol=1e-12)
