"""torch.autograd.Function around the adjoint of the explicit MPM stress solve.

``HMCElastic.apply(theta, spins, euler, nsteps, checkpoint_every, precision, u0, v0)``
with theta = (C11, C12, C44, Ebar_1..6) (a float64 tensor of 9 values; GPa and
Voigt engineering strain) runs ``nsteps`` explicit MPM steps on the frozen
orientation field from the nodal state (u0, v0) (zero when None) and returns
(W, w): the total elastic energy and the per-point field w_p (float64 CPU
tensors).  The backward pass calls the library's reverse sweep
(hmc_adjoint_backward) with the incoming cotangents.  All arithmetic runs in
the CUDA library; torch only carries the values.
"""
from __future__ import annotations

import numpy as np
import torch

from . import HMC, HMC_BC_STRAIN6, HMC_FP32


class HMCElastic(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, spins, euler, nsteps, checkpoint_every, precision=HMC_FP32, u0=None, v0=None):
        th = theta.detach().cpu().double().numpy()
        spins = np.asarray(spins, dtype=np.uint16)
        h = HMC(spins.shape, int(np.asarray(euler).shape[0]), c11=float(th[0]), c12=float(th[1]), c44=float(th[2]),
                bc=HMC_BC_STRAIN6, strain6=tuple(float(x) for x in th[3:9]), mpm_steps_per_mcs=0,
                precision=precision)
        h.set_orientations(euler, spins)
        if u0 is not None or v0 is not None:
            h.set_nodal(u0, v0)
        W, w = h.adjoint_forward(int(nsteps), int(checkpoint_every), want_field=True)
        ctx.h = h
        return torch.tensor(W, dtype=torch.float64), torch.from_numpy(w)

    @staticmethod
    def backward(ctx, gW, gw):
        gWv = 0.0 if gW is None else float(gW)
        g = None if gw is None else gw.detach().cpu().double().numpy()
        grad = ctx.h.adjoint_backward(gWv, g)  # the handle keeps its checkpoints: backward may run again
        return torch.from_numpy(grad), None, None, None, None, None, None, None
