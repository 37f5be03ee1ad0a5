"""PyTorch autograd bridge for the misfit gradient (sbp_misfit_gradient): argument marshalling only.

``misfit(solver, rho, C, ...)`` returns the receiver misfit as a 0-d tensor whose backward yields
dPhi/drho and dPhi/dC per block, C in the pair layout (10 planes) or the Voigt layout (6 planes).  The forward call already runs the
library's checkpointed adjoint (the adjoint needs the forward levels anyway), so backward only
scales the stored gradients by the incoming grad_output.  Material tensors live wherever the caller
keeps them; they are copied to host FP64 arrays for ``sbp_set_material`` (the library copies host
arrays), and the gradients come back as tensors on the same device and dtype.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import C_PAIR10, pair10


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, spec, *mats):
        S, nsteps, dt, observed, u_prev, u_cur, t0, ck, layout = spec
        nb = len(S.problem.blocks)
        rhos, Cs = mats[:nb], mats[nb:]
        for b in range(nb):
            r = np.ascontiguousarray(rhos[b].detach().to("cpu", torch.float64).numpy())
            c = np.ascontiguousarray(Cs[b].detach().to("cpu", torch.float64).numpy())
            S._check(S.L.sbp_set_material(S.h, b, r.ctypes.data_as(_dp()), c.ctypes.data_as(_dp()), layout))
        S.sbp_set_state(u_prev, u_cur, t0)
        phi, gr, gc = S.sbp_misfit_gradient(nsteps, dt, observed, checkpoint_every=ck, layout=layout)
        ctx.grads = [torch.as_tensor(g, dtype=m.dtype, device=m.device) for g, m in zip(gr, rhos)] + \
                    [torch.as_tensor(g, dtype=m.dtype, device=m.device) for g, m in zip(gc, Cs)]
        return torch.tensor(phi, dtype=rhos[0].dtype, device=rhos[0].device)

    @staticmethod
    def backward(ctx, grad_out):
        return (None,) + tuple(grad_out * g for g in ctx.grads)


def _dp():
    import ctypes
    return ctypes.POINTER(ctypes.c_double)


def pair_planes(Cfull):
    """Full stiffness tensor C[I,J,K,L,...] (numpy or tensor) -> the 10 pair planes sbp_set_material takes."""
    if isinstance(Cfull, torch.Tensor):
        return torch.stack([Cfull[p // 2, p % 2, q // 2, q % 2] for p in range(4) for q in range(p, 4)])
    return pair10(Cfull)


def misfit(solver, rho, C, u_prev, u_cur, t0, nsteps, dt, observed, checkpoint_every=0, layout=C_PAIR10):
    """Receiver misfit of ``nsteps`` leapfrog steps from (u_prev, u_cur) at time t0 with the material
    (rho[b]: (N2, N1), C[b]: (10, N2, N1) pair planes, or (6, N2, N1) Voigt planes with layout=C_VOIGT6)
    as a differentiable function of rho and C.
    ``solver`` must have its receivers set (sbp_set_receivers)."""
    spec = (solver, int(nsteps), float(dt), observed, u_prev, u_cur, float(t0), int(checkpoint_every), int(layout))
    return _Misfit.apply(spec, *rho, *C)
