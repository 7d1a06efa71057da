"""torch.autograd entry point of the reverse mode (kbe_backward).

``occupations(system, A, U, nsteps)`` runs the time stepping on the GPU with
the Peierls samples ``A`` (1-D float64 tensor) and the constant interaction
``U`` (0-d float64 tensor) and returns the occupations n_kb(t_nsteps)
(float64 tensor [nk][nb]). Its backward calls kbe_backward on the same
handle: dL/dA and dL/dU come from the library's hand-written adjoint, not
from torch's autograd of any torch operations (none run here).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from ._binding import KBE, KBE_PREC_FP64


class KBEFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, U, system, nsteps):
        sys_ = dataclasses.replace(system, A=A.detach().cpu().numpy().astype(np.float64), U=float(U))
        k = KBE.from_system(sys_, nt_max=max(int(nsteps), len(sys_.A)), precision=KBE_PREC_FP64)
        k.step(int(nsteps))
        nkb, _ = k.observables(int(nsteps))
        ctx.handle = k
        ctx.nA = A.shape[0]
        return torch.from_numpy(nkb).to(A.device)

    @staticmethod
    def backward(ctx, g):
        k = ctx.handle
        dA, dU = k.backward(g.detach().cpu().numpy())
        k.close()
        ctx.handle = None
        gA = torch.from_numpy(dA[: ctx.nA].copy()).to(g.device)
        gU = torch.tensor(dU, dtype=torch.float64, device=g.device)
        return gA, gU, None, None


def occupations(system, A, U, nsteps):
    """n_kb(t_nsteps) of `system` (a kbe_inputs.System) with drive A and interaction U."""
    return KBEFunction.apply(A, U, system, nsteps)
