"""torch.autograd.Function over the hand-written adjoint (shl_grad).

    C = HomogenizeFn.apply(pos, q, iso, t, handle, r, K, alpha, opts)

pos (n,3), q (n,), iso (), t () are float64 CPU tensors (the design
parameters); C is the 6x6 homogenised tensor (float64, CPU).  Forward runs the
whole path on the GPU with the smoothed density and keeps the displacements on
the device; backward passes dE/dC^H to shl_grad with those displacements as
the initial guess, so the backward pass needs no new CG iterations.  Torch is
used for tensors only; every step runs in libshl.
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs, shl


class HomogenizeFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, pos, q, iso, t, handle, r, K, alpha, opts):
        design = inputs.Design(pos=pos.detach().cpu().double().numpy().copy(),
                               q=q.detach().cpu().double().numpy().copy(),
                               alpha=None if alpha is None else np.asarray(alpha, dtype=np.float64),
                               iso=float(iso), K=int(K), t=float(t))
        o = shl.default_solve_opts()
        for f, _ in shl.shl_solve_opts._fields_:
            setattr(o, f, getattr(opts, f))
        o.density = shl.SHL_SMOOTH
        o.warm_start = 0
        u = torch.empty(18 * r ** 3, dtype=torch.float64, device=shl.ctx_device(handle))
        res = shl.shl_grad(handle, design, r, o, np.zeros(36), u=u)
        fctx.state = (handle, design, r, o, u)
        return torch.tensor(res["C"], dtype=torch.float64)

    @staticmethod
    def backward(fctx, gC):
        handle, design, r, o, u = fctx.state
        o.warm_start = 1
        res = shl.shl_grad(handle, design, r, o, gC.detach().cpu().double().numpy(), u=u)
        return (torch.tensor(res["g_pos"]), torch.tensor(res["g_q"]), torch.tensor(res["g_iso"]),
                torch.tensor(res["g_t"]), None, None, None, None, None)
