"""torch.autograd.Function over libeph's hand-written adjoint.

    L = EphLoss.apply(g_ReRp, model, kpts, qpts, w_nk, omega_min)
    L.backward()            # g_ReRp.grad = dL/dRe(g) + i dL/dIm(g)

L = sum_{q,k,nu,m,n} w_nk |g_mnnu(k,q)|^2 / omega_qnu (modes with omega > omega_min),
with the eigenvectors U and e held fixed.  One call of eph_interp_backward
gives both L and its gradient (the Re->k stage is recomputed per k tile, never
stored), so forward keeps the gradient for backward.  This module only moves
tensors; the arithmetic runs in the library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import Context


class EphLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, g_ReRp, model, kpts, qpts, w_nk, omega_min):
        g_host = np.ascontiguousarray(g_ReRp.detach().to("cpu", torch.complex128).numpy())
        c = Context(model.nb, model.na, model.H_Re, model.Phi_Rp, g_host, model.Re, model.Rp, model.masses,
                    model.we, model.wp)
        try:
            L, grad = c.loss_and_grad(np.asarray(kpts, dtype=np.float64), np.asarray(qpts, dtype=np.float64),
                                      np.asarray(w_nk, dtype=np.float64), float(omega_min))
        finally:
            c.close()
        fctx.save_for_backward(torch.from_numpy(grad).to(g_ReRp.device))
        return torch.tensor(L, dtype=torch.float64, device=g_ReRp.device)

    @staticmethod
    def backward(fctx, gL):
        (grad,) = fctx.saved_tensors
        return gL.to(grad.dtype) * grad, None, None, None, None, None
