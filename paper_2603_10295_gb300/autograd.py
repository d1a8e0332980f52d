"""torch.autograd.Functions over libeph's hand-written adjoint.

    L = EphLoss.apply(g_ReRp, model, kpts, qpts, w_nk, omega_min)
    L.backward()            # g_ReRp.grad = dL/dRe(g) + i dL/dIm(g)

    g = EphInterp.apply(g_ReRp, model, kpts, qpts)    # [nq][nk][nm][nb][nb]
    any_loss(g).backward()  # through eph_interp_vjp

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


class EphInterp(torch.autograd.Function):
    """g(k,q) as a differentiable function of g(Re,Rp) (U_k, U_{k+q}, e_q held fixed).

    forward: eph_interp; backward: eph_interp_vjp with the upstream gradient.  The
    context of the forward is kept for the backward, so both see the same gauges.
    """

    @staticmethod
    def forward(fctx, g_ReRp, model, kpts, qpts):
        g_host = np.ascontiguousarray(g_ReRp.detach().to("cpu", torch.complex128).numpy())
        c = Context(model.nb, model.na, model.H_Re, model.Phi_Rp, g_host, model.Re, model.Rp, model.masses,
                    model.we, model.wp)
        kpts = np.ascontiguousarray(kpts, dtype=np.float64)
        qpts = np.ascontiguousarray(qpts, dtype=np.float64)
        _, _, _, g = c.interp(kpts, qpts)
        fctx.lib_ctx, fctx.kpts, fctx.qpts = c, kpts, qpts
        return torch.from_numpy(g).to(g_ReRp.device)

    @staticmethod
    def backward(fctx, grad_g):
        c = fctx.lib_ctx
        try:
            gin = np.ascontiguousarray(grad_g.detach().to("cpu", torch.complex128).numpy())
            grad = c.vjp(fctx.kpts, fctx.qpts, gin)
        finally:
            c.close()
        return torch.from_numpy(grad).to(grad_g.device), None, None, None
