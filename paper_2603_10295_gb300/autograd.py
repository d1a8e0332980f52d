"""torch.autograd.Functions over libeph's hand-written adjoint.

    L = EphLoss.apply(g_ReRp, model, kpts, qpts, w_nk, omega_min)
    L.backward()            # g_ReRp.grad = dL/dRe(g) + i dL/dIm(g)
    # kpts=None: the model's uniform k grid (model.kgrid), sum-factorised Re->k in both directions

    g = EphInterp.apply(g_ReRp, model, kpts, qpts)    # [nq][nk][nm][nb][nb]
    any_loss(g).backward()  # through eph_interp_vjp

L = sum_{q,k,nu,m,n} w_nk |g_mnnu(k,q)|^2 / omega_qnu (modes with omega > omega_min),
with the eigenvectors U and e held fixed.  One call of eph_interp_backward
gives both L and its gradient (the Re->k stage is recomputed per k tile, never
stored), so forward keeps the gradient for backward.

`model` holds the Wannier data that do not change during training (H(Re), Phi(Rp), the R
sets, weights and masses; a synth.Workload or any object with those attributes).  One
device-pointer context per (model, device, stream) is created on first use and kept for the
model's lifetime: each forward only copies the current g(Re,Rp) tensor into it on the device
(eph_set_gw), points, weights and outputs are device tensors, and the upstream gradient of
EphInterp goes to eph_interp_vjp as a device pointer, so nothing crosses to the host.  The
context outlives each backward, so retain_graph=True and repeated backward calls work.  This
module only moves tensors; the arithmetic runs in the library's CUDA kernels.
"""
from __future__ import annotations

import threading
import weakref

import torch

from .binding import Context

_cache: dict = {}
_lock = threading.Lock()


def _device_of(t: torch.Tensor) -> torch.device:
    return t.device if t.is_cuda else torch.device("cuda", torch.cuda.current_device())


def model_context(model, device: torch.device) -> Context:
    """The model's FP64 device-pointer context on `device` and torch's current stream there."""
    stream = torch.cuda.current_stream(device)
    key = (id(model), device.index, int(stream.cuda_stream))
    with _lock:
        ctx = _cache.get(key)
        if ctx is None:
            with torch.cuda.device(device):
                ctx = Context(model.nb, model.na, model.H_Re, model.Phi_Rp, model.g_ReRp, model.Re, model.Rp,
                              model.masses, model.we, model.wp, device_ptrs=True, stream=stream)
            _cache[key] = ctx
            weakref.finalize(model, _drop, key)
    return ctx


def _drop(key):
    with _lock:
        ctx = _cache.pop(key, None)
    if ctx is not None:
        ctx.close()


def _dev(x, device, dtype):
    return torch.as_tensor(x, dtype=dtype).to(device).contiguous()


def _k_points(ctx, model, kpts, dev):
    """(nk, device k list or None).  kpts None: the model's uniform grid (model.kgrid), made the
    context's resident k list once, so that the Re->k sums run sum-factorised."""
    if kpts is not None:
        kd = _dev(kpts, dev, torch.float64)
        return kd.shape[0], kd
    grid = tuple(getattr(model, "kgrid", None) or ())
    if len(grid) != 3:
        raise ValueError("kpts=None needs a model with a uniform k grid (model.kgrid)")
    if getattr(ctx, "_grid", None) != grid or ctx.nk != grid[0] * grid[1] * grid[2]:
        ctx.eph_set_k_grid(*grid)
        ctx._grid = grid
    return ctx.nk, None


class EphLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, g_ReRp, model, kpts, qpts, w_nk, omega_min):
        dev = _device_of(g_ReRp)
        ctx = model_context(model, dev)
        gW = g_ReRp.detach().to(dev, torch.complex128).contiguous()
        qd = _dev(qpts, dev, torch.float64)
        wd = _dev(w_nk, dev, torch.float64)
        L = torch.zeros(1, dtype=torch.float64, device=dev)
        grad = torch.empty(gW.shape, dtype=torch.complex128, device=dev)
        with torch.cuda.device(dev):
            ctx.eph_set_gw(gW)
            nk, kd = _k_points(ctx, model, kpts, dev)
            ctx.eph_interp_backward(nk, kd, qd.shape[0], qd, wd, float(omega_min), L, grad)
            if kd is not None:
                ctx._grid = None   # the call made kpts the resident list
        fctx.save_for_backward(grad.to(g_ReRp.device))
        return L[0].to(g_ReRp.device)

    @staticmethod
    def backward(fctx, gL):
        (grad,) = fctx.saved_tensors
        return gL.to(grad.dtype) * grad, None, None, None, None, None


class EphInterp(torch.autograd.Function):
    """g(k,q) as a differentiable function of g(Re,Rp) (U_k, U_{k+q}, e_q held fixed).

    forward: eph_set_k + eph_interp_q; backward: eph_interp_vjp with the upstream gradient.
    Both run on the model's context, whose gauges depend only on H(Re) and Phi(Rp), so the
    backward sees the gauges of the forward bit for bit.
    """

    @staticmethod
    def forward(fctx, g_ReRp, model, kpts, qpts):
        dev = _device_of(g_ReRp)
        ctx = model_context(model, dev)
        gW = g_ReRp.detach().to(dev, torch.complex128).contiguous()
        kd, qd = _dev(kpts, dev, torch.float64), _dev(qpts, dev, torch.float64)
        nk, nq = kd.shape[0], qd.shape[0]
        g = torch.empty((nq, nk, ctx.nm, ctx.nb, ctx.nb), dtype=torch.complex128, device=dev)
        with torch.cuda.device(dev):
            ctx.eph_set_gw(gW)
            ctx.eph_set_k(nk, kd)
            ctx._grid = None
            ctx.eph_interp_q(nq, qd, None, None, g)
        fctx.model, fctx.dev, fctx.in_device = model, dev, g_ReRp.device
        fctx.save_for_backward(kd, qd)
        return g.to(g_ReRp.device)

    @staticmethod
    def backward(fctx, grad_g):
        kd, qd = fctx.saved_tensors
        dev = fctx.dev
        ctx = model_context(fctx.model, dev)
        gin = grad_g.detach().to(dev, torch.complex128).contiguous()
        out = torch.empty((ctx.np_, ctx.nm, ctx.ne, ctx.nb, ctx.nb), dtype=torch.complex128, device=dev)
        with torch.cuda.device(dev):
            ctx.eph_interp_vjp(kd.shape[0], kd, qd.shape[0], qd, gin, out)
            ctx._grid = None
        return out.to(fctx.in_device), None, None, None
