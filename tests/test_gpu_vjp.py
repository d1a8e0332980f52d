"""GPU vector-Jacobian product (eph_interp_vjp) for arbitrary upstream gradients.

g(k,q) is linear in g(Re,Rp) at fixed gauges, so eph_interp_vjp must be the
adjoint of eph_interp_q: Re<vjp(gbar), d> = Re<gbar, A(d)> for any gbar and d,
with A(d) the library's own forward on d (same H, Phi: the same gauges, bit for
bit).  For gbar = 2 c g it must reproduce eph_interp_backward and the oracle's
loss gradient; through torch.autograd (EphInterp) an arbitrary torch loss on g
backpropagates to g(Re,Rp).
"""
import copy
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("q_batch,k_tile", [(0, 0), (2, 7)])
def test_dot_product_identity(q_batch, k_tile):
    wl = synth.make_workload("si_tiny", nk=30, nq=5)
    rng = np.random.default_rng(3)
    shape_g = (len(wl.qpts), len(wl.kpts), wl.nm, wl.nb, wl.nb)
    gbar = rng.standard_normal(shape_g) + 1j * rng.standard_normal(shape_g)
    d = rng.standard_normal(wl.g_ReRp.shape) + 1j * rng.standard_normal(wl.g_ReRp.shape)
    wd = copy.copy(wl)
    wd.g_ReRp = d
    Ad = binding.Context.from_workload(wd, q_batch=q_batch, k_tile=k_tile).interp(wl.kpts, wl.qpts)[3]
    v = binding.Context.from_workload(wl, q_batch=q_batch, k_tile=k_tile).vjp(wl.kpts, wl.qpts, gbar)
    lhs = np.real(np.vdot(v, d))
    rhs = np.real(np.vdot(gbar, Ad))
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(gbar) * np.abs(Ad))


def test_loss_gradient_is_vjp_of_2cg():
    wl = synth.make_workload("si_tiny", nb=4, nk=24, nq=5)
    rng = np.random.default_rng(4)
    w = rng.uniform(0.0, 1.0, (len(wl.kpts), wl.nb))
    ctx = binding.Context.from_workload(wl)
    _, _, om, g = ctx.interp(wl.kpts, wl.qpts)
    c = oracle.loss_weights(om, w, 1e-6)
    v = ctx.vjp(wl.kpts, wl.qpts, 2 * c[:, :, :, None, :] * g)
    _, grad = binding.Context.from_workload(wl).loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    assert rel(v, grad) <= 1e-13
    _, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    assert rel(v, g_ref) <= 1e-12


def test_mos2_shaped_dot_product():
    box = (synth.centred_range(6), synth.centred_range(6), range(0, 1))
    wl = synth.make_workload("mos2", nk=40, nq=5, box=box)
    rng = np.random.default_rng(5)
    shape_g = (len(wl.qpts), len(wl.kpts), wl.nm, wl.nb, wl.nb)
    gbar = rng.standard_normal(shape_g) + 1j * rng.standard_normal(shape_g)
    d = rng.standard_normal(wl.g_ReRp.shape) + 1j * rng.standard_normal(wl.g_ReRp.shape)
    wd = copy.copy(wl)
    wd.g_ReRp = d
    Ad = binding.Context.from_workload(wd, q_batch=4, k_tile=16).interp(wl.kpts, wl.qpts)[3]
    v = binding.Context.from_workload(wl, q_batch=4, k_tile=16).vjp(wl.kpts, wl.qpts, gbar)
    assert abs(np.real(np.vdot(v, d)) - np.real(np.vdot(gbar, Ad))) <= 1e-12 * np.sum(np.abs(gbar) * np.abs(Ad))


def test_device_mode_matches_host_mode():
    torch = pytest.importorskip("torch")
    wl = synth.make_workload("si_tiny", nk=12, nq=3)
    rng = np.random.default_rng(6)
    shape_g = (len(wl.qpts), len(wl.kpts), wl.nm, wl.nb, wl.nb)
    gbar = rng.standard_normal(shape_g) + 1j * rng.standard_normal(shape_g)
    host = binding.Context.from_workload(wl).vjp(wl.kpts, wl.qpts, gbar)
    dev = torch.device("cuda:0")
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
    out = torch.empty(wl.g_ReRp.shape, dtype=torch.complex128, device=dev)
    ctx.eph_interp_vjp(len(wl.kpts), torch.from_numpy(wl.kpts).to(dev), len(wl.qpts),
                       torch.from_numpy(wl.qpts).to(dev), torch.from_numpy(gbar).to(dev), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), host)


def test_autograd_arbitrary_loss():
    torch = pytest.importorskip("torch")
    from paper_2603_10295_gb300.autograd import EphInterp, EphLoss
    wl = synth.make_workload("si_tiny", nb=4, nk=16, nq=3)
    rng = np.random.default_rng(8)
    w = rng.uniform(0.0, 1.0, (len(wl.kpts), wl.nb))
    # (1) the quadratic loss written in torch on g agrees with the hand-written adjoint
    gW = torch.from_numpy(wl.g_ReRp.copy()).requires_grad_(True)
    g = EphInterp.apply(gW, wl, wl.kpts, wl.qpts)
    om = binding.Context.from_workload(wl).interp(wl.kpts, wl.qpts)[2]
    c = torch.from_numpy(oracle.loss_weights(om, w, 1e-6))[:, :, :, None, :]
    (c * g.abs() ** 2).sum().backward()
    gW2 = torch.from_numpy(wl.g_ReRp.copy()).requires_grad_(True)
    EphLoss.apply(gW2, wl, wl.kpts, wl.qpts, w, 1e-6).backward()
    assert rel(gW.grad.numpy(), gW2.grad.numpy()) <= 1e-12
    # (2) a quartic loss: directional derivative vs central differences along a random d
    gW3 = torch.from_numpy(wl.g_ReRp.copy()).requires_grad_(True)
    (EphInterp.apply(gW3, wl, wl.kpts, wl.qpts).abs() ** 4).sum().backward()
    d = rng.standard_normal(wl.g_ReRp.shape) + 1j * rng.standard_normal(wl.g_ReRp.shape)
    d *= np.linalg.norm(wl.g_ReRp) / np.linalg.norm(d)
    h = 1e-4

    def L4(x):
        w2 = copy.copy(wl)
        w2.g_ReRp = x
        return float(np.sum(np.abs(binding.Context.from_workload(w2).interp(wl.kpts, wl.qpts)[3]) ** 4))

    def D(s):
        return (L4(wl.g_ReRp + s * d) - L4(wl.g_ReRp - s * d)) / (2 * s)

    # L4 along d is a quartic in the step: D(s) = a1 + a3 s^2, so (4 D(h) - D(2h)) / 3 = a1
    fd = (4 * D(h) - D(2 * h)) / 3
    an = float(np.real(np.vdot(gW3.grad.numpy(), d)))
    assert abs(fd - an) <= 1e-8 * abs(an)


def test_autograd_device_path_and_retain_graph():
    # CUDA tensors in and out (the model's context stays on the device; g(Re,Rp) is copied into it
    # on the device), and a second backward through the same graph gives the same gradient
    torch = pytest.importorskip("torch")
    from paper_2603_10295_gb300.autograd import EphInterp, EphLoss, model_context
    dev = torch.device("cuda:0")
    wl = synth.make_workload("si_tiny", nb=4, nk=16, nq=3)
    rng = np.random.default_rng(9)
    w = rng.uniform(0.0, 1.0, (len(wl.kpts), wl.nb))
    kd, qd = torch.from_numpy(wl.kpts).to(dev), torch.from_numpy(wl.qpts).to(dev)
    gW = torch.from_numpy(wl.g_ReRp.copy()).to(dev).requires_grad_(True)
    g = EphInterp.apply(gW, wl, kd, qd)
    assert g.is_cuda
    om = binding.Context.from_workload(wl).interp(wl.kpts, wl.qpts)[2]
    c = torch.from_numpy(oracle.loss_weights(om, w, 1e-6)).to(dev)[:, :, :, None, :]
    loss = (c * g.abs() ** 2).sum()
    loss.backward(retain_graph=True)
    first = gW.grad.clone()
    gW.grad = None
    loss.backward()
    assert torch.equal(gW.grad, first)
    # the loss path on the same cached context, after a different g(Re,Rp) went through it
    gW2 = torch.from_numpy(1.5 * wl.g_ReRp).to(dev).requires_grad_(True)
    EphLoss.apply(gW2, wl, kd, qd, torch.from_numpy(w).to(dev), 1e-6).backward()
    _, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    assert rel(gW2.grad.cpu().numpy(), 1.5 * g_ref) <= 1e-12
    gW3 = torch.from_numpy(wl.g_ReRp.copy()).to(dev).requires_grad_(True)
    EphLoss.apply(gW3, wl, kd, qd, torch.from_numpy(w).to(dev), 1e-6).backward()
    assert rel(first.cpu().numpy(), gW3.grad.cpu().numpy()) <= 1e-12
    assert model_context(wl, dev) is model_context(wl, dev)


def test_vjp_errors():
    wl = synth.make_workload("si_tiny", nk=4, nq=2)
    gbar = np.zeros((2, 4, wl.nm, wl.nb, wl.nb), dtype=np.complex128)
    # a mixed-form context runs the same FP64 chain (H(k+q) and the eigenvectors are all it needs)
    mixed = binding.Context.from_workload(wl, form="mixed")
    assert np.array_equal(mixed.vjp(wl.kpts, wl.qpts, gbar), np.zeros(wl.g_ReRp.shape, dtype=np.complex128))
    ctx = binding.Context.from_workload(wl)
    with pytest.raises(binding.EphError) as ei:
        ctx.eph_interp_vjp(4, wl.kpts, 2, wl.qpts, None, np.empty(wl.g_ReRp.shape, dtype=np.complex128))
    assert ei.value.code == binding.EPH_EINVAL
    assert np.array_equal(ctx.vjp(wl.kpts, wl.qpts, gbar), np.zeros(wl.g_ReRp.shape, dtype=np.complex128))
