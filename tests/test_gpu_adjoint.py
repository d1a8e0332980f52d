"""GPU adjoint (eph_interp_backward) against the FP64 CPU adjoint, central
finite differences, and invariants that hold at any size."""
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


def weights(wl, kpts):
    eps_k, _ = oracle.electron_eigen(oracle.hamiltonian_k(kpts, wl.Re, wl.we, wl.H_Re))
    w, _ = oracle.fermi_weights(eps_k, 2)
    return w


def rel_grad_err(g, r):
    return float(np.abs(g - r).max() / np.abs(r).max())


@pytest.mark.parametrize("q_batch,k_tile", [(0, 0), (2, 7)])
def test_backward_matches_cpu_adjoint(q_batch, k_tile):
    wl = synth.make_workload("si_tiny", nb=4, nk=24, nq=5)
    w = weights(wl, wl.kpts)
    L_ref, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    ctx = binding.Context.from_workload(wl, q_batch=q_batch, k_tile=k_tile)
    L, grad = ctx.loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    assert abs(L - L_ref) <= 1e-12 * abs(L_ref)
    assert rel_grad_err(grad, g_ref) <= 1e-12


def test_backward_mos2_diff_subset():
    wl = synth.make_workload("mos2_diff")
    qs = wl.qpts[:3]
    w = weights(wl, wl.kpts)
    L_ref, g_ref = oracle.loss_and_grad(wl, wl.kpts, qs, w, 1e-6)
    ctx = binding.Context.from_workload(wl)
    L, grad = ctx.loss_and_grad(wl.kpts, qs, w, 1e-6)
    assert abs(L - L_ref) <= 1e-12 * abs(L_ref)
    assert rel_grad_err(grad, g_ref) <= 1e-12


@pytest.mark.parametrize("name,grid,k_tile", [("si_tiny", (3, 4, 5), 0), ("si_tiny", (3, 4, 5), 20),
                                               ("mos2_diff", (48, 48, 1), 0)])
def test_backward_on_a_uniform_grid_sum_factorised(name, grid, k_tile):
    # kpts = NULL after eph_set_k_grid: the forward Re->k sum and its adjoint both run as three
    # one-axis transforms (k_tile 20 = one j1 slab: the axis-1 adjoint accumulates over tiles)
    wl = synth.make_workload(name, nq=3) if name == "mos2_diff" else synth.make_workload(name, nb=4, nq=3)
    kpts = synth.uniform_grid(*grid)
    w = weights(wl, kpts)
    L_ref, g_ref = oracle.loss_and_grad(wl, kpts, wl.qpts, w, 1e-6)
    ctx = binding.Context.from_workload(wl, k_tile=k_tile)
    ctx.set_k_grid(*grid)
    L, grad = ctx.loss_and_grad(None, wl.qpts, w, 1e-6)
    assert abs(L - L_ref) <= 1e-12 * abs(L_ref)
    assert rel_grad_err(grad, g_ref) <= 1e-12
    # the vector-Jacobian product on the grid equals the one on the same points as a list
    rng = np.random.default_rng(12)
    shape_g = (len(wl.qpts), len(kpts), wl.nm, wl.nb, wl.nb)
    gbar = rng.standard_normal(shape_g) + 1j * rng.standard_normal(shape_g)
    v_grid = ctx.vjp(None, wl.qpts, gbar)
    v_list = binding.Context.from_workload(wl).vjp(kpts, wl.qpts, gbar)
    assert rel_grad_err(v_grid, v_list) <= 1e-12


def test_backward_central_differences():
    wl = synth.make_workload("si_tiny", nb=4, nk=16, nq=3)
    w = weights(wl, wl.kpts)
    L0, grad = binding.Context.from_workload(wl).loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    rng = np.random.default_rng(9)
    flat = wl.g_ReRp.reshape(-1)
    h = 1e-6
    for i in rng.choice(flat.size, size=6, replace=False):
        for unit, part in ((1.0, "re"), (1j, "im")):
            Ls = []
            for sgn in (1, -1):
                w2 = copy.copy(wl)
                gg = flat.copy()
                gg[i] += sgn * unit * h
                w2.g_ReRp = gg.reshape(wl.g_ReRp.shape)
                Ls.append(binding.Context.from_workload(w2).loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)[0])
            fd = (Ls[0] - Ls[1]) / (2 * h)
            ref = grad.reshape(-1)[i].real if part == "re" else grad.reshape(-1)[i].imag
            assert abs(fd - ref) <= 1e-6 * max(1.0, np.abs(grad).max())


def test_backward_full_size_invariants():
    # mos2_diff at full size (48x48 k x 256 q): Euler's identity Re<grad, gW> = 2L and
    # additivity over a split of the q list hold exactly for any size.
    wl = synth.make_workload("mos2_diff")
    w = weights(wl, wl.kpts)
    ctx = binding.Context.from_workload(wl)
    L, grad = ctx.loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    assert abs(np.real(np.vdot(grad, wl.g_ReRp)) - 2 * L) <= 1e-11 * abs(L)
    La, ga = ctx.loss_and_grad(wl.kpts, wl.qpts[:100], w, 1e-6)
    Lb, gb = ctx.loss_and_grad(wl.kpts, wl.qpts[100:], w, 1e-6)
    assert abs(La + Lb - L) <= 1e-12 * abs(L)
    assert rel_grad_err(ga + gb, grad) <= 1e-12


def test_device_mode_and_autograd():
    torch = pytest.importorskip("torch")
    from paper_2603_10295_gb300.autograd import EphLoss
    wl = synth.make_workload("si_tiny", nb=4, nk=20, nq=4)
    w = weights(wl, wl.kpts)
    L_ref, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    # device-pointer mode through the C-ABI
    dev = torch.device("cuda:0")
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
    L_d = torch.zeros(1, dtype=torch.float64, device=dev)
    g_d = torch.empty(wl.g_ReRp.shape, dtype=torch.complex128, device=dev)
    ctx.eph_interp_backward(len(wl.kpts), torch.from_numpy(wl.kpts).to(dev), len(wl.qpts),
                            torch.from_numpy(wl.qpts).to(dev), torch.from_numpy(w).to(dev), 1e-6, L_d, g_d)
    torch.cuda.synchronize()
    assert abs(L_d.item() - L_ref) <= 1e-12 * abs(L_ref)
    assert rel_grad_err(g_d.cpu().numpy(), g_ref) <= 1e-12
    # torch.autograd.Function
    gW = torch.from_numpy(wl.g_ReRp.copy()).to(dev).requires_grad_(True)
    L = EphLoss.apply(gW, wl, wl.kpts, wl.qpts, w, 1e-6)
    (3.0 * L).backward()
    assert abs(L.item() - L_ref) <= 1e-12 * abs(L_ref)
    assert rel_grad_err(gW.grad.cpu().numpy(), 3.0 * g_ref) <= 1e-12


def test_backward_on_mixed_form_context():
    # a mixed-form context differentiates through the same FP64 adjoint chain; only its
    # eigensolves are polished to 1e-12 instead of rounding level
    wl = synth.make_workload("si_tiny", nb=4, nk=24, nq=5)
    w = weights(wl, wl.kpts)
    L_ref, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    ctx = binding.Context.from_workload(wl, form="mixed")
    L, grad = ctx.loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    assert abs(L - L_ref) <= 1e-9 * abs(L_ref)
    assert rel_grad_err(grad, g_ref) <= 1e-8
