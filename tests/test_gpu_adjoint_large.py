"""Derived paths of the interpolation for shapes beyond the warp-resident kernels (nb or nm > 16):
the adjoint (eph_interp_backward), the vector-Jacobian product (eph_interp_vjp) and the Bloch ->
Wannier transform of Eq. 6 (eph_bloch_to_wannier).  The band rotation's adjoint runs as FP64
GEMMs batched over (k, nu), like the forward of these shapes, with the loss terms in a kernel of
their own; the mode rotation's adjoint as one GEMM per q batched over Re.

Checked against the FP64 CPU oracle's loss and gradient (gauge invariant), the dot-product
identity <A^H gbar, d> = <gbar, A d> for an arbitrary upstream gradient, and the Wannier round trip
on the Born-von Karman grid of the R sets.  Shapes: large bands with small modes, small bands with
large modes, both large, and the narrowest zigzag-stanene ribbon of the paper's Table 3
(Nb=32, Nm=54) on the stanene workload's 15-vector box."""
import copy
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def weights(wl, kpts):
    eps_k, _ = oracle.electron_eigen(oracle.hamiltonian_k(kpts, wl.Re, wl.we, wl.H_Re))
    return oracle.fermi_weights(eps_k, min(2, wl.nb - 1))[0]


@pytest.mark.parametrize("nb,na", [(20, 2), (8, 7), (24, 6)])
def test_backward_large_shapes(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=9, nq=4)
    w = weights(wl, wl.kpts)
    L_ref, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    L, grad = binding.Context.from_workload(wl, q_batch=3, k_tile=5).loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    print(f"nb={nb} nm={wl.nm}: L {abs(L - L_ref) / abs(L_ref):.3g} grad {rel(grad, g_ref):.3g}")
    assert abs(L - L_ref) <= TOL * abs(L_ref)
    assert rel(grad, g_ref) <= TOL


def test_backward_zsnr_narrowest_ribbon():
    wl = synth.make_workload("stanene", nb=32, na=18, nk=6, nq=3)
    assert (wl.nb, wl.nm, wl.ne) == (32, 54, 15)
    w = weights(wl, wl.kpts)
    L_ref, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    L, grad = binding.Context.from_workload(wl, q_batch=2, k_tile=4).loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    print(f"zsnr 32/54: L {abs(L - L_ref) / abs(L_ref):.3g} grad {rel(grad, g_ref):.3g}")
    assert abs(L - L_ref) <= TOL * abs(L_ref)
    assert rel(grad, g_ref) <= TOL


def test_backward_large_on_mixed_form_context():
    # the same FP64 chain; the electron eigensolves of a mixed-form context stop at 1e-12
    wl = synth.make_workload("si_tiny", nb=20, na=2, nk=9, nq=4)
    w = weights(wl, wl.kpts)
    L_ref, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    L, grad = binding.Context.from_workload(wl, form="mixed", q_batch=3).loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    assert abs(L - L_ref) <= 1e-9 * abs(L_ref)
    assert rel(grad, g_ref) <= 1e-8


def test_backward_large_on_a_uniform_grid():
    wl = synth.make_workload("si_tiny", nb=20, na=2, nq=3)
    grid = (3, 4, 5)
    kpts = synth.uniform_grid(*grid)
    w = weights(wl, kpts)
    L_ref, g_ref = oracle.loss_and_grad(wl, kpts, wl.qpts, w, 1e-6)
    ctx = binding.Context.from_workload(wl, q_batch=2)
    ctx.set_k_grid(*grid)
    L, grad = ctx.loss_and_grad(None, wl.qpts, w, 1e-6)
    assert abs(L - L_ref) <= TOL * abs(L_ref)
    assert rel(grad, g_ref) <= TOL


@pytest.mark.parametrize("nb,na", [(20, 2), (8, 7)])
def test_vjp_large_dot_product_identity(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=8, nq=3)
    rng = np.random.default_rng(nb + na)
    shape_g = (len(wl.qpts), len(wl.kpts), wl.nm, wl.nb, wl.nb)
    gbar = rng.standard_normal(shape_g) + 1j * rng.standard_normal(shape_g)
    d = rng.standard_normal(wl.g_ReRp.shape) + 1j * rng.standard_normal(wl.g_ReRp.shape)
    wd = copy.copy(wl)
    wd.g_ReRp = d
    Ad = binding.Context.from_workload(wd, q_batch=2, k_tile=5).interp(wl.kpts, wl.qpts)[3]
    v = binding.Context.from_workload(wl, q_batch=2, k_tile=5).vjp(wl.kpts, wl.qpts, gbar)
    lhs, rhs = np.real(np.vdot(v, d)), np.real(np.vdot(gbar, Ad))
    assert abs(lhs - rhs) <= TOL * np.sum(np.abs(gbar) * np.abs(Ad))


def test_vjp_large_is_the_loss_gradient():
    # the VJP of 2 c g equals the adjoint's gradient (both FP64 chains of the same context)
    wl = synth.make_workload("si_tiny", nb=20, na=7, nk=8, nq=3)
    w = weights(wl, wl.kpts)
    ctx = binding.Context.from_workload(wl)
    _, _, om, g = ctx.interp(wl.kpts, wl.qpts)
    c = oracle.loss_weights(om, w, 1e-6)
    v = ctx.vjp(wl.kpts, wl.qpts, 2 * c[:, :, :, None, :] * g)
    _, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    assert rel(v, g_ref) <= TOL


@pytest.mark.parametrize("nb,na", [(20, 2), (8, 7)])
def test_eq6_round_trip_large(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na)
    coarse = synth.uniform_grid(3, 3, 3)          # the BvK grid of the [-1,1]^3 box
    ctx = binding.Context.from_workload(wl, q_batch=4, k_tile=10)
    g = ctx.interp(coarse, coarse)[3]
    rec = ctx.bloch_to_wannier(coarse, coarse, g)
    assert rel(rec, wl.g_ReRp) <= TOL


def test_vjp_and_eq6_on_mixed_form_context():
    # the VJP and Eq. 6 need only H(k+q), D(q) and the eigenvectors: FP64 chains in either form
    wl = synth.make_workload("si_tiny")
    coarse = synth.uniform_grid(3, 3, 3)
    g = binding.Context.from_workload(wl).interp(coarse, coarse)[3]
    rec = binding.Context.from_workload(wl, form="mixed").bloch_to_wannier(coarse, coarse, g)
    # the mixed context's electron gauges agree with the FP64 context's to the 1e-12 polish
    assert rel(rec, wl.g_ReRp) <= 1e-9
