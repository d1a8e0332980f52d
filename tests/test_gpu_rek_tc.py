"""FP64 form, k list: the Re->k contraction of Eq. 10 (H(k+q) and G3 = P_k W_q) on the tensor
cores at FP64 accuracy (`k_tc_zgemm64`: seven balanced base-128 digits per operand with a
power-of-two scale per phase row and per W_q column, exact level sums, doubles assembled from
64-bit integers) against the FP64 DFMA GEMM of the same context (option gemm_alu) and against
the FP64 CPU oracle.  The fixed point is relative to each column's largest term, so the bars are
relative to each pair's largest |g|^2 and to the eigenvalue scale: eps_kq and omega within 1e-13,
|g|^2 subspace sums within 1e-12 of the oracle, g element-wise within 1e-12 of the DFMA path.
Shapes: ragged k tiles (M not a multiple of 128), several q per batch (tiles across q), the
silicon- and MoS2-shaped Re sets (K = 2 Ne = 432, 288) and the largest K the scheme allows."""
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth
from tests import gauge

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


def pair_rel(g, gref):
    nq, nk = g.shape[:2]
    d = np.abs(g - gref).reshape(nq, nk, -1).max(axis=2)
    m = np.abs(gref).reshape(nq, nk, -1).max(axis=2)
    return float((d / np.where(m > 0, m, 1.0)).max())


def run(wl, kpts, qpts, **kw):
    return binding.Context.from_workload(wl, **kw).interp(kpts, qpts)


@pytest.mark.parametrize("name,nk,nq,qb,kt", [("si_tiny", 301, 5, 3, 130), ("si_tiny", 97, 4, 4, 0),
                                              ("mos2_diff", 210, 3, 2, 0)])
def test_tensor_core_rek_against_dfma_and_oracle(name, nk, nq, qb, kt):
    wl = synth.make_workload(name, nk=nk, nq=nq)
    tc = run(wl, wl.kpts, wl.qpts, q_batch=qb, k_tile=kt)
    al = run(wl, wl.kpts, wl.qpts, q_batch=qb, k_tile=kt, gemm_alu=True)
    ref = oracle.interpolate(wl)
    e_kq = gauge.max_rel_eps(tc[1], ref[1])
    om = gauge.max_rel_omega(tc[2], ref[2])
    S = gauge.max_rel_S(tc[3], ref[3], ref[0], ref[1], ref[2])
    d = pair_rel(tc[3], al[3])
    print(f"{name}: eps_kq {e_kq:.3g} omega {om:.3g} S {S:.3g} vs DFMA {d:.3g}")
    assert e_kq <= 1e-13 and om <= 1e-13
    assert S <= 1e-12
    assert d <= 1e-12
    assert np.abs(tc[1] - al[1]).max() <= 1e-13 * np.abs(al[1]).max()


def test_tensor_core_rek_si_full_re_set():
    # the silicon benchmark's Re box (Ne = 216: K = 432) on a few k and q
    wl = synth.make_workload("si_full", nk=150, nq=2)
    tc = run(wl, wl.kpts, wl.qpts)
    ref = oracle.interpolate(wl)
    S = gauge.max_rel_S(tc[3], ref[3], ref[0], ref[1], ref[2])
    assert gauge.max_rel_eps(tc[1], ref[1]) <= 1e-13
    assert S <= 1e-12


def test_tensor_core_rek_scaled_and_zero_couplings():
    # per-column scales: g(Re,Rp) scaled by 2^+-300 scales g exactly; zero couplings give g = 0
    wl = synth.make_workload("si_tiny", nk=40, nq=2)
    base = run(wl, wl.kpts, wl.qpts)[3]
    for f in (2.0 ** 300, 2.0 ** -300):
        w2 = synth.make_workload("si_tiny", nk=40, nq=2)
        w2.g_ReRp = wl.g_ReRp * f
        assert np.array_equal(run(w2, w2.kpts, w2.qpts)[3], base * f)
    w0 = synth.make_workload("si_tiny", nk=40, nq=2)
    w0.g_ReRp = np.zeros_like(wl.g_ReRp)
    assert not np.any(run(w0, w0.kpts, w0.qpts)[3])


def test_backward_on_a_k_list_with_tensor_core_rek():
    wl = synth.make_workload("si_tiny", nk=70, nq=3)
    eps_k, _ = oracle.electron_eigen(oracle.hamiltonian_k(wl.kpts, wl.Re, wl.we, wl.H_Re))
    w = oracle.fermi_weights(eps_k, 2)[0]
    L_ref, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    L, grad = binding.Context.from_workload(wl, q_batch=2, k_tile=33).loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    assert abs(L - L_ref) <= 1e-12 * abs(L_ref)
    assert float(np.abs(grad - g_ref).max() / np.abs(g_ref).max()) <= 1e-12


# Eq. 9 (G1 = P_q g(Re,Rp)) and the adjoint's gradient GEMM (grad += P_q^H G1bar) take the same
# tensor-core GEMM: against the DFMA kernels of the same context (option gemm_alu)
# on a uniform grid gemm_alu also selects the FP64 axis transforms of the sum factorisation
# instead of their double-float form (whole unshifted axes of at most 9 slots in the FP64 form:
# the silicon boxes here; the 13-slot MoS2 box keeps FP64 transforms)
@pytest.mark.parametrize("name,grid", [("mos2_diff", None), ("si_tiny", (4, 5, 6)), ("si_tiny", (3, 3, 3))])
def test_eq9_tensor_core_against_dfma_on_the_grid(name, grid):
    wl = synth.make_workload(name, nq=5)
    grid = grid or wl.kgrid
    out = []
    for alu in (False, True):
        ctx = binding.Context.from_workload(wl, q_batch=3, gemm_alu=alu)
        eps_k = ctx.set_k_grid(*grid)
        out.append((eps_k,) + ctx.interp_q(wl.qpts))
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-13 * np.abs(out[1][1]).max()
    d = pair_rel(out[0][3], out[1][3])
    print(f"{name} {grid}: tensor-core Eq. 9 and double-float axes vs DFMA: g {d:.3g}")
    assert d <= 1e-12


def test_backward_gradient_gemm_tensor_core_against_dfma():
    wl = synth.make_workload("mos2_diff", nq=6)
    eps_k, _ = oracle.electron_eigen(oracle.hamiltonian_k(wl.kpts, wl.Re, wl.we, wl.H_Re))
    w = oracle.fermi_weights(eps_k, 2)[0]
    res = []
    for alu in (False, True):
        ctx = binding.Context.from_workload(wl, q_batch=2, gemm_alu=alu)
        ctx.set_k_grid(*wl.kgrid)
        res.append(ctx.loss_and_grad(None, wl.qpts, w, 1e-6))
    (L, g), (La, ga) = res
    print(f"backward tensor cores vs DFMA: L {abs(L - La) / abs(La):.3g} grad {np.abs(g - ga).max() / np.abs(ga).max():.3g}")
    assert abs(L - La) <= 1e-12 * abs(La)
    assert np.abs(g - ga).max() <= 1e-12 * np.abs(ga).max()
