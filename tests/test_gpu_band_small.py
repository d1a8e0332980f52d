"""Fused tensor-core band rotation (nb <= 16, nm nb <= 128): g = V_{k+q}^H G3 V_k as two tcgen05
products of fixed-point BF16 digit operands per tile of (k,q) pairs; four digits in the mixed form,
six digits with exact level sums and integer-assembled doubles in the FP64 form.

Checked against the FP64 CPU oracle on gauge-invariant quantities (|g|^2 subspace sums within the
mixed form's 1e-6) and element by element against the double-float FP32 rotation of the same
context (same G3, same eigenvectors): both round g once to complex64, so they agree to a few
FP32 ulps of each pair's largest element.  Shapes cover every tile arrangement: one, two and four
pairs per tile, K = 16 and 32, ragged last tiles; both inputs: complex64 G3 from the tensor-core
Re->k contraction (k list) and complex128 G3 from the sum-factorised FP64 transforms (uniform grid)."""
import copy
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth
from tests import gauge

pytestmark = pytest.mark.gpu

TOL_S = 1e-6     # mixed form: |g|^2 subspace sums against the FP64 oracle
TOL_FF = 3e-7    # element-wise, relative to the pair's largest |g|: tensor-core vs double-float rotation
TOL_S64 = 1e-12  # FP64 form: |g|^2 subspace sums against the FP64 oracle
TOL_DFMA = 1e-13  # FP64 form, element-wise relative to the pair's largest |g|: six-digit vs DFMA rotation


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


def check(gpu, ref, gff):
    e_k, e_kq, om, g = gpu
    r_k, r_kq, r_om, r_g = ref
    assert g.dtype == np.complex64
    S = gauge.max_rel_S(g, r_g, r_k, r_kq, r_om)
    ff = pair_rel(g, gff)
    print(f"S {S:.3g}  vs double-float {ff:.3g}")
    assert S <= TOL_S
    assert ff <= TOL_FF
    return S, ff


# (nb, na): pairs per tile and K of the tile arrangement
SHAPES = [(8, 2),    # Si-shaped: 48 rows, two pairs per tile, K = 16
          (11, 3),   # MoS2-shaped: 99 rows, one pair, K = 32
          (3, 1),    # 9 rows: four pairs, K = 16
          (9, 1),    # 27 rows: four pairs, K = 32 (N = 128)
          (5, 3),    # 45 rows: two pairs
          (16, 2),   # 96 rows: one pair, K = 32 at its limit
          (1, 1)]    # a single band


@pytest.mark.parametrize("nb,na", SHAPES)
def test_band_small_k_list(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=37, nq=5)
    ref = oracle.interpolate(wl)
    ctx = binding.Context.from_workload(wl, form="mixed", q_batch=3, k_tile=17)
    gpu = ctx.interp(wl.kpts, wl.qpts)
    ff = binding.Context.from_workload(wl, form="mixed", q_batch=3, k_tile=17, band_alu=True)
    gff = ff.interp(wl.kpts, wl.qpts)[3]
    check(gpu, ref, gff)


@pytest.mark.parametrize("nb,na", [(8, 2), (11, 3), (3, 1), (16, 2)])
def test_band_small_grid(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nq=3)
    grid = (3, 4, 5)
    kpts = synth.uniform_grid(*grid)
    ref = oracle.interpolate(wl, kpts, wl.qpts)
    out = []
    for band_alu in (False, True):
        ctx = binding.Context.from_workload(wl, form="mixed", q_batch=2, band_alu=band_alu)
        eps_k = ctx.set_k_grid(*grid)
        out.append((eps_k,) + ctx.interp_q(wl.qpts))
    check(out[0], ref, out[1][3])


def test_band_small_repeated_calls_identical():
    # the tiles are independent of the launch's grid and of earlier calls: same input, same bits
    wl = synth.make_workload("si_tiny", nk=101, nq=4)
    ctx = binding.Context.from_workload(wl, form="mixed")
    a = ctx.interp(wl.kpts, wl.qpts)[3]
    b = ctx.interp(wl.kpts, wl.qpts)[3]
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def check64(gpu, ref, gd):
    e_k, e_kq, om, g = gpu
    r_k, r_kq, r_om, r_g = ref
    assert g.dtype == np.complex128
    S = gauge.max_rel_S(g, r_g, r_k, r_kq, r_om)
    d = pair_rel(g, gd)
    print(f"FP64 S {S:.3g}  vs DFMA {d:.3g}")
    assert S <= TOL_S64
    assert d <= TOL_DFMA
    return S, d


@pytest.mark.parametrize("nb,na", SHAPES)
def test_band_small_fp64_k_list(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=37, nq=5)
    ref = oracle.interpolate(wl)
    gpu = binding.Context.from_workload(wl, q_batch=3, k_tile=17).interp(wl.kpts, wl.qpts)
    gd = binding.Context.from_workload(wl, q_batch=3, k_tile=17, band_alu=True).interp(wl.kpts, wl.qpts)[3]
    check64(gpu, ref, gd)


@pytest.mark.parametrize("nb,na", [(8, 2), (11, 3), (3, 1), (16, 2)])
def test_band_small_fp64_grid(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nq=3)
    grid = (3, 4, 5)
    ref = oracle.interpolate(wl, synth.uniform_grid(*grid), wl.qpts)
    out = []
    for band_alu in (False, True):
        ctx = binding.Context.from_workload(wl, q_batch=2, band_alu=band_alu)
        eps_k = ctx.set_k_grid(*grid)
        out.append((eps_k,) + ctx.interp_q(wl.qpts))
    check64(out[0], ref, out[1][3])


def test_band_small_fp64_scaled_and_zero_inputs():
    # the fixed point is relative to each pair's own scale: couplings scaled by 2^+-200 give the
    # same digits, g scales exactly; an all-zero coupling gives g = 0 exactly
    wl = synth.make_workload("si_tiny", nk=23, nq=3)
    base = binding.Context.from_workload(wl).interp(wl.kpts, wl.qpts)[3]
    for f in (2.0 ** 200, 2.0 ** -200):
        w2 = synth.make_workload("si_tiny", nk=23, nq=3)
        w2.g_ReRp = wl.g_ReRp * f
        g = binding.Context.from_workload(w2).interp(w2.kpts, w2.qpts)[3]
        assert np.array_equal(g, base * f)
    w0 = synth.make_workload("si_tiny", nk=23, nq=3)
    w0.g_ReRp = np.zeros_like(wl.g_ReRp)
    g0 = binding.Context.from_workload(w0).interp(w0.kpts, w0.qpts)[3]
    assert not np.any(g0)


# the adjoint and the VJP take the same FP64 tensor-core rotation, conjugate-transposed, with the
# loss terms in the epilogue of the forward product
TOL_ADJ = 1e-12   # against the FP64 oracle's loss and gradient (relative to the largest element)
TOL_ADJ_ALU = 2e-13  # against the CUDA-core FP64 adjoint of the same context


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("nb,na", [(8, 2), (11, 3), (3, 1), (9, 1), (16, 2), (1, 1)])
def test_band_small_fp64_adjoint(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=29, nq=5)
    rng = np.random.default_rng(nb)
    w = rng.uniform(0.0, 1.0, (len(wl.kpts), wl.nb))
    L, grad = binding.Context.from_workload(wl, q_batch=3, k_tile=13).loss_and_grad(wl.kpts, wl.qpts, w, 1e-6)
    La, ga = binding.Context.from_workload(wl, q_batch=3, k_tile=13, band_alu=True).loss_and_grad(
        wl.kpts, wl.qpts, w, 1e-6)
    Lr, gr = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    print(f"L {abs(L - Lr) / abs(Lr):.3g}  grad {_rel(grad, gr):.3g}  vs ALU {_rel(grad, ga):.3g}")
    assert abs(L - Lr) <= TOL_ADJ * abs(Lr)
    assert _rel(grad, gr) <= TOL_ADJ
    assert abs(L - La) <= TOL_ADJ_ALU * abs(La)
    assert _rel(grad, ga) <= TOL_ADJ_ALU


@pytest.mark.parametrize("nb,na", [(8, 2), (11, 3), (5, 3)])
def test_band_small_fp64_vjp(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=31, nq=4)
    rng = np.random.default_rng(7 + nb)
    shape_g = (len(wl.qpts), len(wl.kpts), wl.nm, wl.nb, wl.nb)
    gbar = rng.standard_normal(shape_g) + 1j * rng.standard_normal(shape_g)
    v = binding.Context.from_workload(wl, q_batch=3, k_tile=11).vjp(wl.kpts, wl.qpts, gbar)
    va = binding.Context.from_workload(wl, q_batch=3, k_tile=11, band_alu=True).vjp(wl.kpts, wl.qpts, gbar)
    # an arbitrary gbar is not gauge covariant: the oracle's eigenvectors give another VJP, so the
    # check is <v, d> = <gbar, A d> with A d from the same context's eigenvectors
    d = rng.standard_normal(wl.g_ReRp.shape) + 1j * rng.standard_normal(wl.g_ReRp.shape)
    wd = copy.copy(wl)
    wd.g_ReRp = d
    Ad = binding.Context.from_workload(wd, q_batch=3, k_tile=11, band_alu=True).interp(wl.kpts, wl.qpts)[3]
    lhs, rhs = np.real(np.vdot(v, d)), np.real(np.vdot(gbar, Ad))
    print(f"vjp dot identity {abs(lhs - rhs) / np.sum(np.abs(gbar) * np.abs(Ad)):.3g}  vs ALU {_rel(v, va):.3g}")
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(gbar) * np.abs(Ad))
    assert _rel(v, va) <= TOL_ADJ_ALU
