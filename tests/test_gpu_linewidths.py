"""GPU parity of the linewidth consumer (eph_linewidths) against the oracle.

The oracle forms g (oracle.interpolate) and then the imaginary Fan-Migdal
self-energy (oracle.linewidths); libeph forms g in its k-tile workspace (over the
G3 rows) and reduces it to Gamma there, never writing g out.
Inside a group of degenerate bands at k only the group sum of Gamma is gauge
invariant, so Gamma is compared through those sums (groups as in tests/gauge.py).
Bar: max |dGamma| / max Gamma per k <= 1e-10.  The Gaussian delta turns an
eigenvalue error de into a relative error de * |x| / sigma^2 of a term at
distance x; with de ~ 1e-12 * |eps| (FP64 form) and |x| up to a few sigma this
stays below 1e-10 for the widths used here.
"""
import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth
from tests import gauge

pytestmark = pytest.mark.gpu

TOL = 1e-10
KT = 0.025852


@pytest.fixture(scope="module", autouse=True)
def lib():
    import os
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


def grouped_err(g_test, g_ref, eps_k):
    on = gauge.group_onehot(eps_k)                         # [nk][nb][G]
    st = np.einsum("kn,knG->kG", g_test, on)
    sr = np.einsum("kn,knG->kG", g_ref, on)
    den = np.abs(sr).max(-1)
    assert (den > 0).all()
    return float((np.abs(st - sr).max(-1) / den).max())


def reference(wl, kpts, qpts, wq, mu, sigma, omega_min):
    e_k, e_kq, om, g = oracle.interpolate(wl, kpts, qpts)
    return oracle.linewidths(e_k, e_kq, om, g, wq, KT, mu, sigma, omega_min), e_k


@pytest.mark.parametrize("q_batch,k_tile", [(0, 0), (3, 20), (1, 7)])
def test_si_tiny_linewidths(q_batch, k_tile):
    wl = synth.make_workload("si_tiny", nk=50, nq=8)
    rng = np.random.default_rng(5)
    wq = rng.uniform(0.1, 1.0, len(wl.qpts))
    ctx = binding.Context.from_workload(wl, q_batch=q_batch, k_tile=k_tile)
    ctx.set_k(wl.kpts)
    mu = float(np.median(oracle.interpolate(wl, wl.kpts, wl.qpts[:1])[0][:, 3]))
    got = ctx.linewidths(wl.qpts, wq, kT=KT, mu=mu, sigma=0.3, omega_min=1e-6)
    ref, e_k = reference(wl, wl.kpts, wl.qpts, wq, mu, 0.3, 1e-6)
    assert ref.max() > 0
    err = grouped_err(got, ref, e_k)
    assert err <= TOL, f"qb={q_batch} kt={k_tile}: {err:.3e}"


def test_default_weights_and_mode_cut():
    wl = synth.make_workload("si_tiny", nk=20, nq=4)
    wl.qpts[0] = 0.0          # Gamma: acoustic modes fall below omega_min and drop out
    ctx = binding.Context.from_workload(wl)
    ctx.set_k(wl.kpts)
    got = ctx.linewidths(wl.qpts, None, kT=KT, mu=0.0, sigma=0.5, omega_min=1e-4)
    ref, e_k = reference(wl, wl.kpts, wl.qpts, np.ones(len(wl.qpts)), 0.0, 0.5, 1e-4)
    assert grouped_err(got, ref, e_k) <= TOL
    # a cut above every frequency leaves nothing
    none = ctx.linewidths(wl.qpts, None, kT=KT, mu=0.0, sigma=0.5, omega_min=1e3)
    assert np.array_equal(none, np.zeros_like(none))


def test_mos2_shaped_linewidths():
    box = (synth.centred_range(6), synth.centred_range(6), range(0, 1))
    wl = synth.make_workload("mos2", nk=64, nq=6, box=box)
    ctx = binding.Context.from_workload(wl, q_batch=4, k_tile=32)
    ctx.set_k(wl.kpts)
    got = ctx.linewidths(wl.qpts, None, kT=KT, mu=0.0, sigma=0.2, omega_min=1e-6)
    ref, e_k = reference(wl, wl.kpts, wl.qpts, np.ones(len(wl.qpts)), 0.0, 0.2, 1e-6)
    assert grouped_err(got, ref, e_k) <= TOL


def test_si_full_sampled_linewidths():
    # full-size k grid, a few q points; the oracle evaluates a k sample
    wl = synth.make_workload("si_full")
    qsel = wl.qpts[:3].copy()
    ctx = binding.Context.from_workload(wl)
    ctx.set_k(wl.kpts)
    got = ctx.linewidths(qsel, None, kT=KT, mu=0.0, sigma=0.1, omega_min=1e-6)
    ks = np.sort(np.random.default_rng(21).choice(len(wl.kpts), size=800, replace=False))
    ref, e_k = reference(wl, wl.kpts[ks], qsel, np.ones(len(qsel)), 0.0, 0.1, 1e-6)
    assert grouped_err(got[ks], ref, e_k) <= TOL


def test_linewidth_errors():
    wl = synth.make_workload("si_tiny", nk=6, nq=2)
    ctx = binding.Context.from_workload(wl)
    with pytest.raises(binding.EphError) as ei:
        ctx.linewidths(wl.qpts)
    assert ei.value.code == binding.EPH_ESTATE
    ctx.set_k(wl.kpts)
    with pytest.raises(binding.EphError) as ei:
        ctx.linewidths(wl.qpts, sigma=0.0)
    assert ei.value.code == binding.EPH_EINVAL
    # the context still works afterwards
    ctx.linewidths(wl.qpts)


def test_tensor_core_rotation_matches_fused_fp64_kernel():
    # g from the FP64-accuracy tensor-core rotation (in place over G3, then the terms) against the
    # fused CUDA-core kernel (band_alu): ~5e-14 of each pair's largest |g| apart
    wl = synth.make_workload("si_tiny", nk=40, nq=5)
    out = []
    for band_alu in (False, True):
        ctx = binding.Context.from_workload(wl, q_batch=2, k_tile=16, band_alu=band_alu)
        ctx.set_k(wl.kpts)
        out.append(ctx.linewidths(wl.qpts, None, kT=KT, mu=0.0, sigma=0.3, omega_min=1e-6))
    e_k = oracle.interpolate(wl, wl.kpts, wl.qpts[:1])[0]
    assert grouped_err(out[0], out[1], e_k) <= 1e-12


@pytest.mark.parametrize("nb,na", [(20, 2), (8, 7)])
def test_large_shape_linewidths(nb, na):
    # nb or nm > 16: g by the GEMM band rotation over the G3 rows, then the terms kernel
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=12, nq=4)
    ctx = binding.Context.from_workload(wl, q_batch=3, k_tile=5)
    ctx.set_k(wl.kpts)
    got = ctx.linewidths(wl.qpts, None, kT=KT, mu=0.0, sigma=0.4, omega_min=1e-6)
    ref, e_k = reference(wl, wl.kpts, wl.qpts, np.ones(len(wl.qpts)), 0.0, 0.4, 1e-6)
    assert grouped_err(got, ref, e_k) <= TOL


def test_zsnr_ribbon_shape_linewidths():
    wl = synth.make_workload("stanene", nb=32, na=18, nk=6, nq=2)
    ctx = binding.Context.from_workload(wl)
    ctx.set_k(wl.kpts)
    got = ctx.linewidths(wl.qpts, None, kT=KT, mu=0.0, sigma=0.3, omega_min=1e-6)
    ref, e_k = reference(wl, wl.kpts, wl.qpts, np.ones(len(wl.qpts)), 0.0, 0.3, 1e-6)
    assert grouped_err(got, ref, e_k) <= TOL


def test_mixed_form_context_linewidths():
    # a mixed-form context runs the same FP64 chain; its electron eigensolves stop at 1e-12, which
    # the Gaussian turns into ~1e-12 |eps| |x| / sigma^2 of a term
    wl = synth.make_workload("si_tiny", nk=30, nq=4)
    ctx = binding.Context.from_workload(wl, form="mixed")
    ctx.set_k(wl.kpts)
    got = ctx.linewidths(wl.qpts, None, kT=KT, mu=0.0, sigma=0.3, omega_min=1e-6)
    ref, e_k = reference(wl, wl.kpts, wl.qpts, np.ones(len(wl.qpts)), 0.0, 0.3, 1e-6)
    assert grouped_err(got, ref, e_k) <= 1e-9
