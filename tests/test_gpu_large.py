"""Shapes beyond the warp-resident kernels (nb or nm > 16): CTA-per-matrix
Jacobi, GEMM-based mode and band rotations (FP64 form; the mixed form runs the
band rotation as double-float GEMMs and returns complex64 g).  The main case is
the narrowest zigzag-stanene ribbon of the paper's Table 3 (Nb=32, Nm=54) on the
15-vector 1-D box of the stanene workload."""
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth
from tests import gauge

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


def check(gpu, ref, what, tol_eig=TOL_FP64, tol_s=TOL_FP64):
    e_k, e_kq, om, g = gpu
    r_k, r_kq, r_om, r_g = ref
    errs = dict(eps_k=gauge.max_rel_eps(e_k, r_k), eps_kq=gauge.max_rel_eps(e_kq, r_kq),
                omega=gauge.max_rel_omega(om, r_om), S=gauge.max_rel_S(g, r_g, r_k, r_kq, r_om))
    print(what, errs)
    for k, v in errs.items():
        assert v <= (tol_s if k == "S" else tol_eig), (what, errs)


def check_mixed(gpu, ref, what):
    assert gpu[3].dtype == np.complex64
    check(gpu, ref, what, tol_eig=1e-10, tol_s=1e-6)


def test_zsnr_narrowest_ribbon_shape():
    wl = synth.make_workload("stanene", nb=32, na=18, nk=6, nq=3)
    assert (wl.nb, wl.nm, wl.ne) == (32, 54, 15)
    ctx = binding.Context.from_workload(wl, q_batch=2, k_tile=4)
    check(ctx.interp(wl.kpts, wl.qpts), oracle.interpolate(wl), "zsnr 32/54")


@pytest.mark.parametrize("nb,na", [(20, 2), (8, 7)])
def test_mixed_small_and_large(nb, na):
    # large bands with small modes, and small bands with large modes
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=9, nq=4)
    ctx = binding.Context.from_workload(wl, q_batch=3)
    check(ctx.interp(wl.kpts, wl.qpts), oracle.interpolate(wl), f"nb={nb} nm={3 * na}")


def test_zsnr_narrowest_ribbon_shape_mixed():
    wl = synth.make_workload("stanene", nb=32, na=18, nk=6, nq=3)
    ctx = binding.Context.from_workload(wl, form="mixed", q_batch=2, k_tile=4)
    check_mixed(ctx.interp(wl.kpts, wl.qpts), oracle.interpolate(wl), "zsnr 32/54 mixed")


@pytest.mark.parametrize("nb,na", [(20, 2), (8, 7)])
def test_mixed_form_small_and_large(nb, na):
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=9, nq=4)
    ctx = binding.Context.from_workload(wl, form="mixed", q_batch=3)
    check_mixed(ctx.interp(wl.kpts, wl.qpts), oracle.interpolate(wl), f"mixed nb={nb} nm={3 * na}")


def test_mixed_large_odd_row_length():
    # Nm Nb odd (17 x 3): the tensor-core band rotation needs an even row length, so this shape
    # takes the FP64 Re->k flow with the double-float band rotation
    wl = synth.make_workload("si_tiny", nb=17, na=1, nk=6, nq=3)
    assert (wl.nm * wl.nb) % 2 == 1
    ctx = binding.Context.from_workload(wl, form="mixed", q_batch=2)
    check_mixed(ctx.interp(wl.kpts, wl.qpts), oracle.interpolate(wl), "mixed nb=17 nm=3")


def test_large_shapes_rejected_where_not_supported():
    # the persistent multi-material rotation keeps its warp-resident kernel: nb, nm <= 16
    import torch
    dev = torch.device("cuda:0")
    wl = synth.make_workload("si_tiny", nb=20, nk=4, nq=2)
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
    ctx.eph_set_k(len(wl.kpts), torch.from_numpy(wl.kpts).to(dev))
    q = torch.from_numpy(wl.qpts).to(dev)
    with pytest.raises(binding.EphError) as ei:
        binding.interp_q_multi([ctx], [2], [q])
    assert ei.value.code == binding.EPH_ENOTSUP


def test_stanene_full_shape_few_points():
    # the stanene-nanoribbon workload's full shapes: Nb=120, Na=60 (Nm=180), Ne=Np=15,
    # g(Re,Rp) 9.33 GB; two k and one q point keep the FP64 oracle affordable
    wl = synth.make_workload("stanene", nk=2, nq=1)
    assert (wl.nb, wl.nm, wl.ne) == (120, 180, 15)
    ctx = binding.Context.from_workload(wl)
    gpu = ctx.interp(wl.kpts, wl.qpts)
    ref = oracle.interpolate(wl)
    check(gpu, ref, "stanene 120/180")
    del ctx
    mixed = binding.Context.from_workload(wl, form="mixed")
    check_mixed(mixed.interp(wl.kpts, wl.qpts), ref, "stanene 120/180 mixed")
