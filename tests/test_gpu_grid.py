"""GPU parity of the product-grid path (eph_set_k_grid): the Re->k contraction as three
one-axis transforms over the bounding box of Re, against the FP64 oracle evaluated on
the same k points (same bar as the list path: 1e-12 on eps, omega and |g|^2 sums)."""
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth
from tests import gauge
from tests.test_gpu_parity import TOL_FP64, check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


def grid_points(n1, n2, n3, shift=(0.0, 0.0, 0.0)):
    return synth.uniform_grid(n1, n2, n3) + np.asarray(shift, dtype=np.float64)[None, :]


def run_grid(ctx, n, qpts, shift=None):
    eps_k = ctx.set_k_grid(*n, shift=shift)
    e_kq, om, g = ctx.interp_q(qpts)
    return eps_k, e_kq, om, g


@pytest.mark.parametrize("n,shift", [((6, 5, 4), None), ((4, 4, 4), (0.125, 0.0, -0.25)), ((1, 7, 2), None),
                                     ((3, 1, 1), (0.5, 0.5, 0.5))])
def test_si_tiny_grid(n, shift):
    wl = synth.make_workload("si_tiny", nq=5)
    ctx = binding.Context.from_workload(wl)
    gpu = run_grid(ctx, n, wl.qpts, shift)
    k = grid_points(*n, shift if shift is not None else (0.0, 0.0, 0.0))
    check(gpu, oracle.interpolate(wl, k, wl.qpts), TOL_FP64, f"grid {n} shift {shift}")


@pytest.mark.parametrize("k_tile", [0, 20, 60])
def test_slab_tiles(k_tile):
    # tiles of whole j1 slabs (20 k each here): the unpaired path on partial j1 ranges
    wl = synth.make_workload("si_tiny", nq=6)
    ctx = binding.Context.from_workload(wl, q_batch=4, k_tile=k_tile)
    gpu = run_grid(ctx, (6, 5, 4), wl.qpts)
    check(gpu, oracle.interpolate(wl, grid_points(6, 5, 4), wl.qpts), TOL_FP64, f"k_tile {k_tile}")


def test_mos2_shaped_grid():
    box = (synth.centred_range(6), synth.centred_range(6), range(0, 1))
    wl = synth.make_workload("mos2", nq=4, box=box)
    ctx = binding.Context.from_workload(wl)
    gpu = run_grid(ctx, (9, 8, 1), wl.qpts)
    check(gpu, oracle.interpolate(wl, grid_points(9, 8, 1), wl.qpts), TOL_FP64, "mos2 grid")


def test_grid_equals_list_path():
    wl = synth.make_workload("si_tiny", nq=4)
    n = (5, 6, 3)
    a = run_grid(binding.Context.from_workload(wl), n, wl.qpts)
    ctx = binding.Context.from_workload(wl)
    b = (ctx.set_k(grid_points(*n)),) + ctx.interp_q(wl.qpts)
    assert gauge.max_rel_eps(a[0], b[0]) <= 1e-13
    assert gauge.max_rel_eps(a[1], b[1]) <= 1e-13
    assert gauge.max_rel_S(a[3], b[3], b[0], b[1], b[2]) <= 1e-12


def test_grid_linewidths_equal_list_path():
    wl = synth.make_workload("si_tiny", nq=4)
    n = (4, 4, 5)
    ctx = binding.Context.from_workload(wl)
    ctx.set_k_grid(*n)
    lw_grid = ctx.linewidths(wl.qpts, sigma=0.3)
    ctx.set_k(grid_points(*n))
    lw_list = ctx.linewidths(wl.qpts, sigma=0.3)
    eps_k = ctx.set_k(grid_points(*n))
    on = gauge.group_onehot(eps_k)
    a = np.einsum("kn,knG->kG", lw_grid, on)
    b = np.einsum("kn,knG->kG", lw_list, on)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()


def test_mixed_form_accepts_grid():
    # the mixed form on a grid: FP64 sum-factorised Re->k, double-float band rotation, complex64 g
    wl = synth.make_workload("si_tiny", nq=3)
    ctx = binding.Context.from_workload(wl, form="mixed")
    eps_k = ctx.set_k_grid(4, 3, 5)
    ref = oracle.interpolate(wl, grid_points(4, 3, 5), wl.qpts)
    assert gauge.max_rel_eps(eps_k, ref[0]) <= 1e-10
    _, _, g = ctx.interp_q(wl.qpts)
    assert gauge.max_rel_S(g, ref[3], ref[0], ref[1], ref[2]) <= 1e-6


def test_grid_errors():
    wl = synth.make_workload("si_tiny", nq=2)
    ctx = binding.Context.from_workload(wl)
    with pytest.raises(binding.EphError) as ei:
        ctx.set_k_grid(0, 4, 4)
    assert ei.value.code == binding.EPH_EINVAL
    with pytest.raises(binding.EphError) as ei:
        ctx.interp_q(wl.qpts)      # the failed call left no k list
    assert ei.value.code == binding.EPH_ESTATE


def test_si_full_grid_sampled():
    torch = pytest.importorskip("torch")
    wl = synth.make_workload("si_full")
    dev = torch.device("cuda:0")
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
    nk, nb, nm = len(wl.kpts), wl.nb, wl.nm
    nq = 4
    qsel = wl.qpts[:nq].copy()
    eps_k = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    eps_kq = torch.empty(nq, nk, nb, dtype=torch.float64, device=dev)
    om = torch.empty(nq, nm, dtype=torch.float64, device=dev)
    g = torch.empty(nq, nk, nm, nb, nb, dtype=torch.complex128, device=dev)
    ctx.eph_set_k_grid(*wl.kgrid, None, eps_k)
    ctx.eph_interp_q(nq, torch.from_numpy(qsel).to(dev), eps_kq, om, g)
    torch.cuda.synchronize()
    ks = np.sort(np.random.default_rng(13).choice(nk, size=1500, replace=False))
    ksel = torch.from_numpy(ks).to(dev)
    gpu = (eps_k[ksel].cpu().numpy(), eps_kq[:, ksel].cpu().numpy(), om.cpu().numpy(), g[:, ksel].cpu().numpy())
    assert np.array_equal(wl.kpts, synth.uniform_grid(*wl.kgrid))
    check(gpu, oracle.interpolate(wl, wl.kpts[ks], qsel), TOL_FP64, "si_full grid")


@pytest.mark.parametrize("k_tile", [0, 24])
def test_mixed_grid_mos2_shaped(k_tile):
    box = (synth.centred_range(6), synth.centred_range(6), range(0, 1))
    wl = synth.make_workload("mos2", nq=4, box=box)
    ctx = binding.Context.from_workload(wl, form="mixed", k_tile=k_tile)
    eps_k = ctx.set_k_grid(8, 6, 1)
    e_kq, om, g = ctx.interp_q(wl.qpts)
    assert g.dtype == np.complex64
    ref = oracle.interpolate(wl, grid_points(8, 6, 1), wl.qpts)
    assert gauge.max_rel_eps(eps_k, ref[0]) <= 1e-10
    assert gauge.max_rel_eps(e_kq, ref[1]) <= 1e-10
    assert gauge.max_rel_omega(om, ref[2]) <= 1e-10
    assert gauge.max_rel_S(g, ref[3], ref[0], ref[1], ref[2]) <= 1e-6
