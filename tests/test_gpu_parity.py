"""GPU parity: libeph (through the C-ABI) against the FP64 CPU oracle.

Eigenvalues and frequencies are compared directly; g through the
gauge-invariant subspace sums S (tests/gauge.py).  FP64 form bar: max relative
error <= 1e-12 (normwise per point for eps and omega, per (k,q) pair for S).
"""
import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth
from tests import gauge

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    import os
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


def check(gpu, ref, tol, what=""):
    e_k, e_kq, om, g = gpu
    r_k, r_kq, r_om, r_g = ref
    errs = dict(eps_k=gauge.max_rel_eps(e_k, r_k), eps_kq=gauge.max_rel_eps(e_kq, r_kq),
                omega=gauge.max_rel_omega(om, r_om), S=gauge.max_rel_S(g, r_g, r_k, r_kq, r_om))
    for k, v in errs.items():
        assert v <= tol, f"{what} {k}: {v:.3e} > {tol:.1e}  (all: {errs})"
    return errs


@pytest.mark.parametrize("q_batch,k_tile", [(0, 0), (3, 20), (16, 64), (1, 1)])
@pytest.mark.parametrize("plain", [False, True])
def test_si_tiny_fp64(q_batch, k_tile, plain):
    # plain: FP64 Jacobi sweeps only; else FP32-preconditioned sweeps finished in FP64
    wl = synth.make_workload("si_tiny")
    ctx = binding.Context.from_workload(wl, q_batch=q_batch, k_tile=k_tile, eig_plain_fp64=plain)
    gpu = ctx.interp(wl.kpts, wl.qpts)
    check(gpu, oracle.interpolate(wl), TOL_FP64, f"si_tiny qb={q_batch} kt={k_tile} plain={plain}")


def test_mos2_shaped_small_fp64():
    box = (synth.centred_range(6), synth.centred_range(6), range(0, 1))
    wl = synth.make_workload("mos2", nk=77, nq=9, box=box)
    ctx = binding.Context.from_workload(wl, q_batch=4, k_tile=32)
    check(ctx.interp(wl.kpts, wl.qpts), oracle.interpolate(wl), TOL_FP64, "mos2 small")


@pytest.mark.parametrize("nb,nk,nq", [(1, 5, 3), (2, 1, 1), (3, 7, 2), (11, 6, 2), (12, 5, 2), (16, 9, 2)])
def test_edge_sizes(nb, nk, nq):
    wl = synth.make_workload("si_tiny", nb=nb, nk=nk, nq=nq)
    ctx = binding.Context.from_workload(wl)
    check(ctx.interp(wl.kpts, wl.qpts), oracle.interpolate(wl), TOL_FP64, f"nb={nb}")


def test_single_atom_and_gamma():
    wl = synth.make_workload("si_tiny", nk=6, nq=3)
    # one atom: nm = 3; include q = Gamma (three zero modes) and k = q = 0
    wl.masses = wl.masses[:1]
    wl.na = 1
    wl.Phi_Rp = np.ascontiguousarray(wl.Phi_Rp[:, :3, :3])
    wl.g_ReRp = np.ascontiguousarray(wl.g_ReRp[:, :3])
    wl.kpts[0] = 0.0
    wl.qpts[0] = 0.0
    ctx = binding.Context.from_workload(wl)
    gpu = ctx.interp(wl.kpts, wl.qpts)
    ref = oracle.interpolate(wl)
    e_k, e_kq, om, g = gpu
    assert gauge.max_rel_eps(e_k, ref[0]) <= TOL_FP64
    # at Gamma the acoustic frequencies are ~sqrt(rounding): compare eigenvalues omega^2 instead
    lam_g = np.sign(om) * om ** 2
    lam_r = np.sign(ref[2]) * ref[2] ** 2
    assert gauge.max_rel_eps(lam_g, lam_r) <= 1e-12
    # S only where the three acoustic modes are excluded (their eigenvectors are arbitrary
    # inside the degenerate zero subspace, which grouping handles)
    assert gauge.max_rel_S(g, ref[3], ref[0], ref[1], ref[2]) <= TOL_FP64


def test_device_pointer_mode_matches_host_mode():
    torch = pytest.importorskip("torch")
    wl = synth.make_workload("si_tiny", nk=40, nq=6)
    host = binding.Context.from_workload(wl).interp(wl.kpts, wl.qpts)
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=st)
    kp = torch.from_numpy(wl.kpts).to(dev)
    qp = torch.from_numpy(wl.qpts).to(dev)
    nk, nq, nb, nm = len(wl.kpts), len(wl.qpts), wl.nb, wl.nm
    eps_k = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    eps_kq = torch.empty(nq, nk, nb, dtype=torch.float64, device=dev)
    om = torch.empty(nq, nm, dtype=torch.float64, device=dev)
    g = torch.empty(nq, nk, nm, nb, nb, dtype=torch.complex128, device=dev)
    ctx.eph_set_k(nk, kp, eps_k)
    ctx.eph_interp_q(nq, qp, eps_kq, om, g)
    torch.cuda.synchronize()
    out = (eps_k.cpu().numpy(), eps_kq.cpu().numpy(), om.cpu().numpy(), g.cpu().numpy())
    # identical kernels and launch shapes: bitwise equal
    for a, b in zip(out, host):
        assert np.array_equal(a, b)
    assert ctx.launches() > 0


def test_error_paths():
    wl = synth.make_workload("si_tiny", nk=4, nq=2)
    ctx = binding.Context.from_workload(wl)
    with pytest.raises(binding.EphError) as ei:
        ctx.interp_q(wl.qpts)
    assert ei.value.code == binding.EPH_ESTATE
    # a sweep cap of 1 cannot converge an 8x8 Jacobi: reported, not hung
    ctx1 = binding.Context.from_workload(wl, max_sweeps=1, eig_plain_fp64=True)
    with pytest.raises(binding.EphError) as ei:
        ctx1.set_k(wl.kpts)
    assert ei.value.code == binding.EPH_ENOTCONV
    # the context stays usable after the error
    ctx.set_k(wl.kpts)
    ctx.interp_q(wl.qpts)


def _sampled_full_size(name, nq_check, nk_sample, seed):
    torch = pytest.importorskip("torch")
    wl = synth.make_workload(name)
    dev = torch.device("cuda:0")
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
    nk, nb, nm = len(wl.kpts), wl.nb, wl.nm
    kp = torch.from_numpy(wl.kpts).to(dev)
    qsel = wl.qpts[:nq_check].copy()
    qp = torch.from_numpy(qsel).to(dev)
    eps_k = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    eps_kq = torch.empty(nq_check, nk, nb, dtype=torch.float64, device=dev)
    om = torch.empty(nq_check, nm, dtype=torch.float64, device=dev)
    g = torch.empty(nq_check, nk, nm, nb, nb, dtype=torch.complex128, device=dev)
    ctx.eph_set_k(nk, kp, eps_k)
    ctx.eph_interp_q(nq_check, qp, eps_kq, om, g)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    ks = np.sort(rng.choice(nk, size=nk_sample, replace=False))
    ksel = torch.from_numpy(ks).to(dev)
    gpu = (eps_k[ksel].cpu().numpy(), eps_kq[:, ksel].cpu().numpy(), om.cpu().numpy(), g[:, ksel].cpu().numpy())
    ref = oracle.interpolate(wl, wl.kpts[ks], qsel)
    return gpu, ref


def test_si_full_sampled_fp64():
    gpu, ref = _sampled_full_size("si_full", nq_check=4, nk_sample=1500, seed=11)
    check(gpu, ref, TOL_FP64, "si_full")


def test_mos2_full_sampled_fp64():
    gpu, ref = _sampled_full_size("mos2", nq_check=3, nk_sample=1200, seed=12)
    check(gpu, ref, TOL_FP64, "mos2")


@pytest.mark.parametrize("form,grid", [("fp64", False), ("fp64", True), ("mixed", True)])
def test_async_host_mode_matches_sync(form, grid):
    # async mode with host buffers: g is copied on a second stream while the next call computes;
    # after eph_sync every output equals the synchronous call's, bit for bit
    torch = pytest.importorskip("torch")
    wl = synth.make_workload("si_tiny", nk=60, nq=9)
    sync = binding.Context.from_workload(wl, form=form, q_batch=3)
    asyn = binding.Context.from_workload(wl, form=form, q_batch=3, async_mode=True)
    if grid:
        sync.set_k_grid(3, 4, 5)
        asyn.eph_set_k_grid(3, 4, 5)
    else:
        sync.set_k(wl.kpts)
        asyn.eph_set_k(len(wl.kpts), wl.kpts)
    nk, nb, nm = sync.nk, wl.nb, wl.nm
    gdt = torch.complex128 if form == "fp64" else torch.complex64
    outs = [(torch.empty(3, nk, nb, dtype=torch.float64).pin_memory(), torch.empty(3, nm, dtype=torch.float64).pin_memory(),
             torch.empty(3, nk, nm, nb, nb, dtype=gdt).pin_memory()) for _ in range(3)]
    q = torch.from_numpy(wl.qpts.copy()).pin_memory()
    for i in range(3):
        asyn.eph_interp_q(3, q[3 * i:3 * i + 3], *outs[i])
    asyn.eph_sync()
    for i in range(3):
        ref = sync.interp_q(wl.qpts[3 * i:3 * i + 3])
        for a, b in zip(outs[i], ref):
            assert np.array_equal(a.numpy(), b)


@pytest.mark.parametrize("grid", [False, True])
def test_async_host_mode_back_to_back_large_copies(grid):
    # g of one q is ~120 MB here, so its device->host copy (on the copy stream) is still running
    # when the next asynchronous call reaches its band rotation into the same staging buffer;
    # that rotation has to wait for the copy.  Four calls in a row, one q each, into distinct
    # pinned buffers, must equal the synchronous calls bit for bit.
    torch = pytest.importorskip("torch")
    wl = synth.make_workload("si_tiny", nk=20000, nq=4)
    sync = binding.Context.from_workload(wl, q_batch=1)
    asyn = binding.Context.from_workload(wl, q_batch=1, async_mode=True)
    if grid:
        sync.set_k_grid(25, 20, 40)
        asyn.eph_set_k_grid(25, 20, 40)
    else:
        sync.set_k(wl.kpts)
        asyn.eph_set_k(len(wl.kpts), wl.kpts)
    nk, nb, nm = sync.nk, wl.nb, wl.nm
    outs = [(torch.empty(1, nk, nb, dtype=torch.float64).pin_memory(), torch.empty(1, nm, dtype=torch.float64).pin_memory(),
             torch.empty(1, nk, nm, nb, nb, dtype=torch.complex128).pin_memory()) for _ in range(4)]
    q = torch.from_numpy(wl.qpts.copy()).pin_memory()
    for i in range(4):
        asyn.eph_interp_q(1, q[i:i + 1], *outs[i])
    asyn.eph_sync()
    for i in range(4):
        ref = sync.interp_q(wl.qpts[i:i + 1])
        for a, b in zip(outs[i], ref):
            assert np.array_equal(a.numpy(), b)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_phase_reduction_exact_far_from_the_cell(form):
    # k and q on a 1/8 grid plus integer offsets up to 2^20: every product k_i n_i and their
    # sum t are exact in FP64, so the exact reduction t - rint(t) gives the phases of the points
    # inside the cell (cell-based phases are periodic); a phase formed in lower precision, or
    # from a rounded 2 pi t, is off by ~1e-9 there.  Both lists match the oracle at the in-cell
    # points (eigenvalues and frequencies directly, g through the subspace sums).
    rng = np.random.default_rng(21)
    wl = synth.make_workload("si_tiny", nk=9, nq=3)
    k0 = rng.integers(0, 8, (9, 3)) / 8.0
    q0 = rng.integers(0, 8, (3, 3)) / 8.0
    kf = k0 + rng.integers(-(1 << 20), 1 << 20, (9, 3))
    qf = q0 + rng.integers(-(1 << 20), 1 << 20, (3, 3))
    ref = oracle.interpolate(wl, k0, q0)
    for pts in ((k0, q0), (kf, qf)):
        got = binding.Context.from_workload(wl, form=form).interp(*pts)
        if form == "fp64":
            check(got, ref, TOL_FP64, "far points")
        else:
            e_k, e_kq, om, g = got
            assert max(gauge.max_rel_eps(e_k, ref[0]), gauge.max_rel_eps(e_kq, ref[1]),
                       gauge.max_rel_omega(om, ref[2])) <= 1e-10
            assert gauge.max_rel_S(g, ref[3], ref[0], ref[1], ref[2]) <= 1e-6


def test_phase_reduction_grid_shift_far_from_the_cell():
    # the uniform-grid path with an integer-plus-dyadic shift of 2^19: the same points as the
    # unshifted grid after reduction, so the oracle at the in-cell points is the reference
    wl = synth.make_workload("si_tiny", nk=2, nq=3)
    n = (4, 2, 8)
    base = (0.125, 0.0, -0.25)
    far = (0.125 + (1 << 19), -3.0 * (1 << 17), -0.25 - 12345.0)
    a = binding.Context.from_workload(wl)
    near = (a.set_k_grid(*n, shift=base),) + a.interp_q(wl.qpts)
    b = binding.Context.from_workload(wl)
    shifted = (b.set_k_grid(*n, shift=far),) + b.interp_q(wl.qpts)
    k = synth.uniform_grid(*n) + np.asarray(base)[None, :]
    ref = oracle.interpolate(wl, k, wl.qpts)
    check(near, ref, TOL_FP64, "grid, in-cell shift")
    check(shifted, ref, TOL_FP64, "grid, far shift")


def test_empty_inputs_rejected_and_context_kept():
    # empty k, q and matrix batches are argument errors; the resident k list survives them
    wl = synth.make_workload("si_tiny", nk=4, nq=2)
    ctx = binding.Context.from_workload(wl)
    ref = ctx.interp(wl.kpts, wl.qpts)
    for call in (lambda: ctx.set_k(np.zeros((0, 3))), lambda: ctx.interp_q(np.zeros((0, 3))),
                 lambda: ctx.eigh(np.zeros((0, 4, 4), dtype=np.complex128))):
        with pytest.raises(binding.EphError) as ei:
            call()
        assert ei.value.code == binding.EPH_EINVAL
    again = ctx.interp_q(wl.qpts)
    for a, b in zip(ref[1:], again):
        assert np.array_equal(a, b)
