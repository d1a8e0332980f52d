"""Rp-partitioned g(Re,Rp) on one GPU: contexts that each hold a block of the Rp vectors.

The paper's pools split the Rp vectors of g(Re,Rp) and sum the partial Eq. 9 results over the
pool before the k stage.  Here the slices live in separate contexts on one GPU; their partial G1
(eph_g1_partial) are summed on the device, and eph_interp_q_g1 on one of them must reproduce the
oracle's interpolation (FP64 form 1e-12, mixed form 1e-6 on the subspace sums).  A whole context
fed its own G1 must give exactly what eph_interp_q gives.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth
from paper_2603_10295_gb300.sharding import rp_slice
from tests import gauge

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


def errors(gpu, ref):
    e_k, e_kq, om, g = gpu
    r_k, r_kq, r_om, r_g = ref
    return dict(eps_k=gauge.max_rel_eps(e_k, r_k), eps_kq=gauge.max_rel_eps(e_kq, r_kq),
                omega=gauge.max_rel_omega(om, r_om), S=gauge.max_rel_S(g, r_g, r_k, r_kq, r_om))


def slice_contexts(wl, nslices, **kw):
    out = []
    for r in range(nslices):
        b, c = rp_slice(wl.np_, r, nslices)
        out.append(binding.Context(wl.nb, wl.na, wl.H_Re, wl.Phi_Rp, wl.g_ReRp[b:b + c], wl.Re, wl.Rp, wl.masses,
                                   wl.we, wl.wp, rp_slice=(b, c), **kw))
    return out


@pytest.mark.parametrize("form,nslices,grid", [("fp64", 2, False), ("fp64", 3, True), ("mixed", 2, False),
                                               ("mixed", 4, True)])
def test_slices_summed_match_oracle(form, nslices, grid):
    wl = synth.make_workload("si_tiny", nk=40, nq=7)
    ctxs = slice_contexts(wl, nslices, form=form, q_batch=3)
    if grid:
        kpts = synth.uniform_grid(3, 4, 2)
        eps_k = ctxs[0].set_k_grid(3, 4, 2)
    else:
        kpts = wl.kpts
        eps_k = ctxs[0].set_k(kpts)
    G1 = sum(c.g1_partial(wl.qpts) for c in ctxs)
    gpu = (eps_k,) + ctxs[0].interp_q_g1(wl.qpts, G1)
    errs = errors(gpu, oracle.interpolate(wl, kpts, wl.qpts))
    tol = 1e-12 if form == "fp64" else 1e-6
    assert errs["S"] <= tol and max(errs["eps_k"], errs["eps_kq"], errs["omega"]) <= 1e-10, errs
    if form == "fp64":
        assert max(errs.values()) <= 1e-12, errs
    # the partials are Eq. 9 restricted to each block
    ref_g1 = oracle.g_rp_to_q(wl.qpts, wl.Rp, wl.wp, wl.g_ReRp)
    assert np.abs(G1 - ref_g1).max() <= 1e-13 * np.abs(ref_g1).max()


def test_device_partials_summed_on_the_device():
    # the one-GPU picture of two ranks: two Rp halves, partial G1 in device tensors, their sum
    # (the all-reduce) formed on the device, then the k stage from it
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()
    wl = synth.make_workload("si_tiny", nk=50, nq=6)
    a, b = slice_contexts(wl, 2, device_ptrs=True, stream=st)
    kd, qd = torch.from_numpy(wl.kpts).to(dev), torch.from_numpy(wl.qpts).to(dev)
    nk, nq, nb, nm = len(wl.kpts), len(wl.qpts), wl.nb, wl.nm
    eps_k = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    a.eph_set_k(nk, kd, eps_k)
    shape = (nq, nm, wl.ne, nb, nb)
    G1a = torch.empty(shape, dtype=torch.complex128, device=dev)
    G1b = torch.empty(shape, dtype=torch.complex128, device=dev)
    a.eph_g1_partial(nq, qd, G1a)
    b.eph_g1_partial(nq, qd, G1b)
    G1a += G1b
    eps_kq = torch.empty(nq, nk, nb, dtype=torch.float64, device=dev)
    om = torch.empty(nq, nm, dtype=torch.float64, device=dev)
    g = torch.empty(nq, nk, nm, nb, nb, dtype=torch.complex128, device=dev)
    a.eph_interp_q_g1(nq, qd, G1a, eps_kq, om, g)
    torch.cuda.synchronize()
    gpu = (eps_k.cpu().numpy(), eps_kq.cpu().numpy(), om.cpu().numpy(), g.cpu().numpy())
    errs = errors(gpu, oracle.interpolate(wl))
    assert max(errs.values()) <= 1e-12, errs


def test_whole_context_given_its_own_g1_is_bit_identical():
    wl = synth.make_workload("si_tiny", nk=30, nq=5)
    ctx = binding.Context.from_workload(wl, q_batch=2)
    ctx.set_k(wl.kpts)
    ref = ctx.interp_q(wl.qpts)
    got = ctx.interp_q_g1(wl.qpts, ctx.g1_partial(wl.qpts))
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)


def test_slice_context_refuses_whole_g_calls():
    wl = synth.make_workload("si_tiny", nk=8, nq=2)
    a, _ = slice_contexts(wl, 2)
    a.set_k(wl.kpts)
    for call in (lambda: a.interp_q(wl.qpts),
                 lambda: a.loss_and_grad(wl.kpts, wl.qpts, np.ones((8, wl.nb)), 1e-6),
                 lambda: a.linewidths(wl.qpts)):
        with pytest.raises(binding.EphError) as ei:
            call()
        assert ei.value.code == binding.EPH_ESTATE
    a.set_k(wl.kpts)   # the context stays usable
    assert a.g1_partial(wl.qpts).shape == (2, wl.nm, wl.ne, wl.nb, wl.nb)


def test_set_gw_replaces_the_resident_coupling():
    # eph_set_gw (the autograd path's update of g(Re,Rp)) equals a context created with that g
    wl = synth.make_workload("si_tiny", nk=20, nq=3)
    rng = np.random.default_rng(4)
    g2 = rng.standard_normal(wl.g_ReRp.shape) + 1j * rng.standard_normal(wl.g_ReRp.shape)
    ctx = binding.Context.from_workload(wl)
    ctx.eph_set_gw(np.ascontiguousarray(g2))
    wl2 = synth.make_workload("si_tiny", nk=20, nq=3)
    wl2.g_ReRp = g2
    fresh = binding.Context.from_workload(wl2)
    for x, y in zip(ctx.interp(wl.kpts, wl.qpts), fresh.interp(wl.kpts, wl.qpts)):
        assert np.array_equal(x, y)
