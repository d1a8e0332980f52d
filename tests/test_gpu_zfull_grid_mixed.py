"""Full-size sampled parity of the mixed form on the uniform-grid path: the si_full
configuration (40x40x40 k grid, Ne = Np = 216, Nb = 8, Nm = 6) in the launch configuration
of the bench's mixed leg (q batch 4, default k tiles, device buffers), 1,500 sampled k of
all 64,000 against the FP64 oracle at those points.  Bars of the mixed form: |g|^2 subspace
sums within 1e-6, eps and omega within 1e-10."""
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


def test_si_full_grid_sampled_mixed():
    torch = pytest.importorskip("torch")
    wl = synth.make_workload("si_full")
    dev = torch.device("cuda:0")
    ctx = binding.Context.from_workload(wl, form="mixed", device_ptrs=True, q_batch=4,
                                        stream=torch.cuda.current_stream())
    nk, nb, nm = len(wl.kpts), wl.nb, wl.nm
    nq = 4
    qsel = wl.qpts[:nq].copy()
    eps_k = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    eps_kq = torch.empty(nq, nk, nb, dtype=torch.float64, device=dev)
    om = torch.empty(nq, nm, dtype=torch.float64, device=dev)
    g = torch.empty(nq, nk, nm, nb, nb, dtype=torch.complex64, device=dev)
    ctx.eph_set_k_grid(*wl.kgrid, None, eps_k)
    ctx.eph_interp_q(nq, torch.from_numpy(qsel).to(dev), eps_kq, om, g)
    torch.cuda.synchronize()
    ctx.close()
    ks = np.sort(np.random.default_rng(14).choice(nk, size=1500, replace=False))
    ksel = torch.from_numpy(ks).to(dev)
    e_k, e_kq = eps_k[ksel].cpu().numpy(), eps_kq[:, ksel].cpu().numpy()
    w, gs = om.cpu().numpy(), g[:, ksel].cpu().numpy()
    assert np.array_equal(wl.kpts, synth.uniform_grid(*wl.kgrid))
    r_k, r_kq, r_om, r_g = oracle.interpolate(wl, wl.kpts[ks], qsel)
    errs = dict(eps_k=gauge.max_rel_eps(e_k, r_k), eps_kq=gauge.max_rel_eps(e_kq, r_kq),
                omega=gauge.max_rel_omega(w, r_om), S=gauge.max_rel_S(gs, r_g, r_k, r_kq, r_om))
    assert max(errs["eps_k"], errs["eps_kq"], errs["omega"]) <= 1e-10, errs
    assert errs["S"] <= 1e-6, errs
