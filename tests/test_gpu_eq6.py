"""GPU Bloch -> Wannier transform (Eq. 6, eph_bloch_to_wannier).

The Wannier round trip on the GPU: g(k',q') interpolated by the library on the
Born-von Karman grid whose supercell vectors are the R sets, transformed back
with Eq. 6 in the same gauges, reproduces g(Re,Rp) to 1e-12 (the oracle's own
round trip is a pin in test_oracle_pins.py).  The gauges depend on H and Phi
only, so a context built with a different g(Re,Rp) recovers the first one.
"""
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


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("q_batch,k_tile", [(0, 0), (4, 5)])
def test_round_trip_si_tiny(q_batch, k_tile):
    wl = synth.make_workload("si_tiny")
    coarse = synth.uniform_grid(3, 3, 3)          # the 3x3x3 BvK grid of the [-1,1]^3 box
    ctx = binding.Context.from_workload(wl, q_batch=q_batch, k_tile=k_tile)
    g = ctx.interp(coarse, coarse)[3]
    rec = ctx.bloch_to_wannier(coarse, coarse, g)
    assert rel(rec, wl.g_ReRp) <= 1e-12


def test_other_context_and_oracle():
    wl = synth.make_workload("si_tiny")
    coarse = synth.uniform_grid(3, 3, 3)
    g = binding.Context.from_workload(wl).interp(coarse, coarse)[3]
    other = copy.copy(wl)
    other.g_ReRp = np.zeros_like(wl.g_ReRp)       # same H, Phi: same gauges
    rec = binding.Context.from_workload(other).bloch_to_wannier(coarse, coarse, g)
    assert rel(rec, wl.g_ReRp) <= 1e-12
    # the oracle's Eq. 6 on its own interpolation lands on the same g(Re,Rp)
    _, _, _, go, ev = oracle.interpolate(wl, coarse, coarse, return_eigvecs=True)
    reco = oracle.g_bloch_to_wannier(coarse, coarse, wl.Re, wl.Rp, go, ev["V_k"], ev["V_kq"], ev["u"])
    assert rel(rec, reco) <= 1e-12


def test_round_trip_mos2_shaped_2d():
    box = (synth.centred_range(4), synth.centred_range(4), range(0, 1))
    wl = synth.make_workload("mos2", box=box, nk=1, nq=1)
    coarse = synth.uniform_grid(4, 4, 1)
    ctx = binding.Context.from_workload(wl)
    g = ctx.interp(coarse, coarse)[3]
    assert rel(ctx.bloch_to_wannier(coarse, coarse, g), wl.g_ReRp) <= 1e-12


@pytest.mark.parametrize("name,grid", [("si_tiny", (3, 3, 3)), ("mos2", (4, 4, 1))])
def test_round_trip_on_the_resident_grid(name, grid):
    # Eq. 6 over the coarse grid set by eph_set_k_grid (kpts = NULL): the k' sum runs as the
    # adjoint of the three axis transforms, with unit weights
    if name == "mos2":
        wl = synth.make_workload("mos2", box=(synth.centred_range(4), synth.centred_range(4), range(0, 1)),
                                 nk=1, nq=1)
    else:
        wl = synth.make_workload(name)
    coarse = synth.uniform_grid(*grid)
    ctx = binding.Context.from_workload(wl)
    ctx.set_k_grid(*grid)
    g = ctx.interp_q(coarse)[2]
    assert rel(ctx.bloch_to_wannier(None, coarse, g), wl.g_ReRp) <= 1e-12


def test_device_mode_matches_host_mode():
    torch = pytest.importorskip("torch")
    wl = synth.make_workload("si_tiny")
    coarse = synth.uniform_grid(3, 3, 3)
    g = binding.Context.from_workload(wl).interp(coarse, coarse)[3]
    host = binding.Context.from_workload(wl).bloch_to_wannier(coarse, coarse, g)
    dev = torch.device("cuda:0")
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
    out = torch.empty(wl.g_ReRp.shape, dtype=torch.complex128, device=dev)
    c_d = torch.from_numpy(coarse).to(dev)
    ctx.eph_bloch_to_wannier(len(coarse), c_d, len(coarse), c_d, torch.from_numpy(g).to(dev), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), host)


def test_eq6_errors():
    wl = synth.make_workload("si_tiny", nk=2, nq=2)
    ctx = binding.Context.from_workload(wl)
    with pytest.raises(binding.EphError) as ei:
        ctx.eph_bloch_to_wannier(2, wl.kpts, 2, wl.qpts, None, np.empty(wl.g_ReRp.shape, dtype=np.complex128))
    assert ei.value.code == binding.EPH_EINVAL
    # a mixed-form context runs the same FP64 chain: zero g gives zero g(Re,Rp)
    mixed = binding.Context.from_workload(wl, form="mixed")
    rec = mixed.bloch_to_wannier(wl.kpts, wl.qpts, np.zeros((2, 2, wl.nm, wl.nb, wl.nb), dtype=np.complex128))
    assert not np.any(rec)
