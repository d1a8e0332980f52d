"""The batching workload: a stanene-nanoribbon-shaped context at full shapes (Nb=120, Na=60 so
Nm=180, Ne=Np=15, g(Re,Rp) 9.33 GB, 512 k) with uneven q batches, captured into one CUDA graph
together with a silicon-shaped (Nb=8) and a MoS2-shaped (Nb=11) context, with the autotuner's
(q_batch, k_tile) applied, in both forms.  After a replay, sampled (k, q) of every material are
compared with the FP64 CPU oracle (not with eager calls): eps_k, eps_{k+q} and omega of q
points from every batch, and g (through the gauge-invariant subspace sums) of the q points of
each material's last call, whose g is still in the material's ring buffer.

The silicon- and MoS2-shaped contexts take the workload's q batch sizes as written
(17, 400, 113, 256, 64, 331, 29, 190: 1400 q).  The stanene context takes the first batches of
that list scaled down (mixed form 17, 40, 11, 25; FP64 form 1, 3, 2): one q costs ~0.17 s in
the mixed form and ~2.1 s in the FP64 form at these shapes, so the full 1400 q would take
minutes to an hour per replay."""
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import binding, build_lib, synth
from tests import gauge

pytestmark = pytest.mark.gpu

BATCHES = list(synth.STANENE_Q_BATCHES)
STANENE = {"mixed": ([17, 40, 11, 25], 4), "fp64": ([1, 3, 2], 1)}


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


@pytest.fixture(scope="module")
def workloads():
    si = synth.make_workload("si_tiny", nk=1024, nq=sum(BATCHES))
    mo = synth.make_workload("mos2_diff", nq=sum(BATCHES))            # 48 x 48 k grid
    st = synth.make_workload("stanene")                                # 512 k grid, full shapes
    assert (st.nb, st.nm, st.ne, len(st.kpts)) == (120, 180, 15, 512)
    return si, mo, st


def _check_material(m, form, rng):
    wl = m.wl
    tol_eig = 1e-12 if form == "fp64" else 1e-10
    tol_s = 1e-12 if form == "fp64" else 1e-6
    nk = m.nk
    ks = np.sort(rng.choice(nk, size=min(4, nk), replace=False))
    # one q from every batch (its first point) and the ring's last-call q points
    starts = np.cumsum([0] + m.batches[:-1])
    ring_q = m.last_call_q()[:2]
    qs = sorted(set(int(s) for s in starts) | set(ring_q))
    kpts = wl.kpts[ks]
    qpts = wl.qpts[qs]
    r_k, r_kq, r_om, r_g = oracle.interpolate(wl, kpts, qpts)
    e_k = m.eps_k.cpu().numpy()[ks]
    e_kq = m.eps_kq.cpu().numpy()[qs][:, ks]
    om = m.omega.cpu().numpy()[qs]
    assert gauge.max_rel_eps(e_k, r_k) <= tol_eig, wl.name
    assert gauge.max_rel_eps(e_kq, r_kq) <= tol_eig, wl.name
    assert gauge.max_rel_omega(om, r_om) <= tol_eig, wl.name
    # g of the last call's q points, still in the ring
    ring = m.g_ring.cpu().numpy()
    last = m.last_call_q()
    sel = [qs.index(q) for q in ring_q]
    g_gpu = np.stack([ring[last.index(q)][ks] for q in ring_q]).astype(np.complex128)
    err = gauge.max_rel_S(g_gpu, r_g[sel], r_k, r_kq[sel], r_om[sel])
    assert err <= tol_s, (wl.name, err)
    return err


@pytest.mark.parametrize("form", ["mixed", "fp64"])
def test_three_materials_in_one_graph_match_oracle(form, workloads):
    torch = pytest.importorskip("torch")
    from paper_2603_10295_gb300.batching import graph_of_materials
    si, mo, st = workloads
    sb, sch = STANENE[form]
    specs = [(si, BATCHES, 16, False), (mo, BATCHES, 16, True), (st, sb, sch, False)]
    gb, mats = graph_of_materials(specs, form, "cuda:0", autotune=True)
    for m in mats:   # the autotuner's choice is what the graph's contexts run with
        assert 1 <= m.tuned[0] <= 16 and 0 <= m.tuned[1] < m.nk
    # clear the outputs the eager priming pass wrote, so that what is checked comes from the replay
    for m in mats:
        m.eps_kq.fill_(float("nan"))
        m.omega.fill_(float("nan"))
        m.g_ring.fill_(float("nan"))
    gb.replay()
    gb.check()
    rng = np.random.default_rng(5)
    for m in mats:
        assert torch.isfinite(m.eps_kq).all() and torch.isfinite(m.omega).all()
        _check_material(m, form, rng)
    for m in mats:
        m.ctx.close()
    del gb, mats
    torch.cuda.empty_cache()
