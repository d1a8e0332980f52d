"""Batching: materials of different shape (silicon-like Nb=8/Nm=6, MoS2-like
Nb=11/Nm=9 and a stanene-family ribbon Nb=32/Nm=54) with uneven q batches, in
both forms, captured into one CUDA graph; replays must reproduce the eager results exactly, also after new q
points are copied into the captured inputs.  The autotuner must pick a valid
decomposition that leaves the results unchanged."""
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


def _materials(form):
    si = synth.make_workload("si_tiny", nk=150, nq=40)
    box = (synth.centred_range(6), synth.centred_range(6), range(0, 1))
    mo = synth.make_workload("mos2", nk=120, nq=40, box=box)
    mats = [(si, [3, 5, 1]), (mo, [2, 7])]
    # a stanene-family ribbon (Table 3's narrowest: Nb=32, Nm=54) on the 15-vector 1-D box
    mats.append((synth.make_workload("stanene", nb=32, na=18, nk=10, nq=40), [1, 2]))
    return mats


def _buffers(torch, wl, nq, form, dev):
    nk, nb, nm = len(wl.kpts), wl.nb, wl.nm
    gdt = torch.complex128 if form == "fp64" else torch.complex64
    return (torch.empty(nq, nk, nb, dtype=torch.float64, device=dev), torch.empty(nq, nm, dtype=torch.float64, device=dev),
            torch.empty(nq, nk, nm, nb, nb, dtype=gdt, device=dev))


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_graph_replay_matches_eager(form):
    torch = pytest.importorskip("torch")
    from paper_2603_10295_gb300.batching import GraphBatcher
    dev = torch.device("cuda:0")
    gb = GraphBatcher(dev)
    eager, keep = [], []
    for wl, batches in _materials(form):
        ctx = binding.Context.from_workload(wl, form=form, device_ptrs=True, async_mode=True, stream=gb.stream)
        ctx.eph_set_k(len(wl.kpts), torch.from_numpy(wl.kpts).to(dev))
        ref_ctx = binding.Context.from_workload(wl, form=form)
        ref_ctx.set_k(wl.kpts)
        q0 = 0
        for nq in batches:
            q = torch.from_numpy(wl.qpts[q0:q0 + nq].copy()).to(dev)
            bufs = _buffers(torch, wl, nq, form, dev)
            gb.add(ctx, q, *bufs)
            eager.append((ref_ctx, wl, q0, nq, bufs))
            q0 += nq
        keep.append(ctx)
    gb.capture()
    for shift in (0, 20):                        # second round: new q points copied into the captured inputs
        if shift:
            for (ref_ctx, wl, q0, nq, _), item in zip(eager, gb.items):
                item[1].copy_(torch.from_numpy(wl.qpts[q0 + shift:q0 + shift + nq].copy()).to(dev))
        gb.replay()
        gb.check()
        for (ref_ctx, wl, q0, nq, bufs) in eager:
            e_kq, om, g = ref_ctx.interp_q(wl.qpts[q0 + shift:q0 + shift + nq])
            assert np.array_equal(bufs[0].cpu().numpy(), e_kq)
            assert np.array_equal(bufs[1].cpu().numpy(), om)
            assert np.array_equal(bufs[2].cpu().numpy(), g)


def test_autotune_picks_valid_tiles_and_keeps_results():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    wl = synth.make_workload("si_tiny", nk=500, nq=6)
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
    nk = len(wl.kpts)
    ctx.eph_set_k(nk, torch.from_numpy(wl.kpts).to(dev))
    q = torch.from_numpy(wl.qpts).to(dev)
    bufs0 = _buffers(torch, wl, 6, "fp64", dev)
    ctx.eph_interp_q(6, q, *bufs0)
    qb, kt = ctx.eph_autotune(6, q)
    assert 1 <= qb <= 6 and 0 <= kt < nk
    bufs1 = _buffers(torch, wl, 6, "fp64", dev)
    ctx.eph_interp_q(6, q, *bufs1)
    torch.cuda.synchronize()
    for a, b in zip(bufs0, bufs1):
        assert np.allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=0, atol=1e-13)
    # second context of the same shape reuses the cached choice
    ctx2 = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
    ctx2.eph_set_k(nk, torch.from_numpy(wl.kpts).to(dev))
    assert ctx2.eph_autotune(6, q) == (qb, kt)
    assert ctx2.tuning()["source"] == "process cache"
    assert ctx2.tuning() == dict(ctx.tuning(), source="process cache")
    # and the results still match the oracle
    ref = oracle.interpolate(wl)
    assert gauge.max_rel_S(bufs1[2].cpu().numpy(), ref[3], ref[0], ref[1], ref[2]) <= 1e-12


def _multi_materials():
    box = (synth.centred_range(6), synth.centred_range(6), range(0, 1))
    return [(synth.make_workload("si_tiny", nk=150, nq=9), 5),
            (synth.make_workload("mos2", nk=120, nq=9, box=box), 9),
            (synth.make_workload("si_tiny", nb=3, na=1, nk=64, nq=9), 2)]


def test_multi_material_persistent_call_matches_separate_calls():
    # eph_interp_q_multi: three materials (nb 8/11/3, nm 6/9/3) with uneven q batches, their band
    # rotations as one persistent launch per round; bit-identical to separate eph_interp_q calls,
    # and on the oracle for every material
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()
    ctxs, qs, outs, refs = [], [], [], []
    for wl, nq in _multi_materials():
        c = binding.Context.from_workload(wl, device_ptrs=True, stream=st, q_batch=4, k_tile=48)
        c.eph_set_k(len(wl.kpts), torch.from_numpy(wl.kpts).to(dev))
        q = torch.from_numpy(wl.qpts[:nq].copy()).to(dev)
        ctxs.append(c)
        qs.append(q)
        outs.append(_buffers(torch, wl, nq, "fp64", dev))
        # the persistent kernel is the FP64 DFMA rotation: compare with separate calls that use it
        r = binding.Context.from_workload(wl, q_batch=4, k_tile=48, band_alu=True)
        r.set_k(wl.kpts)
        refs.append(r.interp_q(wl.qpts[:nq]))
    binding.interp_q_multi(ctxs, [q.shape[0] for q in qs], qs, [o[0] for o in outs], [o[1] for o in outs],
                           [o[2] for o in outs])
    torch.cuda.synchronize()
    for (wl, nq), o, r in zip(_multi_materials(), outs, refs):
        for a, b in zip(o, r):
            assert np.array_equal(a.cpu().numpy(), b)
        ref = oracle.interpolate(wl, wl.kpts, wl.qpts[:nq])
        assert gauge.max_rel_S(o[2].cpu().numpy(), ref[3], ref[0], ref[1], ref[2]) <= 1e-12


def test_multi_material_call_in_a_graph_and_errors():
    torch = pytest.importorskip("torch")
    from paper_2603_10295_gb300.batching import GraphBatcher
    dev = torch.device("cuda:0")
    gb = GraphBatcher(dev)
    ctxs, qs, outs, eager = [], [], [], []
    for wl, nq in _multi_materials():
        c = binding.Context.from_workload(wl, device_ptrs=True, async_mode=True, stream=gb.stream, q_batch=4)
        with torch.cuda.stream(gb.stream):
            c.eph_set_k(len(wl.kpts), torch.from_numpy(wl.kpts).to(dev))
        ctxs.append(c)
        qs.append(torch.from_numpy(wl.qpts[:nq].copy()).to(dev))
        outs.append(_buffers(torch, wl, nq, "fp64", dev))
        r = binding.Context.from_workload(wl, q_batch=4, band_alu=True)
        r.set_k(wl.kpts)
        eager.append(r.interp_q(wl.qpts[:nq]))
    gb.add_multi(ctxs, qs, [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    gb.capture()
    for o in outs:
        o[2].zero_()
    gb.replay()
    gb.check()
    for o, r in zip(outs, eager):
        for a, b in zip(o, r):
            assert np.array_equal(a.cpu().numpy(), b)
    # contexts the persistent rotation does not cover are rejected on the first context
    wl = synth.make_workload("si_tiny", nk=8, nq=2)
    m = binding.Context.from_workload(wl, form="mixed", device_ptrs=True)
    m.eph_set_k(8, torch.from_numpy(wl.kpts).to(dev))
    q = torch.from_numpy(wl.qpts).to(dev)
    with pytest.raises(binding.EphError) as ei:
        binding.interp_q_multi([ctxs[0], m], [2, 2], [q, q])
    assert ei.value.code == binding.EPH_ENOTSUP
    with pytest.raises(binding.EphError) as ei:
        binding.interp_q_multi([ctxs[0], ctxs[0]], [2, 2], [q, q])
    assert ei.value.code == binding.EPH_EINVAL


def test_autotune_file_round_trip(tmp_path):
    # a timed choice (decomposition and kernel variants) goes to the tuning file; after the file
    # is set again (the process cache cleared), a new context of the same shape takes it from there
    import torch
    dev = torch.device("cuda:0")
    wl = synth.make_workload("si_tiny", nk=96, nq=6)
    f = tmp_path / "tune.txt"
    assert binding.tune_file(f) == 0
    try:
        ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
        ctx.eph_set_k(len(wl.kpts), torch.from_numpy(wl.kpts).to(dev))
        q = torch.from_numpy(wl.qpts).to(dev)
        ctx.eph_autotune(6, q)
        t1 = ctx.tuning()
        assert t1["source"] == "timed"
        assert len(f.read_text().splitlines()) == 1
        assert binding.tune_file(f) == 1
        ctx2 = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
        ctx2.eph_set_k(len(wl.kpts), torch.from_numpy(wl.kpts).to(dev))
        ctx2.eph_autotune(6, q)
        assert ctx2.tuning() == dict(t1, source="file")
        # the tuned context still matches the oracle
        e = torch.empty(6, len(wl.kpts), wl.nb, dtype=torch.float64, device=dev)
        o = torch.empty(6, wl.nm, dtype=torch.float64, device=dev)
        g = torch.empty(6, len(wl.kpts), wl.nm, wl.nb, wl.nb, dtype=torch.complex128, device=dev)
        ctx2.eph_interp_q(6, q, e, o, g)
        torch.cuda.synchronize()
        ref = oracle.interpolate(wl)
        assert gauge.max_rel_S(g.cpu().numpy(), ref[3], ref[0], ref[1], ref[2]) <= 1e-12
    finally:
        binding.tune_file(None)
