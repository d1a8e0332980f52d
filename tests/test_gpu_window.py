"""Energy-window prescreening (eph_set_k_window, eph_interp_q_window).

Kept indices and pair masks are integers decided by floating point: the windows
are placed in gaps of the oracle's spectra (far from every eigenvalue compared
with the 1e-12 agreement of the two sides), so both decide the same and the
results are compared exactly.  After screening, the interpolation of the kept
points is bit for bit what the same points give as a plain k list.
"""
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


def gap_window(values, lo_pct, hi_pct, min_gap=1e-6):
    """[lo, hi] with both edges at midpoints of gaps (> min_gap) between sorted values."""
    v = np.unique(np.sort(np.asarray(values).ravel()))
    mids = 0.5 * (v[1:] + v[:-1])
    ok = np.diff(v) > min_gap
    cand = mids[ok]
    lo = cand[np.searchsorted(cand, np.percentile(v, lo_pct))]
    hi = cand[np.searchsorted(cand, np.percentile(v, hi_pct))]
    return float(lo), float(hi)


def test_set_k_window_keeps_exact_indices():
    wl = synth.make_workload("si_tiny", nk=300, nq=4)
    eps_full = oracle.interpolate(wl, wl.kpts, wl.qpts[:1])[0]
    lo, hi = gap_window(eps_full, 40, 48)
    expect = np.nonzero(((eps_full >= lo) & (eps_full <= hi)).any(axis=1))[0]
    assert 0 < len(expect) < len(wl.kpts)
    ctx = binding.Context.from_workload(wl)
    kidx, eps_k = ctx.set_k_window(wl.kpts, lo, hi)
    assert np.array_equal(kidx, expect.astype(np.int32))
    assert np.abs(eps_k - eps_full[expect]).max() <= 1e-12 * np.abs(eps_full).max()
    # the screened context interpolates the kept points exactly as a plain list of them
    got = ctx.interp_q(wl.qpts)
    ref_ctx = binding.Context.from_workload(wl)
    ref_ctx.set_k(wl.kpts[expect])
    ref = ref_ctx.interp_q(wl.qpts)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_empty_window():
    wl = synth.make_workload("si_tiny", nk=20, nq=2)
    ctx = binding.Context.from_workload(wl)
    kidx, eps_k = ctx.set_k_window(wl.kpts, 1e6, 2e6)
    assert len(kidx) == 0
    with pytest.raises(binding.EphError) as ei:
        ctx.interp_q(wl.qpts)
    assert ei.value.code == binding.EPH_ESTATE


@pytest.mark.parametrize("q_batch,k_tile", [(0, 0), (3, 16)])
def test_pair_screening(q_batch, k_tile):
    wl = synth.make_workload("si_tiny", nk=80, nq=7)
    ref = oracle.interpolate(wl)
    lo, hi = gap_window(np.concatenate([ref[0].ravel(), ref[1].ravel()]), 30, 36)
    expect = ((ref[1] >= lo) & (ref[1] <= hi)).any(axis=2).astype(np.int32)   # [nq][nk]
    assert 0 < expect.sum() < expect.size
    ctx = binding.Context.from_workload(wl, q_batch=q_batch, k_tile=k_tile)
    ctx.set_k(wl.kpts)
    e_kq, om, g, keep = ctx.interp_q_window(wl.qpts, lo, hi)
    assert np.array_equal(keep, expect)
    full = binding.Context.from_workload(wl, q_batch=q_batch, k_tile=k_tile)
    full.set_k(wl.kpts)
    e_f, om_f, g_f = full.interp_q(wl.qpts)
    assert np.array_equal(e_kq, e_f) and np.array_equal(om, om_f)
    m = keep.astype(bool)
    assert np.array_equal(g[m], g_f[m])
    assert not np.any(g[~m])


def test_window_errors():
    wl = synth.make_workload("si_tiny", nk=6, nq=2)
    ctx = binding.Context.from_workload(wl)
    with pytest.raises(binding.EphError) as ei:
        ctx.set_k_window(wl.kpts, 1.0, 0.0)
    assert ei.value.code == binding.EPH_EINVAL
    mixed = binding.Context.from_workload(wl, form="mixed")
    mixed.set_k(wl.kpts)
    with pytest.raises(binding.EphError) as ei:
        mixed.interp_q_window(wl.qpts, -1.0, 1.0)
    assert ei.value.code == binding.EPH_ENOTSUP
