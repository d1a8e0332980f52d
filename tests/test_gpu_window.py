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


@pytest.mark.parametrize("grid", [False, True])
def test_pair_screening_mixed_form(grid):
    # the mixed form: tensor-core k-list path (grid False) or the sum-factorised grid path; the
    # screened pairs skip the double-float band rotation.  The mask is decided on FP64 eps_{k+q}
    # that agree with the oracle to 1e-10 (windows sit in gaps wider than that)
    wl = synth.make_workload("si_tiny", nk=60, nq=5)
    kpts = synth.uniform_grid(3, 4, 5) if grid else wl.kpts
    ref = oracle.interpolate(wl, kpts, wl.qpts)
    lo, hi = gap_window(np.concatenate([ref[0].ravel(), ref[1].ravel()]), 30, 36, min_gap=1e-8)
    expect = ((ref[1] >= lo) & (ref[1] <= hi)).any(axis=2).astype(np.int32)
    assert 0 < expect.sum() < expect.size
    ctx = binding.Context.from_workload(wl, form="mixed", q_batch=2)
    full = binding.Context.from_workload(wl, form="mixed", q_batch=2)
    if grid:
        ctx.set_k_grid(3, 4, 5)
        full.set_k_grid(3, 4, 5)
    else:
        ctx.set_k(kpts)
        full.set_k(kpts)
    e_kq, om, g, keep = ctx.interp_q_window(wl.qpts, lo, hi)
    assert g.dtype == np.complex64
    assert np.array_equal(keep, expect)
    e_f, om_f, g_f = full.interp_q(wl.qpts)
    assert np.array_equal(e_kq, e_f) and np.array_equal(om, om_f)
    m = keep.astype(bool)
    assert np.array_equal(g[m], g_f[m])
    assert not np.any(g[~m])


@pytest.mark.parametrize("n,shift", [((4, 4, 4), None), ((6, 4, 2), (0.5 / 6, 0.0, 0.25)), ((5, 3, 1), None)])
def test_time_reversal_ibz_bit_exact(n, shift):
    # kept grid indices and weights are index arithmetic: equal to the oracle's brute-force
    # reduction; eps_k of the kept points equal eph_set_k on those points bit for bit
    wl = synth.make_workload("si_tiny", nb=6, nq=3, real_h=True)
    sh = (0.0, 0.0, 0.0) if shift is None else shift
    idx_ref, w_ref = oracle.ibz_time_reversal(n, sh)
    ctx = binding.Context.from_workload(wl)
    kidx, wk, eps = ctx.set_k_grid_ibz(*n, shift=shift)
    assert np.array_equal(kidx, idx_ref.astype(np.int32)) and np.array_equal(wk, w_ref)
    pts = oracle.grid_points(n, sh)[idx_ref]
    ref = binding.Context.from_workload(wl)
    assert np.array_equal(eps, ref.set_k(pts))
    # a weighted k-sum over the kept points equals the sum over the whole grid
    full = binding.Context.from_workload(wl).set_k_grid(*n, shift=shift)
    f = lambda e: 1.0 / (np.exp((e - 0.2) / 0.05) + 1.0)
    assert abs((wk[:, None] * f(eps)).sum() - f(full).sum()) <= 1e-12 * f(full).sum()
    # the resident list is the kept points: the interpolation matches the oracle there
    ge = ctx.interp_q(wl.qpts)
    from tests import gauge
    r = oracle.interpolate(wl, pts, wl.qpts)
    assert gauge.max_rel_S(ge[2], r[3], r[0], r[1], r[2]) <= 1e-12


def test_time_reversal_ibz_device_mode_and_errors():
    torch = pytest.importorskip("torch")
    wl = synth.make_workload("si_tiny", nb=4, nq=2, real_h=True)
    dev = torch.device("cuda:0")
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=torch.cuda.current_stream())
    n = (4, 6, 2)
    N = 48
    kidx = torch.empty(N, dtype=torch.int32, device=dev)
    wk = torch.empty(N, dtype=torch.float64, device=dev)
    eps = torch.empty(N, wl.nb, dtype=torch.float64, device=dev)
    cnt = ctx.eph_set_k_grid_ibz(*n, None, eps, kidx, wk)
    torch.cuda.synchronize()
    idx_ref, w_ref = oracle.ibz_time_reversal(n)
    assert cnt == len(idx_ref)
    assert np.array_equal(kidx[:cnt].cpu().numpy(), idx_ref) and np.array_equal(wk[:cnt].cpu().numpy(), w_ref)
    host = binding.Context.from_workload(wl)
    with pytest.raises(binding.EphError) as ei:
        host.set_k_grid_ibz(4, 4, 4, shift=(0.1, 0.0, 0.0))    # -k off the grid
    assert ei.value.code == binding.EPH_EINVAL


def test_window_errors():
    wl = synth.make_workload("si_tiny", nk=6, nq=2)
    ctx = binding.Context.from_workload(wl)
    with pytest.raises(binding.EphError) as ei:
        ctx.set_k_window(wl.kpts, 1.0, 0.0)
    assert ei.value.code == binding.EPH_EINVAL
    with pytest.raises(binding.EphError) as ei:
        ctx.interp_q_window(wl.qpts, -1.0, 1.0)   # before eph_set_k
    assert ei.value.code == binding.EPH_ESTATE


@pytest.mark.parametrize("form,nb,na", [("fp64", 20, 2), ("fp64", 8, 7), ("mixed", 20, 2)])
def test_pair_screening_large_shapes(form, nb, na):
    # nb or nm > 16: every pair is rotated (GEMMs, or the mixed form's tensor-core products) and
    # the screened ones are zeroed afterwards; eps_kq, omega and the kept g match the unscreened call
    wl = synth.make_workload("si_tiny", nb=nb, na=na, nk=24, nq=4)
    ref = oracle.interpolate(wl)
    lo, hi = gap_window(np.concatenate([ref[0].ravel(), ref[1].ravel()]), 30, 32, min_gap=1e-8)
    expect = ((ref[1] >= lo) & (ref[1] <= hi)).any(axis=2).astype(np.int32)
    assert 0 < expect.sum() < expect.size
    ctx = binding.Context.from_workload(wl, form=form, q_batch=3, k_tile=10)
    ctx.set_k(wl.kpts)
    e_kq, om, g, keep = ctx.interp_q_window(wl.qpts, lo, hi)
    assert np.array_equal(keep, expect)
    full = binding.Context.from_workload(wl, form=form, q_batch=3, k_tile=10)
    full.set_k(wl.kpts)
    e_f, om_f, g_f = full.interp_q(wl.qpts)
    assert np.array_equal(e_kq, e_f) and np.array_equal(om, om_f)
    m = keep.astype(bool)
    assert np.array_equal(g[m], g_f[m])
    assert not np.any(g[~m])
