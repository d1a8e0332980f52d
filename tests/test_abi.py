"""Host-side checks of the C-ABI library: it builds, loads, exports every
symbol that include/eph.h declares, and rejects bad arguments before touching
the GPU.  No compute call is made here (no GPU on this host)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2603_10295_gb300 import binding, build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(binding.LIB_PATH):
        build_lib.build()
    return binding.load_library()


def header_functions():
    text = open(os.path.join(ROOT, "include", "eph.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eph_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_binding_exports():
    assert header_functions() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if l.strip()}
    for name in header_functions():
        assert name in syms, name
        assert hasattr(lib, name)


def test_status_strings(lib):
    for code in range(0, -7, -1):
        s = lib.eph_strerror(code)
        assert s and s != b"unknown status"
    assert lib.eph_strerror(-99) == b"unknown status"


def test_create_rejects_bad_arguments_without_gpu(lib):
    h = ctypes.c_void_p()
    opt = binding.EphOptions()
    lib.eph_default_options(ctypes.byref(opt))
    assert opt.form == 0 and opt.device_ptrs == 0
    # NULL inputs and non-positive sizes are rejected before any CUDA call
    assert lib.eph_create(ctypes.byref(h), 0, 1, 1, 1, None, None, None, None, None, None, None, None,
                          ctypes.byref(opt), None) == binding.EPH_EINVAL
    assert lib.eph_create(ctypes.byref(h), 4, 1, 1, 1, None, None, None, None, None, None, None, None,
                          ctypes.byref(opt), None) == binding.EPH_EINVAL
    assert not h.value
    assert lib.eph_set_k(None, 1, None, None) == binding.EPH_EINVAL
    assert lib.eph_interp_q(None, 1, None, None, None, None) == binding.EPH_EINVAL
    lib.eph_destroy(None)
    assert lib.eph_last_error(None) == b""


def test_product_path_has_no_fallback(tmp_path):
    with pytest.raises(RuntimeError):
        binding.load_library(str(tmp_path / "missing.so"))


def test_binding_rejects_misshaped_host_arrays():
    # the host-mode conveniences check shapes before any library call, so a (n,) point list or
    # a gradient of the wrong size never reaches the C side as an out-of-range read
    import numpy as np
    assert binding._points([[0.0, 0.5, 0.25]], "kpts").shape == (1, 3)
    assert binding._points(np.zeros((0, 3)), "kpts").shape == (0, 3)
    for bad in (np.zeros(3), np.zeros((4, 2)), np.zeros((2, 3, 1))):
        with pytest.raises(ValueError):
            binding._points(bad, "kpts")
    with pytest.raises(ValueError):
        binding._shaped(np.zeros((2, 3)), (3, 2), np.float64, "w_nk")
    ctx = object.__new__(binding.Context)   # no library handle: any C call would fail differently
    ctx.nb, ctx.nm, ctx.nk, ctx.np_, ctx.ne, ctx.form = 2, 3, 4, 5, 6, "fp64"
    with pytest.raises(ValueError):
        ctx.set_k(np.zeros(3))
    with pytest.raises(ValueError):
        ctx.interp_q(np.zeros((2, 2)))
    with pytest.raises(ValueError):
        ctx.vjp(np.zeros((4, 3)), np.zeros((2, 3)), np.zeros((2, 4, 3, 2)))
    with pytest.raises(ValueError):
        ctx.loss_and_grad(np.zeros((4, 3)), np.zeros((2, 3)), np.zeros((4, 3)), 1e-6)
    with pytest.raises(ValueError):
        ctx.linewidths(np.zeros((2, 3)), wq=np.ones(3))
    with pytest.raises(ValueError):
        ctx.eigh(np.zeros((2, 3, 4)))


def test_every_entry_point_rejects_a_null_context_without_gpu(lib):
    # a NULL context (and, for the context-free entry point, a bad size) is an argument error
    # reported before any CUDA call: these run on a host without a GPU
    E = binding.EPH_EINVAL
    i = ctypes.c_int()
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    assert lib.eph_set_k_grid(None, 2, 2, 2, None, None) == E
    assert lib.eph_set_k_window(None, 1, None, 0.0, 1.0, None, None, ctypes.byref(i)) == E
    assert lib.eph_interp(None, 1, None, 1, None, None, None, None, None) == E
    assert lib.eph_interp_q_window(None, 1, None, 0.0, 1.0, None, None, None, None) == E
    assert lib.eph_interp_backward(None, 1, None, 1, None, None, 0.0, None, None) == E
    assert lib.eph_interp_vjp(None, 1, None, 1, None, None, None) == E
    assert lib.eph_bloch_to_wannier(None, 1, None, 1, None, None, None) == E
    assert lib.eph_linewidths(None, 1, None, None, 0.025, 0.0, 0.1, 1e-6, None) == E
    assert lib.eph_eigh(None, 4, 1, None, None, None) == E
    assert lib.eph_reserve(None, 4) == E
    assert lib.eph_sync(None) == E
    assert lib.eph_autotune(None, 4, None, ctypes.byref(i), ctypes.byref(i)) == E
    assert lib.eph_tuning(None, ctypes.byref(binding.TuningInfo())) == E
    assert lib.eph_profile(None, 1) == E
    assert lib.eph_profile_read(None, 0, ctypes.byref(ms), ctypes.byref(n)) == E
    assert lib.eph_profile_reset(None) == E
    assert lib.eph_kernel_launches(None) == 0
    # the allocation-free entry point: sizes beyond its fixed scratch, nb > 16, NULL pointers
    dummy = ctypes.c_void_p(16)   # never dereferenced: every call below fails its checks first
    assert lib.eph_bands_noalloc(0, dummy, 4, 8, dummy, None, dummy, dummy, dummy, 0, None) == E
    assert lib.eph_bands_noalloc(10, dummy, 17, 8, dummy, None, dummy, dummy, dummy, 0, None) == E
    assert lib.eph_bands_noalloc(100000, dummy, 8, 216, dummy, None, dummy, dummy, dummy, 0, None) == E
    assert lib.eph_bands_noalloc(10, None, 4, 8, dummy, None, dummy, dummy, dummy, 0, None) == E
    # the Rp-partition and g(Re,Rp)-update entry points
    assert lib.eph_g1_partial(None, 1, dummy, dummy) == E
    assert lib.eph_interp_q_g1(None, 1, dummy, dummy, None, None, None) == E
    assert lib.eph_set_gw(None, dummy) == E
    assert lib.eph_interp_q_multi(0, None, None, None, None, None, None) == E
    assert lib.eph_interp_q_multi(1, None, None, None, None, None, None) == E


def test_rp_slice_bounds_checked_without_gpu(lib):
    # an Rp slice outside [0, np) is rejected before the context touches the device
    import numpy as np
    h = ctypes.c_void_p()
    opt = binding.EphOptions()
    lib.eph_default_options(ctypes.byref(opt))
    nb, na, ne, np_ = 2, 1, 3, 3
    H = np.zeros((ne, nb, nb), np.complex128)
    Phi = np.zeros((np_, 3, 3))
    g = np.zeros((np_, 3, ne, nb, nb), np.complex128)
    R = np.zeros((3, 3), np.int32)
    m = np.ones(1)
    for begin, count in ((-1, 1), (0, 0), (2, 2), (3, 1)):
        assert lib.eph_create_rp_slice(ctypes.byref(h), nb, na, ne, np_, H.ctypes.data, Phi.ctypes.data,
                                       g.ctypes.data, R.ctypes.data, None, R.ctypes.data, None, m.ctypes.data,
                                       begin, count, ctypes.byref(opt), None) == binding.EPH_EINVAL
        assert not h.value


def test_tuning_file_is_read_and_checked_without_gpu(tmp_path):
    # eph_tune_file reads the autotuner's file format on the host (no CUDA call): comments and
    # entries of any device; a malformed line rejects the file and leaves the cache empty
    binding.load_library()
    f = tmp_path / "tune.txt"
    assert binding.tune_file(f) == 0                 # absent: created by the first timed entry
    f.write_text("# libeph tuning\n"
                 "eph-tune 1 NVIDIA_GB300 152 0 0 1 8 6 216 216 64000 4 : 4 0 0 0\n"
                 "\n"
                 "eph-tune 1 Other_GPU 80 1 0 0 11 9 144 144 2304 16 : 8 1152 1 0\n")
    assert binding.tune_file(f) == 2
    for bad in ("eph-tune 2 X 1 0 0 0 1 1 1 1 1 1 : 1 0 0 0\n",          # unknown version
                "eph-tune 1 X 1 0 0 0 1 1 1 1 1 1 : 1 0 0 2\n",          # gemm_alu not 0/1
                "eph-tune 1 X 1 0 0 0 1 1 1 1 1 1 : 1 0 0 0 extra\n",    # trailing text
                "eph-tune 1 X 1 0 0 0 1 1 1 1 1 1 : 17 0 0 0\n",         # q_batch above 16
                "eph-tune 1 X 1 0 0 0 1 1 1 1 1\n"):                     # truncated
        f.write_text(bad)
        with pytest.raises(binding.EphError) as ei:
            binding.tune_file(f)
        assert ei.value.code == binding.EPH_EINVAL
    assert binding.tune_file(None) == 0
