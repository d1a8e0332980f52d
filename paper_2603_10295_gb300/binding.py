"""ctypes binding of libeph (argument marshalling only).

The names follow the C-ABI in include/eph.h: eph_create, eph_set_k,
eph_interp_q, eph_interp, eph_interp_backward, eph_destroy.  Every step of the
computation runs in the library's CUDA kernels; this module only converts
numpy arrays / torch tensors to pointers.  If the shared library is missing,
loading fails loudly: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libeph.so")

EPH_OK, EPH_EINVAL, EPH_ENOMEM, EPH_ECUDA, EPH_ENOTCONV, EPH_ESTATE, EPH_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
FORMS = {"fp64": 0, "mixed": 1}

#: every symbol declared in include/eph.h
EXPORTS = ("eph_default_options", "eph_create", "eph_set_k", "eph_interp_q", "eph_interp",
           "eph_interp_backward", "eph_destroy", "eph_strerror", "eph_last_error", "eph_kernel_launches",
           "eph_profile", "eph_profile_read", "eph_profile_reset", "eph_bands_noalloc",
           "eph_reserve", "eph_sync", "eph_autotune", "eph_linewidths", "eph_interp_vjp",
           "eph_set_k_grid", "eph_bloch_to_wannier", "eph_set_k_window", "eph_interp_q_window", "eph_eigh",
           "eph_create_rp_slice", "eph_g1_partial", "eph_interp_q_g1", "eph_set_gw", "eph_set_k_grid_ibz",
           "eph_interp_q_multi", "eph_tune_file", "eph_tuning")
NOALLOC_SCRATCH_BYTES = 32 << 20
STAGES = ("phase", "ft_q", "eig", "mode", "ft_k", "band", "adj", "tc")


class EphOptions(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("device_ptrs", ctypes.c_int), ("q_batch", ctypes.c_int),
                ("k_tile", ctypes.c_int), ("max_sweeps", ctypes.c_int), ("workspace_mb", ctypes.c_int),
                ("mixed_scheme", ctypes.c_int), ("eig_plain_fp64", ctypes.c_int), ("async_", ctypes.c_int),
                ("band_alu", ctypes.c_int),
                ("gemm_alu", ctypes.c_int)]


class TuningInfo(ctypes.Structure):
    """eph_tuning_info of include/eph.h."""
    _fields_ = [("q_batch", ctypes.c_int), ("k_tile", ctypes.c_int), ("band_alu", ctypes.c_int),
                ("gemm_alu", ctypes.c_int), ("source", ctypes.c_int)]


def tune_file(path):
    """eph_tune_file: the process's tuning file (None: none); returns the number of entries read."""
    lib = load_library()
    rc = lib.eph_tune_file(None if path is None else str(path).encode())
    if rc < 0:
        raise EphError(rc, "eph_tune_file: malformed tuning file")
    return rc


class EphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libeph error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Loads libeph.so (raises if it has not been built: no fallback exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libeph is not built ({p} missing); run `python -m paper_2603_10295_gb300.build_lib`")
    lib = ctypes.CDLL(p)
    vp, ip, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.eph_default_options.argtypes = [ctypes.POINTER(EphOptions)]
    lib.eph_default_options.restype = None
    lib.eph_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, dp, dp, dp, vp, dp, vp, dp, dp,
                               ctypes.POINTER(EphOptions), vp]
    lib.eph_create.restype = i
    lib.eph_set_k.argtypes = [vp, i, dp, dp]
    lib.eph_set_k.restype = i
    lib.eph_interp_q.argtypes = [vp, i, dp, dp, dp, vp]
    lib.eph_interp_q.restype = i
    lib.eph_interp.argtypes = [vp, i, dp, i, dp, dp, dp, dp, vp]
    lib.eph_interp.restype = i
    lib.eph_interp_backward.argtypes = [vp, i, dp, i, dp, dp, d, dp, dp]
    lib.eph_interp_backward.restype = i
    lib.eph_destroy.argtypes = [vp]
    lib.eph_destroy.restype = None
    lib.eph_strerror.argtypes = [i]
    lib.eph_strerror.restype = ctypes.c_char_p
    lib.eph_last_error.argtypes = [vp]
    lib.eph_last_error.restype = ctypes.c_char_p
    lib.eph_kernel_launches.argtypes = [vp]
    lib.eph_kernel_launches.restype = ctypes.c_longlong
    lib.eph_profile.argtypes = [vp, i]
    lib.eph_profile.restype = i
    lib.eph_profile_read.argtypes = [vp, i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    lib.eph_profile_read.restype = i
    lib.eph_profile_reset.argtypes = [vp]
    lib.eph_profile_reset.restype = i
    lib.eph_bands_noalloc.argtypes = [i, dp, i, i, vp, dp, dp, dp, dp, i, vp]
    lib.eph_bands_noalloc.restype = i
    lib.eph_reserve.argtypes = [vp, i]
    lib.eph_reserve.restype = i
    lib.eph_sync.argtypes = [vp]
    lib.eph_sync.restype = i
    lib.eph_autotune.argtypes = [vp, i, dp, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.eph_autotune.restype = i
    lib.eph_tune_file.argtypes = [ctypes.c_char_p]
    lib.eph_tune_file.restype = i
    lib.eph_tuning.argtypes = [vp, ctypes.POINTER(TuningInfo)]
    lib.eph_tuning.restype = i
    lib.eph_linewidths.argtypes = [vp, i, dp, dp, d, d, d, d, dp]
    lib.eph_linewidths.restype = i
    lib.eph_interp_vjp.argtypes = [vp, i, dp, i, dp, vp, dp]
    lib.eph_interp_vjp.restype = i
    lib.eph_set_k_grid.argtypes = [vp, i, i, i, dp, dp]
    lib.eph_set_k_grid.restype = i
    lib.eph_bloch_to_wannier.argtypes = [vp, i, dp, i, dp, vp, dp]
    lib.eph_bloch_to_wannier.restype = i
    lib.eph_set_k_window.argtypes = [vp, i, dp, d, d, dp, vp, ctypes.POINTER(i)]
    lib.eph_set_k_window.restype = i
    lib.eph_interp_q_window.argtypes = [vp, i, dp, d, d, dp, dp, vp, vp]
    lib.eph_interp_q_window.restype = i
    lib.eph_eigh.argtypes = [vp, i, i, vp, dp, vp]
    lib.eph_eigh.restype = i
    lib.eph_create_rp_slice.argtypes = [ctypes.POINTER(vp), i, i, i, i, dp, dp, dp, vp, dp, vp, dp, dp, i, i,
                                        ctypes.POINTER(EphOptions), vp]
    lib.eph_create_rp_slice.restype = i
    lib.eph_g1_partial.argtypes = [vp, i, dp, dp]
    lib.eph_g1_partial.restype = i
    lib.eph_interp_q_g1.argtypes = [vp, i, dp, dp, dp, dp, vp]
    lib.eph_interp_q_g1.restype = i
    lib.eph_set_gw.argtypes = [vp, dp]
    lib.eph_set_gw.restype = i
    lib.eph_set_k_grid_ibz.argtypes = [vp, i, i, i, dp, dp, vp, dp, ctypes.POINTER(i)]
    lib.eph_set_k_grid_ibz.restype = i
    lib.eph_interp_q_multi.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(i), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.eph_interp_q_multi.restype = i
    del ip
    if path is None:
        _lib = lib
    return lib


def _ptr(x):
    """Pointer of a contiguous numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libeph must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to libeph must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _points(x, name):
    """A (n, 3) C-contiguous float64 copy (or view) of a list of points in crystal coordinates."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError(f"{name} must have shape (n, 3), got {a.shape}")
    return a


def _shaped(x, shape, dtype, name):
    """A C-contiguous array of exactly `shape` (host-mode inputs whose size the library assumes)."""
    a = np.ascontiguousarray(x, dtype=dtype)
    if a.shape != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {a.shape}")
    return a


class Context:
    """One eph_ctx: Wannier data resident on the current CUDA device.

    host mode (device_ptrs=False): k/q lists and outputs are numpy arrays;
    device mode (device_ptrs=True): they are CUDA torch tensors (or raw device
    pointers as ints) and calls are ordered on `stream`.
    """

    def __init__(self, nb, na, H_Re, Phi_Rp, g_ReRp, Re, Rp, masses, we=None, wp=None, form="fp64",
                 device_ptrs=False, q_batch=0, k_tile=0, max_sweeps=0, workspace_mb=0, stream=None,
                 mixed_scheme="digits", eig_plain_fp64=False, async_mode=False, rp_slice=None,
                 band_alu=False, gemm_alu=False):
        """rp_slice = (rp_begin, rp_count): g_ReRp holds only those Rp rows (eph_create_rp_slice)."""
        self.lib = load_library()
        self.nb, self.na, self.nm = int(nb), int(na), 3 * int(na)
        H_Re = np.ascontiguousarray(H_Re, dtype=np.complex128)
        Phi_Rp = np.ascontiguousarray(Phi_Rp, dtype=np.float64)
        g_ReRp = np.ascontiguousarray(g_ReRp, dtype=np.complex128)
        Re = np.ascontiguousarray(Re, dtype=np.int32)
        Rp = np.ascontiguousarray(Rp, dtype=np.int32)
        masses = np.ascontiguousarray(masses, dtype=np.float64)
        we = None if we is None else np.ascontiguousarray(we, dtype=np.float64)
        wp = None if wp is None else np.ascontiguousarray(wp, dtype=np.float64)
        self.ne, self.np_ = len(Re), len(Rp)
        self.form = form
        self.device_ptrs = bool(device_ptrs)
        self.async_mode = bool(async_mode)
        opt = EphOptions()
        self.lib.eph_default_options(ctypes.byref(opt))
        opt.form = FORMS[form]
        opt.device_ptrs = int(device_ptrs)
        opt.q_batch, opt.k_tile, opt.max_sweeps, opt.workspace_mb = q_batch, k_tile, max_sweeps, workspace_mb
        opt.mixed_scheme = {"digits": 0, "tf32": 1}[mixed_scheme]
        opt.eig_plain_fp64 = int(bool(eig_plain_fp64))
        opt.async_ = int(bool(async_mode))
        opt.band_alu = int(bool(band_alu))
        opt.gemm_alu = int(bool(gemm_alu))
        handle = ctypes.c_void_p()
        st = None
        if stream is not None:
            st = stream if isinstance(stream, int) else int(stream.cuda_stream)
        self.rp_slice = (0, self.np_) if rp_slice is None else (int(rp_slice[0]), int(rp_slice[1]))
        if rp_slice is None:
            rc = self.lib.eph_create(ctypes.byref(handle), self.nb, self.na, self.ne, self.np_, _ptr(H_Re),
                                     _ptr(Phi_Rp), _ptr(g_ReRp), _ptr(Re), _ptr(we), _ptr(Rp), _ptr(wp), _ptr(masses),
                                     ctypes.byref(opt), st)
        else:
            if g_ReRp.shape[0] != self.rp_slice[1]:
                raise ValueError(f"g_ReRp holds {g_ReRp.shape[0]} Rp rows, the slice {self.rp_slice[1]}")
            rc = self.lib.eph_create_rp_slice(ctypes.byref(handle), self.nb, self.na, self.ne, self.np_, _ptr(H_Re),
                                              _ptr(Phi_Rp), _ptr(g_ReRp), _ptr(Re), _ptr(we), _ptr(Rp), _ptr(wp),
                                              _ptr(masses), self.rp_slice[0], self.rp_slice[1], ctypes.byref(opt), st)
        if rc != EPH_OK:
            raise EphError(rc, self.lib.eph_strerror(rc).decode())
        self.handle = handle
        self.nk = 0

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl.nb, wl.na, wl.H_Re, wl.Phi_Rp, wl.g_ReRp, wl.Re, wl.Rp, wl.masses, wl.we, wl.wp, **kw)

    def _check(self, rc):
        if rc != EPH_OK:
            raise EphError(rc, self.lib.eph_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.eph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launches(self) -> int:
        return int(self.lib.eph_kernel_launches(self.handle))

    def profile(self, enable=True):
        self._check(self.lib.eph_profile(self.handle, int(bool(enable))))

    def profile_reset(self):
        self._check(self.lib.eph_profile_reset(self.handle))

    def profile_read(self):
        """{stage: (milliseconds, launches)} accumulated since the last reset."""
        out = {}
        for i, name in enumerate(STAGES):
            ms = ctypes.c_double()
            n = ctypes.c_longlong()
            self._check(self.lib.eph_profile_read(self.handle, i, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    # -- raw calls (buffers already allocated by the caller) -----------------
    def eph_set_k(self, nk, kpts, eps_k=None):
        self._check(self.lib.eph_set_k(self.handle, int(nk), _ptr(kpts), _ptr(eps_k)))
        self.nk = int(nk)

    def eph_set_k_grid(self, n1, n2, n3, shift=None, eps_k=None):
        sh = None if shift is None else np.ascontiguousarray(shift, dtype=np.float64)
        self._check(self.lib.eph_set_k_grid(self.handle, int(n1), int(n2), int(n3), _ptr(sh), _ptr(eps_k)))
        self.nk = int(n1) * int(n2) * int(n3)

    def eph_interp_q(self, nq, qpts, eps_kq=None, omega=None, g=None):
        self._check(self.lib.eph_interp_q(self.handle, int(nq), _ptr(qpts), _ptr(eps_kq), _ptr(omega), _ptr(g)))

    def eph_g1_partial(self, nq, qpts, G1):
        self._check(self.lib.eph_g1_partial(self.handle, int(nq), _ptr(qpts), _ptr(G1)))

    def eph_interp_q_g1(self, nq, qpts, G1, eps_kq=None, omega=None, g=None):
        self._check(self.lib.eph_interp_q_g1(self.handle, int(nq), _ptr(qpts), _ptr(G1), _ptr(eps_kq), _ptr(omega),
                                             _ptr(g)))

    def eph_set_gw(self, g_ReRp):
        self._check(self.lib.eph_set_gw(self.handle, _ptr(g_ReRp)))

    def g1_partial(self, qpts):
        """Eq. 9 over this context's Rp slice: G1 [nq][nm][ne][nb][nb] (host mode)."""
        qpts = _points(qpts, "qpts")
        G1 = np.empty((len(qpts), self.nm, self.ne, self.nb, self.nb), dtype=np.complex128)
        self.eph_g1_partial(len(qpts), qpts, G1)
        return G1

    def interp_q_g1(self, qpts, G1, want_g=True):
        """eph_interp_q with a given G1 (host mode): (eps_kq, omega, g)."""
        qpts = _points(qpts, "qpts")
        nq = len(qpts)
        G1 = _shaped(G1, (nq, self.nm, self.ne, self.nb, self.nb), np.complex128, "G1")
        eps_kq = np.empty((nq, self.nk, self.nb))
        omega = np.empty((nq, self.nm))
        g = None
        if want_g:
            dt = np.complex128 if self.form == "fp64" else np.complex64
            g = np.empty((nq, self.nk, self.nm, self.nb, self.nb), dtype=dt)
        self.eph_interp_q_g1(nq, qpts, G1, eps_kq, omega, g)
        return eps_kq, omega, g

    def eph_reserve(self, nq):
        self._check(self.lib.eph_reserve(self.handle, int(nq)))

    def eph_sync(self):
        self._check(self.lib.eph_sync(self.handle))

    def eph_autotune(self, nq, qpts):
        qb, kt = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.eph_autotune(self.handle, int(nq), _ptr(qpts), ctypes.byref(qb), ctypes.byref(kt)))
        return qb.value, kt.value

    def tuning(self):
        """The context's (q_batch, k_tile, band_alu, gemm_alu) and their source (eph_tuning)."""
        t = TuningInfo()
        self._check(self.lib.eph_tuning(self.handle, ctypes.byref(t)))
        return {"q_batch": t.q_batch, "k_tile": t.k_tile, "band_alu": t.band_alu, "gemm_alu": t.gemm_alu,
                "source": ("none", "timed", "process cache", "file")[t.source]}

    def eph_interp_vjp(self, nk, kpts, nq, qpts, grad_g, grad_g_ReRp):
        self._check(self.lib.eph_interp_vjp(self.handle, int(nk), _ptr(kpts), int(nq), _ptr(qpts), _ptr(grad_g),
                                            _ptr(grad_g_ReRp)))

    def vjp(self, kpts, qpts, grad_g):
        """dL/dg(Re,Rp) for an upstream gradient grad_g [nq][nk][nm][nb][nb] (complex128).
        kpts = None: the resident k list (a uniform grid runs sum-factorised)."""
        kpts, nk = (None, self.nk) if kpts is None else (_points(kpts, "kpts"), len(kpts))
        qpts = _points(qpts, "qpts")
        grad_g = _shaped(grad_g, (len(qpts), nk, self.nm, self.nb, self.nb), np.complex128, "grad_g")
        out = np.empty((self.np_, self.nm, self.ne, self.nb, self.nb), dtype=np.complex128)
        self.eph_interp_vjp(nk, kpts, len(qpts), qpts, grad_g, out)
        self.nk = nk   # the call replaces the context's k list
        return out

    def eph_bloch_to_wannier(self, nk, kpts, nq, qpts, g, g_ReRp):
        self._check(self.lib.eph_bloch_to_wannier(self.handle, int(nk), _ptr(kpts), int(nq), _ptr(qpts), _ptr(g),
                                                  _ptr(g_ReRp)))

    def bloch_to_wannier(self, kpts, qpts, g):
        """Eq. 6: g(Re,Rp) [np][nm][ne][nb][nb] from g(k',q') [nq][nk][nm][nb][nb] on coarse grids.
        kpts = None: the resident k list (e.g. the coarse grid of set_k_grid)."""
        kpts, nk = (None, self.nk) if kpts is None else (_points(kpts, "kpts"), len(kpts))
        qpts = _points(qpts, "qpts")
        g = _shaped(g, (len(qpts), nk, self.nm, self.nb, self.nb), np.complex128, "g")
        out = np.empty((self.np_, self.nm, self.ne, self.nb, self.nb), dtype=np.complex128)
        self.eph_bloch_to_wannier(nk, kpts, len(qpts), qpts, g, out)
        self.nk = nk   # the call replaces the context's k list
        return out

    def eph_set_k_window(self, nk, kpts, e_lo, e_hi, eps_k, kidx):
        n = ctypes.c_int(0)
        self._check(self.lib.eph_set_k_window(self.handle, int(nk), _ptr(kpts), float(e_lo), float(e_hi), _ptr(eps_k),
                                              _ptr(kidx), ctypes.byref(n)))
        self.nk = n.value
        return n.value

    def eph_set_k_grid_ibz(self, n1, n2, n3, shift, eps_k, kidx, wk):
        n = ctypes.c_int(0)
        sh = None if shift is None else np.ascontiguousarray(shift, dtype=np.float64)
        self._check(self.lib.eph_set_k_grid_ibz(self.handle, int(n1), int(n2), int(n3), _ptr(sh), _ptr(eps_k),
                                                _ptr(kidx), _ptr(wk), ctypes.byref(n)))
        self.nk = n.value
        return n.value

    def set_k_grid_ibz(self, n1, n2, n3, shift=None):
        """Time-reversal irreducible half of a uniform grid: (kept grid indices, weights, eps_k)."""
        nk = int(n1) * int(n2) * int(n3)
        kidx = np.empty(nk, dtype=np.int32)
        wk = np.empty(nk)
        eps = np.empty((nk, self.nb))
        n = self.eph_set_k_grid_ibz(n1, n2, n3, shift, eps, kidx, wk)
        return kidx[:n].copy(), wk[:n].copy(), eps[:n].copy()

    def set_k_window(self, kpts, e_lo, e_hi):
        """Keeps the k points with a band in [e_lo, e_hi]: (kept indices, their eps_k)."""
        kpts = _points(kpts, "kpts")
        kidx = np.empty(len(kpts), dtype=np.int32)
        eps = np.empty((len(kpts), self.nb))
        n = self.eph_set_k_window(len(kpts), kpts, e_lo, e_hi, eps, kidx)
        return kidx[:n].copy(), eps[:n].copy()

    def eph_interp_q_window(self, nq, qpts, e_lo, e_hi, eps_kq=None, omega=None, g=None, keep=None):
        self._check(self.lib.eph_interp_q_window(self.handle, int(nq), _ptr(qpts), float(e_lo), float(e_hi),
                                                 _ptr(eps_kq), _ptr(omega), _ptr(g), _ptr(keep)))

    def interp_q_window(self, qpts, e_lo, e_hi):
        """(eps_kq, omega, g, keep) with g = 0 on the pairs screened out by the window."""
        qpts = _points(qpts, "qpts")
        nq = len(qpts)
        eps_kq = np.empty((nq, self.nk, self.nb))
        omega = np.empty((nq, self.nm))
        dt = np.complex128 if self.form == "fp64" else np.complex64
        g = np.empty((nq, self.nk, self.nm, self.nb, self.nb), dtype=dt)
        keep = np.empty((nq, self.nk), dtype=np.int32)
        self.eph_interp_q_window(nq, qpts, e_lo, e_hi, eps_kq, omega, g, keep)
        return eps_kq, omega, g, keep

    def eph_linewidths(self, nq, qpts, wq, kT, mu, sigma, omega_min, gamma):
        self._check(self.lib.eph_linewidths(self.handle, int(nq), _ptr(qpts), _ptr(wq), float(kT), float(mu),
                                            float(sigma), float(omega_min), _ptr(gamma)))

    def eph_eigh(self, n, batch, A, w, V):
        self._check(self.lib.eph_eigh(self.handle, int(n), int(batch), _ptr(A), _ptr(w), _ptr(V)))

    def eigh(self, A):
        """Batched Hermitian eigendecomposition of A [batch][n][n] (host mode): (w, V), ascending."""
        A = np.ascontiguousarray(A, dtype=np.complex128)
        if A.ndim != 3 or A.shape[1] != A.shape[2]:
            raise ValueError(f"A must have shape (batch, n, n), got {A.shape}")
        batch, n = A.shape[0], A.shape[1]
        w = np.empty((batch, n))
        V = np.empty((batch, n, n), dtype=np.complex128)
        self.eph_eigh(n, batch, A, w, V)
        return w, V

    def linewidths(self, qpts, wq=None, kT=0.025852, mu=0.0, sigma=0.05, omega_min=1e-6):
        qpts = _points(qpts, "qpts")
        wq = None if wq is None else _shaped(wq, (len(qpts),), np.float64, "wq")
        gamma = np.empty((self.nk, self.nb))
        self.eph_linewidths(len(qpts), qpts, wq, kT, mu, sigma, omega_min, gamma)
        return gamma

    def eph_interp_backward(self, nk, kpts, nq, qpts, w_nk, omega_min, L_out, grad):
        self._check(self.lib.eph_interp_backward(self.handle, int(nk), _ptr(kpts), int(nq), _ptr(qpts), _ptr(w_nk),
                                                 float(omega_min), _ptr(L_out), _ptr(grad)))

    # -- host-mode conveniences (numpy in, numpy out) ----------------------
    def set_k(self, kpts):
        kpts = _points(kpts, "kpts")
        eps_k = np.empty((len(kpts), self.nb))
        self.eph_set_k(len(kpts), kpts, eps_k)
        return eps_k

    def set_k_grid(self, n1, n2, n3, shift=None):
        eps_k = np.empty((int(n1) * int(n2) * int(n3), self.nb))
        self.eph_set_k_grid(n1, n2, n3, shift, eps_k)
        return eps_k

    def interp_q(self, qpts, want_g=True):
        qpts = _points(qpts, "qpts")
        nq = len(qpts)
        eps_kq = np.empty((nq, self.nk, self.nb))
        omega = np.empty((nq, self.nm))
        g = None
        if want_g:
            dt = np.complex128 if self.form == "fp64" else np.complex64
            g = np.empty((nq, self.nk, self.nm, self.nb, self.nb), dtype=dt)
        self.eph_interp_q(nq, qpts, eps_kq, omega, g)
        return eps_kq, omega, g

    def interp(self, kpts, qpts, want_g=True):
        eps_k = self.set_k(kpts)
        eps_kq, omega, g = self.interp_q(qpts, want_g)
        return eps_k, eps_kq, omega, g

    def loss_and_grad(self, kpts, qpts, w_nk, omega_min):
        """(L, dL/dg(Re,Rp)); kpts = None: the resident k list (a uniform grid runs sum-factorised)."""
        kpts, nk = (None, self.nk) if kpts is None else (_points(kpts, "kpts"), len(kpts))
        qpts = _points(qpts, "qpts")
        w_nk = _shaped(w_nk, (nk, self.nb), np.float64, "w_nk")
        L = np.zeros(1)
        grad = np.empty((self.np_, self.nm, self.ne, self.nb, self.nb), dtype=np.complex128)
        self.eph_interp_backward(nk, kpts, len(qpts), qpts, w_nk, omega_min, L, grad)
        self.nk = nk
        return float(L[0]), grad


def interp_q_multi(ctxs, nqs, qpts, eps_kq=None, omega=None, g=None):
    """eph_interp_q_multi over device-pointer contexts: list arguments per context (entries may
    be None).  Errors are raised from the first context."""
    n = len(ctxs)
    lib = ctxs[0].lib
    vp = ctypes.c_void_p
    arr = lambda xs: (vp * n)(*[_ptr(x) for x in (xs if xs is not None else [None] * n)])
    handles = (vp * n)(*[c.handle for c in ctxs])
    nq_arr = (ctypes.c_int * n)(*[int(x) for x in nqs])
    ctxs[0]._check(lib.eph_interp_q_multi(n, handles, nq_arr, arr(qpts), arr(eps_kq), arr(omega), arr(g)))

