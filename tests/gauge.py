"""Gauge-invariant comparison helpers (test infrastructure).

Eigenvectors are fixed only up to a phase (or a unitary mixing inside a
degenerate subspace), so g itself is compared through
S_{MNV}(k,q) = sum_{m in M, n in N, nu in V} |g_mn nu(k,q)|^2 over groups of
(near-)degenerate eigenvalues: consecutive sorted values whose gap is below
tau = rel * (max - min) of that spectrum.
"""
import numpy as np


def group_onehot(vals, rel=1e-4):
    """vals [..., n] sorted ascending -> one-hot [..., n, n] (group id along last axis)."""
    vals = np.asarray(vals, dtype=np.float64)
    span = vals[..., -1:] - vals[..., :1]
    tau = rel * np.maximum(span, 1e-300)
    brk = np.diff(vals, axis=-1) > tau
    gid = np.concatenate([np.zeros(vals.shape[:-1] + (1,), dtype=np.int64), np.cumsum(brk, axis=-1)], axis=-1)
    n = vals.shape[-1]
    return (gid[..., :, None] == np.arange(n)).astype(np.float64)


def subspace_sums(g, eps_k, eps_kq, omega, rel=1e-4):
    """g [nq][nk][nm][nb][nb] -> S [nq][nk][V][M][N] with groups from the given spectra."""
    a2 = np.abs(np.asarray(g, dtype=np.complex128)) ** 2
    Om = group_onehot(eps_kq, rel)            # [nq][nk][nb][G]
    On = group_onehot(eps_k, rel)             # [nk][nb][G]
    Ov = group_onehot(omega, rel)             # [nq][nm][G]
    return np.einsum("qkvmn,qkmM,knN,qvV->qkVMN", a2, Om, On, Ov, optimize=True)


def max_rel_S(g_test, g_ref, eps_k, eps_kq, omega, rel=1e-4):
    """max over (k,q) of max|S_test - S_ref| / max S_ref at that pair (groups from the reference)."""
    St = subspace_sums(g_test, eps_k, eps_kq, omega, rel)
    Sr = subspace_sums(g_ref, eps_k, eps_kq, omega, rel)
    den = Sr.reshape(Sr.shape[0], Sr.shape[1], -1).max(-1)
    num = np.abs(St - Sr).reshape(Sr.shape[0], Sr.shape[1], -1).max(-1)
    return float((num / np.maximum(den, 1e-300)).max())


def max_rel_eps(e_test, e_ref):
    """max |d eps| / max_n |eps| per point."""
    e_ref = np.asarray(e_ref)
    den = np.abs(e_ref).max(-1, keepdims=True)
    return float((np.abs(np.asarray(e_test) - e_ref) / np.maximum(den, 1e-300)).max())


def max_rel_omega(w_test, w_ref):
    """max |d omega| / max_nu omega per q."""
    w_ref = np.asarray(w_ref)
    den = np.abs(w_ref).max(-1, keepdims=True)
    return float((np.abs(np.asarray(w_test) - w_ref) / np.maximum(den, 1e-300)).max())
