"""Plain FP64 CPU oracle: Wannier interpolation of electron-phonon matrix elements.

TEST INFRASTRUCTURE ONLY: used by the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; the product path never imports it, and it
imports nothing from the product.

Every function follows the paper's definitions directly (numpy complex128, no
blocking or fusion beyond the equation it cites).  Library primitives used as
single steps: ``np.matmul``/``np.einsum`` (sums), ``np.linalg.eigh`` (Hermitian
eigendecomposition), ``np.linalg.inv``.

Conventions (readings of the paper where it is silent):
  * Phases: e^{i k.R} means e^{2 pi i sum_j k_j n_j} with k in crystal
    coordinates and R = (n1, n2, n3) integer lattice coordinates; the argument
    t = k.n is formed in FP64 and reduced to r = t - rint(t) before cos/sin.
    A per-R weight w_R (Wigner-Seitz degeneracy weight; 1 in all workloads)
    multiplies each phase.
  * H(k) = sum_Re w_e e^{i k.Re} H(Re) and D(q) = sum_Rp w_p e^{i q.Rp}
    Phi(Rp)/sqrt(M_kappa M_kappa') (implied by Eqs. 4-5 and the phonon
    eigenvector of Eq. 2; the paper does not print them).
  * U_{nn'k} of Eqs. 4-7 is (V_k^H)_{nn'} where V_k holds the eigenvectors of
    H(k) as columns (ascending eigenvalues), so Eq. 7 reads
    g_nu(k,q) = V_{k+q}^H [sum ...] V_k.
  * u_{kappa alpha, nu}(q) = e_{kappa alpha, nu}(q)/sqrt(M_kappa) (mass-scaled
    phonon eigenvector; no sqrt(hbar/2 omega) factor), index kappa alpha = 3 kappa + alpha.
  * omega = sign(lambda) sqrt(|lambda|) * hbar sqrt(eV/(A^2 amu)), in eV.

Pins (tests/test_oracle_pins.py; tests/test_oracle_mutations.py plants a mistake in each
function below and checks that a pin fails):
  * phases: unit modulus, R = 0, periodicity (bit-level 2^20 cells out), product rule, e^{i pi/2}.
  * hamiltonian_k, electron_eigen: one-band chain and complex-hopping chain dispersions (the
    latter fixes the sign of the phase, at k and at k+q); plane-wave case with a DFT-matrix H0.
  * dynamical_matrix, phonon_eigen: hermiticity and the three zero modes at Gamma (acoustic sum
    rule); monatomic spring chain (stable and unstable: the sign of omega); diatomic chain mode
    vectors (the sign of the phase and u = e/sqrt(M), seen through |g|); the eV unit against
    the textbook THz factor.
  * g_rp_to_q, g_req_to_bloch, interpolate: single-(Re,Rp) plane-wave closed form; Eq. 7 by
    brute force on tiny inputs; the Wannier round trip through Eq. 6; the gauge-free norm
    identity, periodicity and linearity.
  * loss_weights, loss, loss_and_grad, vjp: L in closed form on the plane-wave inputs (1/omega,
    the weight on the k-side band n, the omega_min cut); central differences (exact for a
    quadratic form), Euler's identity, the dot-product identity <vjp(gbar), dg> = <gbar, g(dg)>.
  * linewidths (with bose, fermi, gaussian): the sigma -> 0 limit on two tight-binding chain
    bands with degenerate Einstein modes and a constant coupling, against the analytic chain
    density of states; detailed balance at eps = mu (both weights equal csch(omega/kT)); the
    zero-temperature limit (emission only above mu, absorption only below); the omega_min cut,
    positivity and linearity in the q weights.
  * g_bloch_to_wannier (Eq. 6): the round trip above.
  * grid_points, ibz_time_reversal: the number of kept points (N + N_self)/2 with N_self, the
    points that are their own partner, counted axis by axis in closed form; weights summing to
    N; on real-H(Re) inputs eps(partner) = eps(k) and weighted sums over the kept points equal
    the sums over the whole grid.
"""
from __future__ import annotations

import math

import numpy as np

# CODATA 2018 exact / recommended values.
_HBAR_J_S = 1.054571817e-34
_EV_J = 1.602176634e-19
_AMU_KG = 1.66053906660e-27
_ANGSTROM_M = 1.0e-10
#: hbar * sqrt(eV / (Angstrom^2 amu)) expressed in eV (= 0.06465415... eV).
OMEGA_UNIT_EV = _HBAR_J_S * math.sqrt(_EV_J / (_ANGSTROM_M ** 2 * _AMU_KG)) / _EV_J


# ----------------------------------------------------------------------------
# Phases: the e^{i k.Re}, e^{i q.Rp} factors of Eq. 7 (Eqs. 9-10 split them).
# ----------------------------------------------------------------------------
def phases(pts: np.ndarray, R: np.ndarray, w: np.ndarray | None = None) -> np.ndarray:
    """P[i][r] = w_r exp(2 pi i pts_i . R_r), argument reduced exactly before cos/sin.

    pts: [n][3] crystal coordinates; R: [N][3] integers; returns [n][N] complex128.
    """
    pts = np.asarray(pts, dtype=np.float64)
    Rf = np.asarray(R, dtype=np.float64)
    t = pts[:, None, 0] * Rf[None, :, 0] + pts[:, None, 1] * Rf[None, :, 1] + pts[:, None, 2] * Rf[None, :, 2]
    r = t - np.rint(t)
    P = np.cos(2.0 * np.pi * r) + 1j * np.sin(2.0 * np.pi * r)
    if w is not None:
        P = P * np.asarray(w, dtype=np.float64)[None, :]
    return P


# ----------------------------------------------------------------------------
# Electron Hamiltonian and dynamical matrix (implied by Eqs. 4-5 and Eq. 2).
# ----------------------------------------------------------------------------
def hamiltonian_k(kpts, Re, we, H_Re) -> np.ndarray:
    """H(k) = sum_Re w_e e^{i k.Re} H(Re): [nk][nb][nb]."""
    P = phases(kpts, Re, we)
    ne, nb, _ = H_Re.shape
    return (P @ H_Re.reshape(ne, nb * nb)).reshape(-1, nb, nb)


def dynamical_matrix(qpts, Rp, wp, Phi_Rp, masses) -> np.ndarray:
    """D(q) = sum_Rp w_p e^{i q.Rp} Phi(Rp) / sqrt(M_kappa M_kappa'): [nq][nm][nm]."""
    P = phases(qpts, Rp, wp)
    np_, nm, _ = Phi_Rp.shape
    m = np.repeat(np.asarray(masses, dtype=np.float64), 3)
    scale = 1.0 / np.sqrt(np.outer(m, m))
    D = (P @ Phi_Rp.reshape(np_, nm * nm).astype(np.complex128)).reshape(-1, nm, nm)
    return D * scale[None]


def electron_eigen(Hk: np.ndarray):
    """Eigenvalues (ascending) and eigenvectors (columns) of each H(k) (Eqs. 4-5 gauge)."""
    eps, V = np.linalg.eigh(Hk)
    return eps, V


def phonon_eigen(Dq: np.ndarray, masses):
    """omega [nq][nm] in eV, e (columns), u = e / sqrt(M) [nq][nm][nm] (Eq. 2 mode eigenvector)."""
    lam, e = np.linalg.eigh(Dq)
    omega = np.sign(lam) * np.sqrt(np.abs(lam)) * OMEGA_UNIT_EV
    m = np.repeat(np.asarray(masses, dtype=np.float64), 3)
    u = e / np.sqrt(m)[None, :, None]
    return omega, e, u


# ----------------------------------------------------------------------------
# Eq. 9: Fourier transform over the phonon WS vectors Rp (outer q loop).
# ----------------------------------------------------------------------------
def g_rp_to_q(qpts, Rp, wp, g_ReRp) -> np.ndarray:
    """g(Re, q) = sum_Rp g(Re, Rp) e^{i q.Rp}  -> [nq][nm][ne][nb][nb]  (Eq. 9)."""
    P = phases(qpts, Rp, wp)
    np_ = g_ReRp.shape[0]
    rest = g_ReRp.shape[1:]
    return (P @ g_ReRp.reshape(np_, -1)).reshape((len(qpts),) + rest)


# ----------------------------------------------------------------------------
# Eq. 10: FT over Re, then the U_{k+q}, U_k* and u(q) rotations (inner k loop).
# ----------------------------------------------------------------------------
def g_req_to_bloch(kpts, Re, we, G1q, V_k, V_kq, u_q) -> np.ndarray:
    """Eq. 10 for one q.

    G1q: [nm][ne][nb][nb] = g(Re, q); V_k, V_kq: [nk][nb][nb] eigenvectors as
    columns at k and k+q; u_q: [nm][nm] (rows kappa alpha, columns nu).
    Returns g[nk][nu][m][n].
    """
    P = phases(kpts, Re, we)                                   # [nk][ne]
    nm, ne, nb, _ = G1q.shape
    # sum over Re: Gk[k][ka][m'][n']
    Gk = np.einsum("ke,cemn->kcmn", P, G1q)
    # band rotation U_{mm',k+q} U*_{nn',k}: V_{k+q}^H Gk V_k (two matrix products per (k, ka))
    Gb = np.matmul(np.matmul(V_kq.conj().transpose(0, 2, 1)[:, None], Gk), V_k[:, None])
    # mode rotation by u_{kappa alpha, nu}(q)
    return np.einsum("cv,kcmn->kvmn", u_q, Gb)


# ----------------------------------------------------------------------------
# Full interpolation (nested-loop algorithm, Eqs. 9-10).
# ----------------------------------------------------------------------------
def interpolate(wl_or_arrays, kpts=None, qpts=None, return_eigvecs=False):
    """eps_k [nk][nb], eps_kq [nq][nk][nb], omega [nq][nm], g [nq][nk][nm][nb][nb].

    Accepts any object with attributes H_Re, Phi_Rp, g_ReRp, Re, Rp, we, wp,
    masses (e.g. a synthetic workload).  k+q phases are formed from the sum
    k + q (no wrapping; every quantity is periodic).
    """
    a = wl_or_arrays
    kpts = a.kpts if kpts is None else np.asarray(kpts, dtype=np.float64)
    qpts = a.qpts if qpts is None else np.asarray(qpts, dtype=np.float64)
    nb = a.H_Re.shape[1]
    nm = a.Phi_Rp.shape[1]
    eps_k, V_k = electron_eigen(hamiltonian_k(kpts, a.Re, a.we, a.H_Re))
    omega, _, u = phonon_eigen(dynamical_matrix(qpts, a.Rp, a.wp, a.Phi_Rp, a.masses), a.masses)
    G1 = g_rp_to_q(qpts, a.Rp, a.wp, a.g_ReRp)
    nk, nq = len(kpts), len(qpts)
    g = np.empty((nq, nk, nm, nb, nb), dtype=np.complex128)
    eps_kq = np.empty((nq, nk, nb))
    Vkq_all = [] if return_eigvecs else None
    for iq in range(nq):
        e_kq, V_kq = electron_eigen(hamiltonian_k(kpts + qpts[iq][None, :], a.Re, a.we, a.H_Re))
        eps_kq[iq] = e_kq
        g[iq] = g_req_to_bloch(kpts, a.Re, a.we, G1[iq], V_k, V_kq, u[iq])
        if return_eigvecs:
            Vkq_all.append(V_kq)
    if return_eigvecs:
        return eps_k, eps_kq, omega, g, dict(V_k=V_k, V_kq=np.stack(Vkq_all), u=u)
    return eps_k, eps_kq, omega, g


# ----------------------------------------------------------------------------
# Eq. 7 literally (single-loop algorithm, Fig. 1a) -- tiny inputs only.
# ----------------------------------------------------------------------------
def g_single_loop(k, q, Re, we, Rp, wp, g_ReRp, V_k, V_kq, u_q) -> np.ndarray:
    """g[nu][m][n] at one (k, q) from Eq. 7 with the full double phase e^{i(q.Rp + k.Re)}.

    U_{mm',k+q} = conj(V_kq[m'][m]) and U*_{nn',k} = V_k[n'][n].
    """
    Ref = np.asarray(Re, dtype=np.float64)
    Rpf = np.asarray(Rp, dtype=np.float64)
    t = (Rpf @ np.asarray(q, dtype=np.float64))[:, None] + (Ref @ np.asarray(k, dtype=np.float64))[None, :]
    t = t - np.rint(t)
    E = (np.cos(2 * np.pi * t) + 1j * np.sin(2 * np.pi * t)) * np.outer(wp, we)   # [np][ne]
    U_kq = V_kq.conj().T          # U_{m m'}
    Ustar_k = V_k.T               # U*_{n n'}
    return np.einsum("pcexy,pe,mx,ny,cv->vmn", g_ReRp, E, U_kq, Ustar_k, u_q)


# ----------------------------------------------------------------------------
# Eq. 6: Bloch -> Wannier on a commensurate coarse grid.
# ----------------------------------------------------------------------------
def g_bloch_to_wannier(kc, qc, Re, Rp, g_bloch, V_k, V_kq, u_q) -> np.ndarray:
    """Eq. 6: g(Re,Rp) = 1/(Ne Np) sum g_mnnu(k',q') U*_{mm',k'+q'} U_{nn',k'} u^{-1}_{nu,ka}(q') e^{-i(q'.Rp + k'.Re)}.

    g_bloch: [nq'][nk'][nm][nb][nb]; V_k: [nk'][nb][nb]; V_kq: [nq'][nk'][nb][nb]; u_q: [nq'][nm][nm].
    Returns [np][nm][ne][nb][nb].
    """
    ne, np_ = len(Re), len(Rp)
    Pk = phases(kc, Re).conj()     # e^{-i k'.Re}  [nk'][ne]
    Pq = phases(qc, Rp).conj()     # e^{-i q'.Rp}  [nq'][np]
    uinv = np.linalg.inv(u_q)      # [nq'][nu][ka]
    # U*_{mm',k'+q'} = V_kq[m'][m];  U_{nn',k'} = conj(V_k[n'][n])
    # X[q][k][nu][m'][n'] = sum_mn g[q][k][nu][m][n] V_kq[q][k][m'][m] conj(V_k[k][n'][n])
    X = np.einsum("qkvmn,qkxm,kyn->qkvxy", g_bloch, V_kq, V_k.conj())
    Y = np.einsum("qkvxy,qvc->qkcxy", X, uinv)
    out = np.einsum("qkcxy,ke,qp->pcexy", Y, Pk, Pq)
    return out / (ne * np_)


# ----------------------------------------------------------------------------
# Differentiable scalar and its adjoint (hand-written reverse chain).
# ----------------------------------------------------------------------------
def loss_weights(omega, w_nk, omega_min):
    """c[q][k][nu][n] = w_nk / omega_qnu for omega > omega_min, else 0."""
    inv = np.where(omega > omega_min, 1.0 / np.where(omega > omega_min, omega, 1.0), 0.0)   # [nq][nm]
    return inv[:, None, :, None] * np.asarray(w_nk)[None, :, None, :]


def loss(g, omega, w_nk, omega_min) -> float:
    """L = sum_{q,k,nu,m,n} w_nk |g_mnnu(k,q)|^2 / omega_qnu over modes with omega > omega_min."""
    c = loss_weights(omega, w_nk, omega_min)                       # [nq][nk][nm][nb(n)]
    return float(np.sum(c[:, :, :, None, :] * np.abs(g) ** 2))


def loss_and_grad(a, kpts, qpts, w_nk, omega_min):
    """L and dL/dg(Re,Rp) (= dL/dRe + i dL/dIm) with U, e held fixed.

    Forward: Eqs. 9-10.  Reverse: gbar = 2 c g; Gk_bar = sum_nu conj(u) V_kq gbar V_k^H;
    G1_bar = sum_k conj(P_k) Gk_bar; grad = sum_q conj(P_q) G1_bar.
    """
    kpts = np.asarray(kpts, dtype=np.float64)
    qpts = np.asarray(qpts, dtype=np.float64)
    eps_k, eps_kq, omega, g, ev = interpolate(a, kpts, qpts, return_eigvecs=True)
    L = loss(g, omega, w_nk, omega_min)
    c = loss_weights(omega, w_nk, omega_min)
    gbar = 2.0 * c[:, :, :, None, :] * g                           # [nq][nk][nu][m][n]
    return L, vjp(a, kpts, qpts, gbar, ev)


def vjp(a, kpts, qpts, gbar, ev):
    """A^H gbar for the linear map A: g(Re,Rp) -> g(k,q) (Eqs. 9-10 and the band rotation of
    Eq. 7) at fixed gauges ev = interpolate(..., return_eigvecs=True)[4]; gbar [nq][nk][nm][nb][nb]
    in the dL/dRe + i dL/dIm convention.  Reverse chain: Gk_bar = sum_nu conj(u) V_kq gbar V_k^H;
    G1_bar = sum_k conj(P_k) Gk_bar; grad = sum_q conj(P_q) G1_bar.
    """
    kpts = np.asarray(kpts, dtype=np.float64)
    qpts = np.asarray(qpts, dtype=np.float64)
    Pk = phases(kpts, a.Re, a.we)                                  # [nk][ne]
    Pq = phases(qpts, a.Rp, a.wp)                                  # [nq][np]
    V_k, V_kq, u = ev["V_k"], ev["V_kq"], ev["u"]
    nq = len(qpts)
    nm, ne, nb = a.g_ReRp.shape[1], a.g_ReRp.shape[2], a.g_ReRp.shape[3]
    G1bar = np.empty((nq, nm, ne, nb, nb), dtype=np.complex128)
    for iq in range(nq):
        Gb_bar = np.einsum("kam,kvmn,kbn->kvab", V_kq[iq], gbar[iq], V_k.conj())   # V_kq gbar V_k^H
        Gk_bar = np.einsum("cv,kvab->kcab", u[iq].conj(), Gb_bar)
        G1bar[iq] = np.einsum("ke,kcab->ceab", Pk.conj(), Gk_bar)
    return (Pq.conj().T @ G1bar.reshape(nq, -1)).reshape(a.g_ReRp.shape)


def fermi_weights(eps_k, band_index, kT=0.025852):
    """w_nk = 1/(exp((eps-mu)/kT)+1) with mu the median of band `band_index` over the k grid."""
    mu = float(np.median(eps_k[:, band_index]))
    return 1.0 / (np.exp((eps_k - mu) / kT) + 1.0), mu


# ----------------------------------------------------------------------------
# Downstream consumer: electron linewidths (imaginary part of the Fan-Migdal self-energy).
# ----------------------------------------------------------------------------
def bose(omega, kT):
    """n_B(omega) = 1 / (exp(omega/kT) - 1)."""
    return 1.0 / np.expm1(omega / kT)


def fermi(eps, mu, kT):
    """f(eps) = 1 / (exp((eps - mu)/kT) + 1)."""
    return 1.0 / (np.exp((eps - mu) / kT) + 1.0)


def gaussian(x, sigma):
    return np.exp(-0.5 * (x / sigma) ** 2) / (sigma * np.sqrt(2.0 * np.pi))


def linewidths(eps_k, eps_kq, omega, g, wq, kT, mu, sigma, omega_min):
    """Gamma_nk = pi sum_q w_q sum_{m, nu: omega > omega_min} |g_mnnu(k,q)|^2 / (2 omega_qnu)
         x [ (n_qnu + f_{m,k+q}) delta(eps_nk - eps_{m,k+q} + omega_qnu)
           + (n_qnu + 1 - f_{m,k+q}) delta(eps_nk - eps_{m,k+q} - omega_qnu) ]
    with Gaussian delta of width sigma (phonon absorption and emission terms of the
    imaginary part of the Fan-Migdal self-energy).  Returns [nk][nb] in units of |g|^2/eV^2.
    eps_k [nk][nb], eps_kq [nq][nk][nb], omega [nq][nm], g [nq][nk][nm][nb][nb], wq [nq].
    """
    om = np.asarray(omega)[:, None, :, None, None]                 # q, -, nu, -, -
    ok = om > omega_min
    oms = np.where(ok, om, 1.0)
    nB = np.where(ok, bose(oms, kT), 0.0)
    fm = fermi(np.asarray(eps_kq), mu, kT)[:, :, None, :, None]      # q, k, -, m, -
    de = np.asarray(eps_k)[None, :, None, None, :] - np.asarray(eps_kq)[:, :, None, :, None]   # eps_nk - eps_mk+q
    term = (nB + fm) * gaussian(de + oms, sigma) + (nB + 1.0 - fm) * gaussian(de - oms, sigma)
    contrib = np.where(ok, np.abs(g) ** 2 / (2.0 * oms) * term, 0.0)  # [q][k][nu][m][n]
    return np.pi * np.einsum("q,qkvmn->kn", np.asarray(wq, dtype=np.float64), contrib)


# ----------------------------------------------------------------------------
# Irreducible k list under time reversal (the transport workflow's reduced fine k grid).
# ----------------------------------------------------------------------------
def grid_points(n, shift=(0.0, 0.0, 0.0)) -> np.ndarray:
    """k = (j1/n1, j2/n2, j3/n3) + shift in the order (j1 n2 + j2) n3 + j3 -> [n1 n2 n3][3]."""
    n1, n2, n3 = n
    j = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1).reshape(-1, 3)
    return j / np.array([n1, n2, n3], dtype=np.float64) + np.asarray(shift, dtype=np.float64)[None, :]


def ibz_time_reversal(n, shift=(0.0, 0.0, 0.0)):
    """(kept grid indices ascending, weights) of the reduction k ~ -k of a uniform grid.

    With real H(Re), H(-k) = conj H(k) and eps(-k) = eps(k), so a grid sum is the weighted sum
    over one point of each pair {k, -k} (-k taken modulo reciprocal lattice vectors).  Brute
    force: the partner of each point is the grid point whose coordinates add to an integer
    vector with it; a point is kept if its index is not above its partner's, with weight 2, or 1
    if it is its own partner.  Small grids only (all pairs are compared).
    """
    pts = grid_points(n, shift)
    s = pts[:, None, :] + pts[None, :, :]
    d = np.abs(s - np.rint(s)).max(-1)
    match = d < 1e-9
    if not np.all(match.sum(1) == 1):
        raise ValueError("-k is not on the grid (2 shift n must be an integer on every axis)")
    partner = match.argmax(1)
    idx = np.arange(len(pts))
    keep = idx <= partner
    w = np.where(partner == idx, 1.0, 2.0)
    return idx[keep], w[keep]
