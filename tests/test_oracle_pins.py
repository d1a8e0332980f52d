"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each compares the oracle with a
closed form, an invariant, a brute-force evaluation of Eq. 7, a round trip
through Eq. 6, or a value printed in the paper.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_10295_gb300 import synth
from tests import gauge

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- constants
def test_omega_unit_matches_textbook_thz():
    # sqrt(eV/(A^2 amu)) / (2 pi) = 15.633302 THz (standard conversion factor);
    # h = 4.135667696e-15 eV s.
    f_thz = 15.633302
    h_ev_s = 4.135667696e-15
    assert abs(oracle.OMEGA_UNIT_EV - f_thz * 1e12 * h_ev_s) < 1e-8


# ---------------------------------------------------------------- phases
def test_phase_properties():
    rng = np.random.default_rng(1)
    k = rng.random((50, 3))
    R = rng.integers(-9, 10, size=(40, 3)).astype(np.int32)
    P = oracle.phases(k, R)
    assert np.allclose(np.abs(P), 1.0, atol=1e-15)
    # R = 0 column is exactly 1
    P0 = oracle.phases(k, np.zeros((1, 3), np.int32))
    assert np.all(P0 == 1.0)
    # periodic in k with period 1 (integer shift), product rule e^{ik.R}e^{ik'.R} = e^{i(k+k').R}
    G = rng.integers(-3, 4, size=(50, 3))
    assert np.abs(oracle.phases(k + G, R) - P).max() < 1e-12
    k2 = rng.random((50, 3))
    assert np.abs(oracle.phases(k, R) * oracle.phases(k2, R) - oracle.phases(k + k2, R)).max() < 1e-12
    # dyadic points 2^20 cells away: k.R is exact in FP64, so the exact reduction t - rint(t)
    # returns the in-cell argument up to the sign of r = +-1/2 (rint rounds half to even), i.e.
    # the in-cell phases to the last bit of sin(pi) (an unreduced sin(2 pi t) is off by ~1e-8)
    kd = rng.integers(0, 8, size=(50, 3)) / 8.0
    Gd = rng.integers(-(1 << 20), 1 << 20, size=(50, 3))
    assert np.abs(oracle.phases(kd + Gd, R) - oracle.phases(kd, R)).max() <= 1e-15
    # explicit value: k=(1/4,0,0), R=(1,0,0) -> i
    assert abs(oracle.phases(np.array([[0.25, 0, 0]]), np.array([[1, 0, 0]]))[0, 0] - 1j) < 1e-15


# ---------------------------------------------------------------- hermiticity / ASR
@pytest.mark.parametrize("box", [None, (synth.centred_range(4), synth.centred_range(4), synth.centred_range(4))])
def test_hermiticity_and_asr(box):
    wl = synth.make_workload("si_tiny", nq=8, nk=8, box=box, with_coupling=False)
    # H(-R) = H(R)^dagger and Phi(-R) = Phi(R)^T imply Hermitian H(k), D(q)
    Hk = oracle.hamiltonian_k(wl.kpts, wl.Re, wl.we, wl.H_Re)
    assert np.abs(Hk - Hk.conj().transpose(0, 2, 1)).max() < 1e-14 * np.abs(Hk).max()
    Dq = oracle.dynamical_matrix(wl.qpts, wl.Rp, wl.wp, wl.Phi_Rp, wl.masses)
    assert np.abs(Dq - Dq.conj().transpose(0, 2, 1)).max() < 1e-14 * np.abs(Dq).max()
    # ASR: three zero modes at Gamma, eigenvectors along sqrt(M) translations
    D0 = oracle.dynamical_matrix(np.zeros((1, 3)), wl.Rp, wl.wp, wl.Phi_Rp, wl.masses)[0]
    lam, e = np.linalg.eigh(D0)
    assert np.all(np.abs(lam[:3]) <= 1e-12 * lam[-1])
    assert lam[3] > 1e-6 * lam[-1]
    m = np.repeat(wl.masses, 3)
    for a in range(3):
        t = np.zeros(3 * wl.na)
        t[a::3] = np.sqrt(m[a::3])
        t /= np.linalg.norm(t)
        # translation lies in the zero-mode subspace
        assert np.linalg.norm(e[:, :3].conj().T @ t) > 1 - 1e-10
    # spring model is positive semidefinite at every q
    om, _, _ = oracle.phonon_eigen(Dq, wl.masses)
    assert np.all(om >= -1e-6 * om.max())


# ---------------------------------------------------------------- closed forms
def test_one_band_chain_closed_form():
    eps0, t = 0.37, -1.25
    R = np.array([[-1, 0, 0], [0, 0, 0], [1, 0, 0]], np.int32)
    H = np.array([t, eps0, t], dtype=np.complex128).reshape(3, 1, 1)
    k = np.stack([np.linspace(0, 1, 41), np.zeros(41), np.zeros(41)], -1)
    eps, _ = oracle.electron_eigen(oracle.hamiltonian_k(k, R, np.ones(3), H))
    assert np.abs(eps[:, 0] - (eps0 + 2 * t * np.cos(2 * np.pi * k[:, 0]))).max() < 1e-14


def test_spring_chain_closed_form():
    K, M = 3.7, 28.0855
    R = np.array([[-1, 0, 0], [0, 0, 0], [1, 0, 0]], np.int32)
    Phi = np.zeros((3, 3, 3))
    Phi[1, 0, 0] = 2 * K
    Phi[0, 0, 0] = Phi[2, 0, 0] = -K
    q = np.stack([np.linspace(0, 1, 37), np.zeros(37), np.zeros(37)], -1)
    om, _, _ = oracle.phonon_eigen(oracle.dynamical_matrix(q, R, np.ones(3), Phi, [M]), [M])
    # y, z modes carry no springs: zero; the x mode is the textbook chain
    expect = 2 * np.sqrt(K / M) * np.abs(np.sin(np.pi * q[:, 0])) * 0.0646541513
    assert np.abs(om[:, 2] - expect).max() < 1e-9 * expect.max()
    assert np.abs(om[:, :2]).max() < 1e-12



def test_unstable_spring_chain_negative_frequency():
    # a negative spring constant: lambda(q) = 4K/M sin^2(pi q) < 0, reported as
    # omega = -sqrt(|lambda|) (the sign convention for unstable modes)
    K, M = -2.3, 28.0855
    R = np.array([[-1, 0, 0], [0, 0, 0], [1, 0, 0]], np.int32)
    Phi = np.zeros((3, 3, 3))
    Phi[1, 0, 0] = 2 * K
    Phi[0, 0, 0] = Phi[2, 0, 0] = -K
    q = np.stack([np.linspace(0.05, 0.95, 19), np.zeros(19), np.zeros(19)], -1)
    om, _, _ = oracle.phonon_eigen(oracle.dynamical_matrix(q, R, np.ones(3), Phi, [M]), [M])
    expect = -2 * np.sqrt(-K / M) * np.abs(np.sin(np.pi * q[:, 0])) * 0.0646541513
    assert np.abs(om[:, 0] - expect).max() < 1e-9 * np.abs(expect).max()
    assert np.abs(om[:, 1:]).max() < 1e-12


class _Arrays:
    pass


def _chain_model(eps0, t, K1, K2, M, Gt):
    """One band with complex hopping t on the bond to the next cell (t* back), two equal
    masses M per cell with x springs K1 inside the cell and K2 to the next cell, and a
    coupling Gt[6] at Re = Rp = 0 only.  R list: -x, 0, +x."""
    R = np.array([[-1, 0, 0], [0, 0, 0], [1, 0, 0]], np.int32)
    H = np.array([np.conj(t), eps0, t], dtype=np.complex128).reshape(3, 1, 1)
    Phi = np.zeros((3, 6, 6))
    Phi[1, 0, 0] = Phi[1, 3, 3] = K1 + K2
    Phi[1, 0, 3] = Phi[1, 3, 0] = -K1
    Phi[2, 3, 0] = -K2      # atom 1 of the home cell to atom 0 of the cell at +x
    Phi[0, 0, 3] = -K2      # its transpose at -x
    gW = np.zeros((3, 6, 3, 1, 1), np.complex128)
    gW[1, :, 1, 0, 0] = Gt
    a = _Arrays()
    a.H_Re, a.Phi_Rp, a.g_ReRp, a.Re, a.Rp = H, Phi, gW, R, R
    a.we, a.wp, a.masses = np.ones(3), np.ones(3), np.array([M, M])
    return a


def test_complex_hopping_and_diatomic_chain_closed_forms():
    # electrons: eps(k) = eps0 + 2|t| cos(2 pi k + arg t) for the e^{+ik.R} convention
    # (distinguishes k from -k), at k and at k+q.  Phonons: the diatomic chain,
    # D(q) = [[a, b], [conj(b), a]] on the two x displacements with a = (K1+K2)/M and
    # b = -(K1 + K2 e^{-2 pi i q})/M; branches a -+ |b| with eigenvectors
    # (1, -+e^{-i beta})/sqrt(2), beta = arg b.  With one band, V = 1 and g_nu = u_nu^T Gt,
    # so |g| of the two x branches is |Gt_0 -+ e^{-i beta} Gt_3| / sqrt(2M) (the sign of
    # the phase convention, the mass factor and the mode index all enter).
    eps0, t = 0.4, 0.9 * np.exp(0.7j)
    K1, K2, M = 3.1, 1.2, 20.0
    rng = np.random.default_rng(8)
    Gt = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    a = _chain_model(eps0, t, K1, K2, M, Gt)
    k = np.stack([rng.random(7), rng.random(7), rng.random(7)], -1)
    q = np.stack([np.linspace(0.07, 0.93, 9), rng.random(9), rng.random(9)], -1)
    eps_k, eps_kq, omega, g = oracle.interpolate(a, k, q)
    band = lambda x: eps0 + 2 * abs(t) * np.cos(2 * np.pi * x + np.angle(t))
    assert np.abs(eps_k[:, 0] - band(k[:, 0])).max() < 1e-14
    assert np.abs(eps_kq[:, :, 0] - band(k[None, :, 0] + q[:, None, 0])).max() < 1e-14
    av = (K1 + K2) / M
    b = -(K1 + K2 * np.exp(-2j * np.pi * q[:, 0])) / M
    beta = np.angle(b)
    unit = 0.0646541513
    assert (omega[:, :4] ** 2).max() < 1e-14 * av * unit ** 2      # y, z: no springs (lambda at rounding level)
    assert np.abs(omega[:, 4] - np.sqrt(av - np.abs(b)) * unit).max() < 1e-9
    assert np.abs(omega[:, 5] - np.sqrt(av + np.abs(b)) * unit).max() < 1e-9
    for s, nu in ((-1, 4), (1, 5)):
        expect = np.abs(Gt[0] + s * np.exp(-1j * beta) * Gt[3]) / np.sqrt(2 * M)
        assert np.abs(np.abs(g[:, :, nu, 0, 0]) - expect[:, None]).max() < 1e-12

def _plane_wave_inputs(nb=4, na=2, seed=3):
    rng = np.random.default_rng(seed)
    R = synth.box_vectors(range(-1, 2), range(-1, 2), range(0, 1))
    ne = len(R)
    nm = 3 * na
    masses = np.array([12.0, 31.0][:na])
    # H nonzero only at R=0: H0 = Q diag(1..nb) Q^H with Q the unitary DFT matrix
    Q = np.exp(2j * np.pi * np.outer(np.arange(nb), np.arange(nb)) / nb) / np.sqrt(nb)
    H = np.zeros((ne, nb, nb), np.complex128)
    i0 = int(np.where((R == 0).all(1))[0][0])
    H[i0] = Q @ np.diag(np.arange(1.0, nb + 1)) @ Q.conj().T
    # Phi nonzero only at R=0, diagonal with D = Phi/M ascending and distinct
    dvals = np.arange(1.0, nm + 1) * 0.7
    Phi = np.zeros((ne, nm, nm))
    Phi[i0] = np.diag(dvals * np.repeat(masses, 3))
    e0, p0 = 5, 2          # Re0 index, Rp0 index
    Gt = rng.standard_normal((nm, nb, nb)) + 1j * rng.standard_normal((nm, nb, nb))
    gW = np.zeros((ne, nm, ne, nb, nb), np.complex128)
    gW[p0, :, e0] = Gt
    we = rng.uniform(0.5, 1.5, ne)
    wp = rng.uniform(0.5, 1.5, ne)

    class A:
        pass
    a = A()
    a.H_Re, a.Phi_Rp, a.g_ReRp, a.Re, a.Rp, a.we, a.wp, a.masses = H, Phi, gW, R, R, we, wp, masses
    return a, Q, Gt, e0, p0, dvals, i0


def test_single_R_plane_wave_closed_form():
    a, Q, Gt, e0, p0, dvals, i0 = _plane_wave_inputs()
    rng = np.random.default_rng(4)
    k = rng.random((7, 3))
    q = rng.random((5, 3))
    eps_k, eps_kq, omega, g = oracle.interpolate(a, k, q)
    nb = Q.shape[0]
    # H(k) = we(0) H0 and D(q) = wp(0) Phi0/M at every point
    assert np.abs(eps_k - a.we[i0] * np.arange(1.0, nb + 1)).max() < 1e-13
    assert np.abs(omega - np.sqrt(a.wp[i0] * dvals) * 0.0646541513).max() < 1e-9
    m = np.repeat(a.masses, 3)
    # |g_mn nu| = we0 wp0 |(Q^H Gt_nu Q)_mn| / sqrt(M_nu); the phase of g(k,q)/g(0,0)
    # is exactly e^{2 pi i (k.Re0 + q.Rp0)} (same gauge at every point).
    QGQ = np.einsum("am,vab,bn->vmn", Q.conj(), Gt, Q)
    expect_abs = a.we[e0] * a.wp[p0] * np.abs(QGQ) / np.sqrt(m)[:, None, None]
    assert np.abs(np.abs(g) - expect_abs[None, None]).max() < 1e-12
    _, _, _, g00 = oracle.interpolate(a, np.zeros((1, 3)), np.zeros((1, 3)))
    ph = np.exp(2j * np.pi * (k @ a.Re[e0])[None, :] + 2j * np.pi * (q @ a.Rp[p0])[:, None])
    assert np.abs(g - ph[:, :, None, None, None] * g00[0, 0][None, None]).max() < 1e-12


# ---------------------------------------------------------------- factorisation vs Eq. 7
def test_nested_equals_single_loop():
    wl = synth.make_workload("si_tiny", nb=3, nk=6, nq=5)
    eps_k, eps_kq, omega, g, ev = oracle.interpolate(wl, return_eigvecs=True)
    for iq in range(len(wl.qpts)):
        for ik in range(len(wl.kpts)):
            ref = oracle.g_single_loop(wl.kpts[ik], wl.qpts[iq], wl.Re, wl.we, wl.Rp, wl.wp, wl.g_ReRp,
                                       ev["V_k"][ik], ev["V_kq"][iq, ik], ev["u"][iq])
            assert np.abs(g[iq, ik] - ref).max() < 1e-13 * max(1.0, np.abs(ref).max())


# ---------------------------------------------------------------- Wannier round trip (Eq. 7 then Eq. 6)
def test_wannier_round_trip():
    wl = synth.make_workload("si_tiny")
    coarse = synth.uniform_grid(3, 3, 3)          # the 3x3x3 BvK grid of the [-1,1]^3 box
    eps_k, eps_kq, omega, g, ev = oracle.interpolate(wl, coarse, coarse, return_eigvecs=True)
    rec = oracle.g_bloch_to_wannier(coarse, coarse, wl.Re, wl.Rp, g, ev["V_k"], ev["V_kq"], ev["u"])
    assert np.abs(rec - wl.g_ReRp).max() < 1e-12 * np.abs(wl.g_ReRp).max()


# ---------------------------------------------------------------- gauge-free invariants
def test_unitarity_invariant_and_periodicity():
    wl = synth.make_workload("si_tiny", nk=9, nq=4)
    eps_k, eps_kq, omega, g, ev = oracle.interpolate(wl, return_eigvecs=True)
    G1 = oracle.g_rp_to_q(wl.qpts, wl.Rp, wl.wp, wl.g_ReRp)
    P = oracle.phases(wl.kpts, wl.Re, wl.we)
    for iq in range(4):
        Gk = np.einsum("ke,cemn->kcmn", P, G1[iq])
        Gv = np.einsum("cv,kcmn->kvmn", ev["u"][iq], Gk)
        lhs = (np.abs(g[iq]) ** 2).sum((-1, -2))
        rhs = (np.abs(Gv) ** 2).sum((-1, -2))
        assert np.abs(lhs - rhs).max() < 1e-12 * rhs.max()
    # periodicity g(k+G, q+G') equals g(k,q) on gauge-invariant subspace sums
    rng = np.random.default_rng(5)
    Gk_shift = rng.integers(-2, 3, size=wl.kpts.shape)
    Gq_shift = rng.integers(-2, 3, size=wl.qpts.shape)
    e2k, e2kq, om2, g2 = oracle.interpolate(wl, wl.kpts + Gk_shift, wl.qpts + Gq_shift)
    assert gauge.max_rel_S(g2, g, eps_k, eps_kq, omega) < 1e-11
    assert gauge.max_rel_eps(e2k, eps_k) < 1e-13


def test_linearity_in_coupling():
    wl = synth.make_workload("si_tiny", nk=5, nq=3)
    rng = np.random.default_rng(6)
    _, _, _, g1, ev = oracle.interpolate(wl, return_eigvecs=True)
    import copy
    wl2 = copy.copy(wl)
    extra = rng.standard_normal(wl.g_ReRp.shape) + 1j * rng.standard_normal(wl.g_ReRp.shape)
    wl2.g_ReRp = extra
    _, _, _, g2 = oracle.interpolate(wl2)
    wl3 = copy.copy(wl)
    alpha = 0.3 - 1.7j
    wl3.g_ReRp = wl.g_ReRp + alpha * extra
    _, _, _, g3 = oracle.interpolate(wl3)
    # same H, Phi -> same eigenvectors (deterministic), so g is linear elementwise
    assert np.abs(g3 - (g1 + alpha * g2)).max() < 1e-12 * np.abs(g3).max()


# ---------------------------------------------------------------- adjoint
def test_adjoint_central_differences_and_euler():
    wl = synth.make_workload("si_tiny", nb=4, nk=6, nq=3)
    eps_k, _, _, _ = oracle.interpolate(wl)
    w_nk, _ = oracle.fermi_weights(eps_k, 2)
    L, grad = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w_nk, 1e-6)
    # Euler: L is homogeneous of degree 2 in gW -> Re<grad, gW> = 2L
    assert abs(np.real(np.vdot(grad, wl.g_ReRp)) - 2 * L) < 1e-12 * abs(L)
    import copy
    rng = np.random.default_rng(7)
    flat = wl.g_ReRp.reshape(-1)
    idx = rng.choice(flat.size, size=25, replace=False)
    h = 1e-6
    for i in idx:
        for part, unit in (("re", 1.0), ("im", 1j)):
            plus = copy.copy(wl)
            minus = copy.copy(wl)
            gp = flat.copy()
            gm = flat.copy()
            gp[i] += unit * h
            gm[i] -= unit * h
            plus.g_ReRp = gp.reshape(wl.g_ReRp.shape)
            minus.g_ReRp = gm.reshape(wl.g_ReRp.shape)
            _, _, om, gpl = oracle.interpolate(plus)
            _, _, _, gmi = oracle.interpolate(minus)
            d = (oracle.loss(gpl, om, w_nk, 1e-6) - oracle.loss(gmi, om, w_nk, 1e-6)) / (2 * h)
            ref = grad.reshape(-1)[i].real if part == "re" else grad.reshape(-1)[i].imag
            assert abs(d - ref) <= 1e-6 * max(1.0, np.abs(grad).max())



def test_loss_closed_form_on_plane_wave():
    # on the plane-wave inputs |g_mn nu| and omega_nu are known in closed form and the same at
    # every (k, q), so L = nq sum_k sum_n w_nk sum_nu (sum_m |g_mn nu|^2) / omega_nu, with the
    # weight on the band index n of the k side and modes at or below omega_min left out; the
    # oracle's L (and, by Euler's identity, its gradient) must give exactly this
    a, Q, Gt, e0, p0, dvals, i0 = _plane_wave_inputs()
    rng = np.random.default_rng(9)
    k = rng.random((5, 3))
    q = rng.random((4, 3))
    nb = Q.shape[0]
    w_nk = rng.uniform(0.0, 1.0, (len(k), nb))
    m = np.repeat(a.masses, 3)
    QGQ = np.einsum("am,vab,bn->vmn", Q.conj(), Gt, Q)
    g2 = (a.we[e0] * a.wp[p0]) ** 2 * np.abs(QGQ) ** 2 / m[:, None, None]      # [nu][m][n]
    om = np.sqrt(a.wp[i0] * dvals) * oracle.OMEGA_UNIT_EV     # [nu], ascending (unit pinned above)
    for omega_min in (1e-6, 0.5 * (om[2] + om[3])):
        keep = om > omega_min
        per_n = (g2.sum(axis=1)[keep] / om[keep][:, None]).sum(axis=0)         # [n]
        expect = len(q) * float((w_nk * per_n[None, :]).sum())
        L, grad = oracle.loss_and_grad(a, k, q, w_nk, omega_min)
        assert abs(L - expect) < 1e-12 * expect
        assert abs(np.real(np.vdot(grad, a.g_ReRp)) - 2 * expect) < 1e-12 * expect

def test_vjp_is_the_adjoint_of_the_interpolation():
    # g(k,q) is linear in g(Re,Rp) at fixed H, Phi (fixed gauges), so for any upstream gbar
    # and direction d: Re<vjp(gbar), d> = Re<gbar, A(d)>, A(d) = interpolation of d.
    import copy
    wl = synth.make_workload("si_tiny", nb=3, nk=5, nq=3)
    rng = np.random.default_rng(31)
    _, _, _, g, ev = oracle.interpolate(wl, return_eigvecs=True)
    gbar = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
    d = rng.standard_normal(wl.g_ReRp.shape) + 1j * rng.standard_normal(wl.g_ReRp.shape)
    wd = copy.copy(wl)
    wd.g_ReRp = d
    _, _, _, Ad = oracle.interpolate(wd)
    lhs = np.real(np.vdot(oracle.vjp(wl, wl.kpts, wl.qpts, gbar, ev), d))
    rhs = np.real(np.vdot(gbar, Ad))
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(gbar) * np.abs(Ad))
    # and the loss gradient is the vjp of 2 c g
    w_nk = rng.uniform(0.0, 1.0, (len(wl.kpts), wl.nb))
    _, grad = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w_nk, 1e-6)
    _, _, om, _ = oracle.interpolate(wl)
    c = oracle.loss_weights(om, w_nk, 1e-6)
    assert np.abs(oracle.vjp(wl, wl.kpts, wl.qpts, 2 * c[:, :, :, None, :] * g, ev) - grad).max() \
        <= 1e-14 * np.abs(grad).max()


# ---------------------------------------------------------------- paper-printed values
def test_table3_sizes_and_cost_ratio():
    rows = [list(map(float, l.split())) for l in open(os.path.join(HERE, "golden", "zsnr_gw_sizes.txt"))
            if l.strip() and not l.startswith("#")]
    for w, nb, nm, ne, np_, size in rows:
        gib = 16 * nb * nb * nm * ne * np_ / 2 ** 30
        # printed with 2 significant digits (1 decimal below 10)
        assert abs(gib - size) <= max(0.05, 0.005 * size) + 0.5 * (size >= 10), (w, gib, size)
    # Eq. 12: NL/SL ratio for silicon is about 1/93 when Nk >> Np
    nb, nm, ne, np_, nk = 8, 6, 617, 93, 10 ** 6
    sl = (nb * nb * nm * ne * np_ + nb * nb * nm * ne + 2 * nb * nb * nm + nb * nb * nm * nm) * nk
    nl = nb * nb * nm * ne * np_ + (nb * nb * nm * ne + 2 * nb * nb * nm + nb * nb * nm * nm) * nk
    assert abs(sl / nl - 93) < 1.0


# ---------------------------------------------------------------- linewidth consumer
# Two one-band chains eps_m(k) = e0_m + 2 t_m cos(2 pi k) (textbook tight-binding bands) and
# three degenerate Einstein modes omega0 (one atom, on-site springs only: D(q) = K/M for every
# q), with a coupling that does not depend on k or q: g_mn,nu = G_mn e_{x,nu}(q)/sqrt(M), e a
# random unitary basis of the degenerate mode space at every q (sum_nu |e_{x,nu}|^2 = 1).  On a
# uniform q grid with w_q = 1/Nq, sum_q w_q delta(E - eps_m(k+q)) tends to the chain density of
# states rho_m(E) = 1/(pi sqrt(4 t_m^2 - (E - e0_m)^2)) as sigma -> 0, so the Fan-Migdal
# linewidth has the closed form
#   Gamma_nk = pi/(2 omega0 M) sum_m |G_mn|^2 [ (n_B + f(E+)) rho_m(E+) + (n_B + 1 - f(E-)) rho_m(E-) ],
# E+- = eps_nk +- omega0 (absorption lands at E+, emission at E-).  The Gaussian delta converges
# as sigma^2 (Gamma(sigma) = Gamma_0 + c sigma^2 + O(sigma^4)), so two widths and one Richardson
# step reach the limit to ~1e-6.
_LW_BANDS = ((0.0, 0.5), (0.3, -0.4))
_LW_G = np.array([[0.3 + 0.2j, -0.5 + 0.1j], [0.7j, 0.25]])
_LW_W0, _LW_M = 0.06, 20.0


def _chain_dos(E, e0, t):
    return 1.0 / (np.pi * np.sqrt(4.0 * t * t - (E - e0) ** 2))


def _einstein_chain_linewidths(kx, kT, mu, sigmas, nq=20000, seed=5):
    rng = np.random.default_rng(seed)
    q = np.arange(nq) / nq
    eps_k = np.stack([e0 + 2 * t * np.cos(2 * np.pi * kx) for e0, t in _LW_BANDS], -1)
    eps_kq = np.stack([e0 + 2 * t * np.cos(2 * np.pi * (kx[None, :] + q[:, None])) for e0, t in _LW_BANDS], -1)
    omega = np.full((nq, 3), _LW_W0)
    e, _ = np.linalg.qr(rng.standard_normal((nq, 3, 3)) + 1j * rng.standard_normal((nq, 3, 3)))
    g = _LW_G[None, None, None] * (e[:, 0, :] / np.sqrt(_LW_M))[:, None, :, None, None]
    g = np.broadcast_to(g, (nq, len(kx), 3, 2, 2)).copy()
    wq = np.full(nq, 1.0 / nq)
    return eps_k, [oracle.linewidths(eps_k, eps_kq, omega, g, wq, kT, mu, s, 1e-6) for s in sigmas]


def test_linewidths_sigma_to_zero_limit_on_chain_bands():
    kx = np.array([0.13, 0.23, 0.29])
    kT, mu = 0.025852, 0.1
    eps_k, (g1, g2) = _einstein_chain_linewidths(kx, kT, mu, (0.004, 0.002))
    gamma0 = (4.0 * g2 - g1) / 3.0  # Richardson: removes the sigma^2 term
    nB = 1.0 / (math.exp(_LW_W0 / kT) - 1.0)
    occ = lambda E: 1.0 / (np.exp((E - mu) / kT) + 1.0)
    expect = np.zeros_like(gamma0)
    for n in range(2):
        Ep, Em = eps_k[:, n] + _LW_W0, eps_k[:, n] - _LW_W0
        for m, (e0, t) in enumerate(_LW_BANDS):
            expect[:, n] += np.pi * abs(_LW_G[m, n]) ** 2 / (2 * _LW_W0 * _LW_M) * (
                (nB + occ(Ep)) * _chain_dos(Ep, e0, t) + (nB + 1.0 - occ(Em)) * _chain_dos(Em, e0, t))
    assert np.abs(gamma0 / expect - 1.0).max() < 2e-5


def test_linewidths_detailed_balance_at_the_chemical_potential():
    # For eps_nk = mu the absorption weight n_B + f(mu + w) and the emission weight
    # n_B + 1 - f(mu - w) are both 1/(e^x - 1) + 1/(e^x + 1) = 1/sinh(x), x = w/kT, so
    # Gamma = pi/(2 w M) csch(w/kT) sum_m |G_mn|^2 [rho_m(mu + w) + rho_m(mu - w)].
    kx = np.array([0.23])
    kT = 0.025852
    mu = _LW_BANDS[0][0] + 2 * _LW_BANDS[0][1] * math.cos(2 * math.pi * 0.23)  # eps of band 0 at k = 0.23
    eps_k, (g1, g2) = _einstein_chain_linewidths(kx, kT, mu, (0.004, 0.002))
    assert abs(eps_k[0, 0] - mu) < 1e-15
    gamma0 = (4.0 * g2 - g1) / 3.0
    expect = sum(np.pi * abs(_LW_G[m, 0]) ** 2 / (2 * _LW_W0 * _LW_M) / math.sinh(_LW_W0 / kT)
                 * (_chain_dos(mu + _LW_W0, e0, t) + _chain_dos(mu - _LW_W0, e0, t))
                 for m, (e0, t) in enumerate(_LW_BANDS))
    assert abs(gamma0[0, 0] / expect - 1.0) < 2e-5


def test_linewidths_zero_temperature_limit():
    # kT -> 0: no thermal phonons (n_B -> 0) and step occupations.  An electron above mu + w
    # can only emit (Gamma ~ rho(eps - w)); a hole below mu - w is filled only through the
    # absorption term, whose final states at eps + w are occupied (Gamma ~ rho(eps + w)).
    kx = np.array([0.13, 0.23, 0.29])
    kT, mu = 0.003, 0.0
    eps_k, (g1, g2) = _einstein_chain_linewidths(kx, kT, mu, (0.004, 0.002))
    gamma0 = (4.0 * g2 - g1) / 3.0
    expect = np.zeros_like(gamma0)
    for i in range(len(kx)):
        for n in range(2):
            e = eps_k[i, n]
            assert abs(e - mu) > _LW_W0 + 20 * kT  # occupations are 0 or 1 to e^-20
            E = e - _LW_W0 if e > mu else e + _LW_W0
            expect[i, n] = sum(np.pi * abs(_LW_G[m, n]) ** 2 / (2 * _LW_W0 * _LW_M) * _chain_dos(E, e0, t)
                               for m, (e0, t) in enumerate(_LW_BANDS))
    assert np.abs(gamma0 / expect - 1.0).max() < 2e-5


def test_linewidths_properties():
    # modes at or below omega_min contribute nothing; Gamma >= 0 and linear in the q weights
    kT = 0.025852
    eps_k = np.array([[0.17]])
    eps_kq = np.array([[[0.13]]])
    g = np.full((1, 1, 1, 1, 1), 0.3 + 0.4j)
    assert oracle.linewidths(eps_k, eps_kq, np.array([[0.05]]), g, [1.0], kT, 0.1, 0.02, 0.06)[0, 0] == 0.0
    assert oracle.linewidths(eps_k, eps_kq, np.array([[0.05]]), g, [1.0], kT, 0.1, 0.02, 0.04)[0, 0] > 0.0
    wl = synth.make_workload("si_tiny", nk=5, nq=3)
    ek, ekq, om, gg = oracle.interpolate(wl)
    G1 = oracle.linewidths(ek, ekq, om, gg, [1.0, 2.0, 0.5], kT, 0.0, 0.1, 1e-6)
    G2 = oracle.linewidths(ek, ekq, om, gg, [2.0, 4.0, 1.0], kT, 0.0, 0.1, 1e-6)
    assert np.all(G1 >= 0) and np.abs(G2 - 2 * G1).max() < 1e-13 * np.abs(G1).max()


# ---------------------------------------------------------------- time-reversal k reduction
@pytest.mark.parametrize("n,shift", [((4, 4, 4), (0, 0, 0)), ((5, 3, 1), (0, 0, 0)), ((6, 4, 2), (0.5 / 6, 0, 0.25)),
                                     ((2, 2, 2), (0, 0, 0)), ((7, 1, 1), (0.5 / 7, 0, 0))])
def test_ibz_time_reversal_counts_and_weights(n, shift):
    idx, w = oracle.ibz_time_reversal(n, shift)
    N = n[0] * n[1] * n[2]
    # points equal to their own partner: 2 j_a + t_a = 0 mod n_a on every axis (t_a = 2 s_a n_a)
    nself = 1
    for na, sa in zip(n, shift):
        t = int(round(2 * sa * na))
        nself *= sum(1 for j in range(na) if (2 * j + t) % na == 0)
    assert len(idx) == (N + nself) // 2
    assert w.sum() == N and set(np.unique(w)) <= {1.0, 2.0} and (w == 1.0).sum() == nself
    assert np.all(np.diff(idx) > 0)


def test_ibz_time_reversal_preserves_grid_sums_for_real_hamiltonians():
    wl = synth.make_workload("si_tiny", nb=5, real_h=True)
    n = (4, 3, 5)
    k = oracle.grid_points(n)
    eps, _ = oracle.electron_eigen(oracle.hamiltonian_k(k, wl.Re, wl.we, wl.H_Re))
    epm, _ = oracle.electron_eigen(oracle.hamiltonian_k(-k, wl.Re, wl.we, wl.H_Re))
    assert np.abs(eps - epm).max() < 1e-13 * np.abs(eps).max()        # eps(-k) = eps(k)
    idx, w = oracle.ibz_time_reversal(n)
    f = 1.0 / (np.exp((eps - 0.3) / 0.05) + 1.0)
    assert abs((w[:, None] * f[idx]).sum() - f.sum()) < 1e-12 * f.sum()
    assert abs((w[:, None] * eps[idx] ** 2).sum() - (eps ** 2).sum()) < 1e-12 * (eps ** 2).sum()
    # a complex H(R) has no such symmetry: the reduction would be wrong there
    wc = synth.make_workload("si_tiny", nb=5)
    ec, _ = oracle.electron_eigen(oracle.hamiltonian_k(k, wc.Re, wc.we, wc.H_Re))
    ecm, _ = oracle.electron_eigen(oracle.hamiltonian_k(-k, wc.Re, wc.we, wc.H_Re))
    assert np.abs(ec - ecm).max() > 1e-3
