"""Planted mistakes in the oracle must each fail at least one pin.

Each mutation replaces one oracle function (on the CPU) by a plausible wrong
variant: a flipped phase sign, a missing conjugate, a transposed operand, a
dropped mass factor or weight, a wrong eigenvalue order or sign, k - q for k + q.  The pins in test_oracle_pins.py are then run against the
mutated oracle and at least one of them has to fail.
"""
import numpy as np
import pytest

import oracle
import oracle.eph_oracle as eo
from tests import test_oracle_pins as pins

PIN_FUNCS = [
    pins.test_phase_properties,
    pins.test_one_band_chain_closed_form,
    pins.test_spring_chain_closed_form,
    pins.test_single_R_plane_wave_closed_form,
    pins.test_nested_equals_single_loop,
    pins.test_wannier_round_trip,
    pins.test_unitarity_invariant_and_periodicity,
    pins.test_vjp_is_the_adjoint_of_the_interpolation,
    pins.test_unstable_spring_chain_negative_frequency,
    pins.test_complex_hopping_and_diatomic_chain_closed_forms,
    pins.test_loss_closed_form_on_plane_wave,
    pins.test_linewidths_sigma_to_zero_limit_on_chain_bands,
    pins.test_linewidths_detailed_balance_at_the_chemical_potential,
    pins.test_linewidths_zero_temperature_limit,
    pins.test_linewidths_properties,
    lambda: pins.test_ibz_time_reversal_counts_and_weights((4, 4, 4), (0, 0, 0)),
    pins.test_ibz_time_reversal_preserves_grid_sums_for_real_hamiltonians,
]

_orig_phases = eo.phases
_orig_g_req = eo.g_req_to_bloch
_orig_phonon = eo.phonon_eigen
_orig_vjp = eo.vjp
_orig_hk = eo.hamiltonian_k
_orig_dq = eo.dynamical_matrix
_orig_eig = eo.electron_eigen
_orig_g1 = eo.g_rp_to_q
_orig_loss_weights = eo.loss_weights
_orig_b2w = eo.g_bloch_to_wannier
_orig_linewidths = eo.linewidths
_orig_ibz = eo.ibz_time_reversal


def _phase_sign(pts, R, w=None):
    return _orig_phases(pts, R, w).conj()


def _phase_unreduced_wrong_scale(pts, R, w=None):
    # forgets the 2 pi (uses e^{i k.R} with k in crystal units)
    pts = np.asarray(pts, dtype=np.float64)
    t = pts @ np.asarray(R, dtype=np.float64).T
    P = np.exp(1j * t)
    return P if w is None else P * np.asarray(w)[None, :]


def _g_req_no_conj(kpts, Re, we, G1q, V_k, V_kq, u_q):
    return _orig_g_req(kpts, Re, we, G1q, V_k, V_kq.conj(), u_q)


def _g_req_swap_gauges(kpts, Re, we, G1q, V_k, V_kq, u_q):
    return _orig_g_req(kpts, Re, we, G1q, V_kq, V_k, u_q)


def _g_req_u_transposed(kpts, Re, we, G1q, V_k, V_kq, u_q):
    return _orig_g_req(kpts, Re, we, G1q, V_k, V_kq, u_q.T)


def _phonon_no_mass(Dq, masses):
    om, e, u = _orig_phonon(Dq, masses)
    return om, e, e


def _vjp_u_unconjugated(a, kpts, qpts, gbar, ev):
    return _orig_vjp(a, kpts, qpts, gbar, dict(ev, u=ev["u"].conj()))


def _vjp_kq_gauge_conjugated(a, kpts, qpts, gbar, ev):
    return _orig_vjp(a, kpts, qpts, gbar, dict(ev, V_kq=ev["V_kq"].conj()))


def _hk_minus_k(kpts, Re, we, H_Re):
    # e^{-ik.R} in H(k): the same spectrum only with time-reversal symmetry
    return _orig_hk(-np.asarray(kpts), Re, we, H_Re)


def _hk_transposed(kpts, Re, we, H_Re):
    return _orig_hk(kpts, Re, we, np.ascontiguousarray(np.swapaxes(H_Re, 1, 2)))


def _hk_no_weight(kpts, Re, we, H_Re):
    return _orig_hk(kpts, Re, None, H_Re)


def _dq_minus_q(qpts, Rp, wp, Phi_Rp, masses):
    # e^{-iq.Rp} in D(q): same frequencies (real force constants), conjugated mode vectors
    return _orig_dq(-np.asarray(qpts), Rp, wp, Phi_Rp, masses)


def _dq_without_masses(qpts, Rp, wp, Phi_Rp, masses):
    return _orig_dq(qpts, Rp, wp, Phi_Rp, np.ones(len(masses)))


def _eig_descending(Hk):
    e, V = _orig_eig(Hk)
    return e[..., ::-1], V[..., ::-1]


def _omega_unsigned(Dq, masses):
    om, e, u = _orig_phonon(Dq, masses)
    return np.abs(om), e, u


def _mode_vector_times_mass(Dq, masses):
    om, e, u = _orig_phonon(Dq, masses)
    return om, e, e * np.sqrt(np.repeat(np.asarray(masses, dtype=np.float64), 3))[None, :, None]


def _g1_no_weight(qpts, Rp, wp, g_ReRp):
    return _orig_g1(qpts, Rp, None, g_ReRp)


def _g_req_bands_swapped(kpts, Re, we, G1q, V_k, V_kq, u_q):
    return np.swapaxes(_orig_g_req(kpts, Re, we, G1q, V_k, V_kq, u_q), 2, 3)


def _interpolate_k_minus_q(a, kpts=None, qpts=None, return_eigvecs=False):
    # the oracle's steps with H(k - q) in place of H(k + q)
    kpts = a.kpts if kpts is None else np.asarray(kpts, dtype=np.float64)
    qpts = a.qpts if qpts is None else np.asarray(qpts, dtype=np.float64)
    eps_k, V_k = eo.electron_eigen(eo.hamiltonian_k(kpts, a.Re, a.we, a.H_Re))
    omega, _, u = eo.phonon_eigen(eo.dynamical_matrix(qpts, a.Rp, a.wp, a.Phi_Rp, a.masses), a.masses)
    G1 = eo.g_rp_to_q(qpts, a.Rp, a.wp, a.g_ReRp)
    eps_kq, g, vkq = [], [], []
    for iq in range(len(qpts)):
        e_kq, V_kq = eo.electron_eigen(eo.hamiltonian_k(kpts - qpts[iq][None, :], a.Re, a.we, a.H_Re))
        eps_kq.append(e_kq)
        vkq.append(V_kq)
        g.append(eo.g_req_to_bloch(kpts, a.Re, a.we, G1[iq], V_k, V_kq, u[iq]))
    out = (eps_k, np.stack(eps_kq), omega, np.stack(g))
    return out + (dict(V_k=V_k, V_kq=np.stack(vkq), u=u),) if return_eigvecs else out


def _loss_weights_omega_squared(omega, w_nk, omega_min):
    c = _orig_loss_weights(omega, w_nk, omega_min)
    return c / np.where(omega > omega_min, omega, 1.0)[:, None, :, None]


def _loss_k_plus_q_band(g, omega, w_nk, omega_min):
    # the weight w_nk applied on the band index of the k+q side (m) instead of the k side (n)
    c = eo.loss_weights(omega, w_nk, omega_min)
    return float(np.sum(c[:, :, :, :, None] * np.abs(g) ** 2))


def _eq6_unnormalised(kc, qc, Re, Rp, g_bloch, V_k, V_kq, u_q):
    # Eq. 6 without its 1/(Ne Np)
    return _orig_b2w(kc, qc, Re, Rp, g_bloch, V_k, V_kq, u_q) * (len(Re) * len(Rp))


def _eq6_forward_phases(kc, qc, Re, Rp, g_bloch, V_k, V_kq, u_q):
    # e^{+i(k'.Re + q'.Rp)} in the back transform: the same grid read as -k', -q'
    return _orig_b2w(-np.asarray(kc), -np.asarray(qc), Re, Rp, g_bloch, V_k, V_kq, u_q)


def _swap_terms(eps_k, eps_kq, omega, g, wq, kT, mu, sigma, omega_min):
    # phonon absorption weighted at the emission energy and vice versa
    om = np.asarray(omega)[:, None, :, None, None]
    ok = om > omega_min
    w = np.where(ok, om, 1.0)
    nB = eo.bose(w, kT)
    f = eo.fermi(np.asarray(eps_kq)[:, :, None, :, None], mu, kT)
    de = np.asarray(eps_k)[None, :, None, None, :] - np.asarray(eps_kq)[:, :, None, :, None]
    term = (nB + f) * eo.gaussian(de - w, sigma) + (nB + 1.0 - f) * eo.gaussian(de + w, sigma)
    c = np.where(ok, np.pi * np.abs(g) ** 2 / (2.0 * w), 0.0) * term
    return np.einsum("q,qkvmn->kn", np.ones(len(omega)) if wq is None else np.asarray(wq), c)


def _lw_no_half_omega(eps_k, eps_kq, omega, g, wq, kT, mu, sigma, omega_min):
    # drops the 1/(2 omega) of the coupling's zero-point amplitude (|g|^2 scaled by 2 omega
    # cancels it)
    scale = np.sqrt(2.0 * np.abs(np.asarray(omega)))[:, None, :, None, None]
    return _orig_linewidths(eps_k, eps_kq, omega, g * scale, wq, kT, mu, sigma, omega_min)


def _lw_g_transposed(eps_k, eps_kq, omega, g, wq, kT, mu, sigma, omega_min):
    # |g_nm| in place of |g_mn| (the k-side and k+q-side band indices exchanged)
    return _orig_linewidths(eps_k, eps_kq, omega, np.swapaxes(g, -1, -2), wq, kT, mu, sigma, omega_min)


def _lw_fermi_at_k(eps_k, eps_kq, omega, g, wq, kT, mu, sigma, omega_min):
    # occupation of the initial state n,k in place of the final state m,k+q
    om = np.asarray(omega)[:, None, :, None, None]
    ok = om > omega_min
    w = np.where(ok, om, 1.0)
    nB = eo.bose(w, kT)
    f = eo.fermi(np.asarray(eps_k)[None, :, None, None, :], mu, kT)
    de = np.asarray(eps_k)[None, :, None, None, :] - np.asarray(eps_kq)[:, :, None, :, None]
    term = (nB + f) * eo.gaussian(de + w, sigma) + (nB + 1.0 - f) * eo.gaussian(de - w, sigma)
    c = np.where(ok, np.pi * np.abs(g) ** 2 / (2.0 * w), 0.0) * term
    return np.einsum("q,qkvmn->kn", np.asarray(wq, dtype=np.float64), c)


def _ibz_partner_is_itself(n, shift=(0.0, 0.0, 0.0)):
    # forgets the negation: every point "pairs" with itself (nothing reduced, weights 1)
    N = n[0] * n[1] * n[2]
    return np.arange(N), np.ones(N)


def _ibz_weights_one(n, shift=(0.0, 0.0, 0.0)):
    idx, w = _orig_ibz(n, shift)
    return idx, np.ones_like(w)


MUTATIONS = {
    "phase_sign": ("phases", _phase_sign),
    "phase_missing_2pi": ("phases", _phase_unreduced_wrong_scale),
    "band_rotation_missing_conj": ("g_req_to_bloch", _g_req_no_conj),
    "band_rotation_swapped_gauges": ("g_req_to_bloch", _g_req_swap_gauges),
    "mode_rotation_transposed": ("g_req_to_bloch", _g_req_u_transposed),
    "mode_vector_without_mass": ("phonon_eigen", _phonon_no_mass),
    "vjp_mode_rotation_unconjugated": ("vjp", _vjp_u_unconjugated),
    "vjp_band_gauge_conjugated": ("vjp", _vjp_kq_gauge_conjugated),
    "hamiltonian_phase_sign": ("hamiltonian_k", _hk_minus_k),
    "hamiltonian_transposed": ("hamiltonian_k", _hk_transposed),
    "hamiltonian_without_weights": ("hamiltonian_k", _hk_no_weight),
    "dynamical_matrix_phase_sign": ("dynamical_matrix", _dq_minus_q),
    "dynamical_matrix_without_masses": ("dynamical_matrix", _dq_without_masses),
    "eigenvalues_descending": ("electron_eigen", _eig_descending),
    "unstable_mode_sign_dropped": ("phonon_eigen", _omega_unsigned),
    "mode_vector_times_mass": ("phonon_eigen", _mode_vector_times_mass),
    "eq9_without_weights": ("g_rp_to_q", _g1_no_weight),
    "band_indices_swapped": ("g_req_to_bloch", _g_req_bands_swapped),
    "k_minus_q": ("interpolate", _interpolate_k_minus_q),
    "loss_over_omega_squared": ("loss_weights", _loss_weights_omega_squared),
    "loss_weight_on_wrong_band": ("loss", _loss_k_plus_q_band),
    "eq6_without_normalisation": ("g_bloch_to_wannier", _eq6_unnormalised),
    "eq6_forward_phases": ("g_bloch_to_wannier", _eq6_forward_phases),
    "linewidth_terms_swapped": ("linewidths", _swap_terms),
    "linewidth_without_1_over_2omega": ("linewidths", _lw_no_half_omega),
    "linewidth_coupling_band_indices_swapped": ("linewidths", _lw_g_transposed),
    "linewidth_occupation_at_k": ("linewidths", _lw_fermi_at_k),
    "ibz_without_negation": ("ibz_time_reversal", _ibz_partner_is_itself),
    "ibz_unit_weights": ("ibz_time_reversal", _ibz_weights_one),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(eo, attr, fn)
    monkeypatch.setattr(oracle, attr, fn)
    caught = []
    for pin in PIN_FUNCS:
        try:
            pin()
        except AssertionError:
            caught.append(pin.__name__)
            break
    assert caught, f"mutation {name} passed every pin"
