"""Planted mistakes in the oracle must each fail at least one pin.

Each mutation replaces one oracle function (on the CPU) by a plausible wrong
variant: a flipped phase sign, a missing conjugate, a transposed operand, a
dropped mass factor.  The pins in test_oracle_pins.py are then run against the
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
]

_orig_phases = eo.phases
_orig_g_req = eo.g_req_to_bloch
_orig_phonon = eo.phonon_eigen
_orig_vjp = eo.vjp


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


MUTATIONS = {
    "phase_sign": ("phases", _phase_sign),
    "phase_missing_2pi": ("phases", _phase_unreduced_wrong_scale),
    "band_rotation_missing_conj": ("g_req_to_bloch", _g_req_no_conj),
    "band_rotation_swapped_gauges": ("g_req_to_bloch", _g_req_swap_gauges),
    "mode_rotation_transposed": ("g_req_to_bloch", _g_req_u_transposed),
    "mode_vector_without_mass": ("phonon_eigen", _phonon_no_mass),
    "vjp_mode_rotation_unconjugated": ("vjp", _vjp_u_unconjugated),
    "vjp_band_gauge_conjugated": ("vjp", _vjp_kq_gauge_conjugated),
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
    assert caught, f"mutation {name} passed every pin"
