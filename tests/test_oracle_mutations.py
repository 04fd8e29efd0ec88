"""Planted mistakes in the oracle must be caught by at least one pin.

Each case monkeypatches one oracle function with a plausible error (sign of
Eq. 6, the 1/2 of Eq. 10, the sign of Eq. 14, a transposed momentum block,
a missing |A|^2 term in the energy, a missing diamagnetic current, the sign of
the A.P term) and checks that the pin aimed at it fails.  Everything
here runs on the CPU.
"""
import numpy as np
import pytest

import oracle as O
from oracle import vgtb_oracle as ov
from paper_2308_09782_gb300 import inputs
from oracle import crank_nicolson as ocn
from tests import test_oracle_pins as pins
from tests import test_oracle_cn as cnpins

C = ov.C_LIGHT


def _si8():
    s, A, n = inputs.config("si8_pulse")
    ctx = O.setup(s)
    gs = O.ground_state(s, ctx=ctx)
    return s, A, n, ctx, gs


def _wrong_sign_ddot(D, H, Sinv):
    return 1j * (Sinv @ H @ D - D @ H @ Sinv)


def _no_half_h2(H0, S, P, A, eps_orb):
    A = np.asarray(A, float)
    H = H0 + (eps_orb[:, None] * S + S * eps_orb[None, :])
    H = H + (A[0] * P[0] + A[1] * P[1] + A[2] * P[2]) / C
    return H + (A @ A) / (2.0 * C ** 2) * S


def _minus_ap(H0, S, P, A, eps_orb):
    A = np.asarray(A, float)
    H = H0 + 0.5 * (eps_orb[:, None] * S + S * eps_orb[None, :])
    H = H - (A[0] * P[0] + A[1] * P[1] + A[2] * P[2]) / C
    return H + (A @ A) / (2.0 * C ** 2) * S


def _energy_no_a2(D_list, H0_list, P_list, S_list, A, wk, gamma, dq):
    A = np.asarray(A, float)
    e = 0.0
    for D, H0, P, S, w in zip(D_list, H0_list, P_list, S_list, wk):
        Hn = H0 + (A[0] * P[0] + A[1] * P[1] + A[2] * P[2]) / C
        e += w * np.real(np.sum(D * Hn.T))
    return e + 0.5 * dq @ gamma @ dq


def _current_no_diamagnetic(D_list, P_list, S_list, A, omega, wk):
    J = np.zeros(3)
    for D, P, S, w in zip(D_list, P_list, S_list, wk):
        for a in range(3):
            J[a] += w * np.real(np.sum(D * P[a].T))
    return -J / omega


def _plus_current(D_list, P_list, S_list, A, omega, wk):
    J = np.zeros(3)
    for D, P, S, w in zip(D_list, P_list, S_list, wk):
        for a in range(3):
            J[a] += w * np.real(np.sum(D * (P[a] + (A[a] / C) * S).T))
    return J / omega


_orig_bloch = ov.bloch_matrices


def _transposed_p(sysd, kred):
    S, H0, P = _orig_bloch(sysd, kred)
    return S, H0, P.transpose(0, 2, 1).copy()


def _cn_backward(S, H, Cc, theta):
    return np.linalg.solve(S - 1j * theta * H, (S + 1j * theta * H) @ Cc)


def _cn_full_dt(S, H, Cc, theta):
    return np.linalg.solve(S + 2j * theta * H, (S - 2j * theta * H) @ Cc)


def _cn_orthogonal(S, H, Cc, theta):
    one = np.eye(S.shape[0])
    return np.linalg.solve(one + 1j * theta * H, (one - 1j * theta * H) @ Cc)


def _cn_h_at_tn(A_table, n, eps_n, eps_prev):
    return np.asarray(A_table[n], float), eps_n


def _cn_shift_not_extrapolated(A_table, n, eps_n, eps_prev):
    return 0.5 * (np.asarray(A_table[n], float) + np.asarray(A_table[n + 1], float)), eps_n


@pytest.mark.parametrize("mutant,pin", [
    (("cn_step", _cn_backward), "cn1"),
    (("cn_step", _cn_full_dt), "cn1"),
    (("cn_step", _cn_orthogonal), "cn2"),
    (("cn_midpoint", _cn_h_at_tn), "cn4"),
    (("cn_midpoint", _cn_shift_not_extrapolated), "cn4"),
])
def test_cn_pin_catches_planted_mistake(monkeypatch, mutant, pin):
    monkeypatch.setattr(ocn, mutant[0], mutant[1])
    with pytest.raises(AssertionError):
        if pin == "cn1":
            cnpins.test_cn1_closed_form_time_independent(cnpins.si8d_nonscc.__wrapped__())
        elif pin == "cn2":
            cnpins.test_cn2_unitary_in_s_metric(cnpins.si8d.__wrapped__())
        elif pin == "cn4":
            d = cnpins.si8d.__wrapped__()
            cnpins.test_cn4_second_order(d, cnpins._rk4_reference(*d, 0.0125))


@pytest.mark.parametrize("target,mutant,pin", [
    ("ddot", _wrong_sign_ddot, "p6"),
    ("hamiltonian", _no_half_h2, "p14"),
    ("energy", _energy_no_a2, "p4"),
    ("current", _plus_current, "p8"),
    ("current", _current_no_diamagnetic, "p8"),
    ("bloch_matrices", _transposed_p, "p14"),
    ("hamiltonian", _minus_ap, "p13"),
])
def test_pin_catches_planted_mistake(monkeypatch, target, mutant, pin):
    monkeypatch.setattr(ov, target, mutant)
    with pytest.raises(AssertionError):
        if pin == "p6":
            pins.test_p6_leapfrog_closed_form_constant_hamiltonian()
        elif pin == "p14":
            pins.test_p14_brute_force_loops_gamma()
        elif pin == "p4":
            pins.test_p4_a_squared_term_is_a_pure_phase(_si8())
        elif pin == "p8":
            pins.test_p8_work_theorem_second_order(_si8())
        elif pin == "p13":
            pins.test_p13_constant_a_is_a_gauge_transformation_to_first_order()
