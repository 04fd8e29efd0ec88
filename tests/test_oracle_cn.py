"""Pins of the Crank-Nicolson coefficient propagation of the oracle (Eq. 5).

Each pin fixes the scheme by something other than the oracle itself:
  CN-1  time-independent H (no SCC, constant A): n steps equal the closed form
        V diag(((1 - i t e)/(1 + i t e))^n) V^dagger S C0 from the generalized
        eigenpairs H V = S V e (t = dt/2), the Cayley map of each eigenvalue;
  CN-2  with a pulse and the SCC term, C_k^dagger S_k C_k stays the identity
        (the scheme is unitary in the S metric) and the electron count stays N_el;
  CN-3  the SCC ground state does not move without a field;
  CN-4  against a fine RK4 integration of Eq. 6 with the SCC shift at every
        stage, the error falls four-fold per halving of dt (second order: a
        Hamiltonian taken at t_n instead of t_{n+1/2}, or a shift that is not
        extrapolated, falls two-fold).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from oracle import crank_nicolson as cn
from paper_2308_09782_gb300 import inputs

C_LIGHT = 137.035999084


@pytest.fixture(scope="module")
def si8d():
    """Distorted 8-atom cell (charge transfer present), MP 2x2x2, with its ground state."""
    s = inputs.diamond_si(1, sigma=0.3, seed=5, kgrid="mp2", dt=0.2)
    ctx = O.setup(s)
    return s, ctx, O.ground_state(s, ctx=ctx)


@pytest.fixture(scope="module")
def si8d_nonscc():
    s = inputs.diamond_si(1, sigma=0.3, seed=5, kgrid="mp2", dt=0.2, gamma_scale=0.0)
    ctx = O.setup(s)
    return s, ctx, O.ground_state(s, ctx=ctx)


def test_cn1_closed_form_time_independent(si8d_nonscc):
    s, ctx, gs = si8d_nonscc
    A = np.array([7.0, -4.0, 3.0])
    n = 60
    r = cn.propagate_cn(s, np.tile(A, (n + 1, 1)), n, gs["C"], ctx=ctx)
    theta = 0.5 * s["dt"]
    for ik in range(len(ctx["S"])):
        S, H0, P = ctx["S"][ik], ctx["H0"][ik], ctx["P"][ik]
        H = H0 + (A[0] * P[0] + A[1] * P[1] + A[2] * P[2]) / C_LIGHT
        e, VS = sla.eigh(H, S)          # H VS = S VS e,  VS^dagger S VS = 1
        lam = (1.0 - 1j * theta * e) / (1.0 + 1j * theta * e)
        Cn = VS @ (lam[:, None] ** n * (VS.conj().T @ S @ gs["C"][ik]))
        assert np.abs(r["C"][ik] - Cn).max() <= 1e-12 * np.abs(Cn).max()
    # the states really moved (A.P does not commute with H0)
    assert max(np.abs(r["C"][ik] - gs["C"][ik]).max() for ik in range(len(ctx["S"]))) > 1e-3


def test_cn2_unitary_in_s_metric(si8d):
    s, ctx, gs = si8d
    n = 100
    A = inputs.pulse_field(n, s["dt"], 0.05, 0.3)
    r = cn.propagate_cn(s, A, n, gs["C"], ctx=ctx)
    for ik, C in enumerate(r["C"]):
        G = C.conj().T @ ctx["S"][ik] @ C
        assert np.abs(G - np.eye(G.shape[0])).max() <= 1e-12
    nel = float(s["n_electrons"])
    assert np.abs(r["q"].sum(axis=1) - nel).max() <= 1e-11 * nel
    assert np.abs(r["J"]).max() > 1e-6        # the pulse drove a current


def test_cn3_ground_state_stationary(si8d):
    s, ctx, gs = si8d
    n = 40
    r = cn.propagate_cn(s, np.zeros((n + 1, 3)), n, gs["C"], ctx=ctx)
    D = cn.density(r["C"])
    for ik in range(len(D)):
        assert np.abs(D[ik] - gs["D"][ik]).max() <= 1e-10
    assert np.abs(r["q"] - r["q"][0]).max() <= 1e-10
    assert np.abs(r["J"]).max() <= 1e-10


# ---------------------------------------------------------------------------
# CN-4: order of accuracy against RK4 on Eq. 6
# ---------------------------------------------------------------------------
T_END, E0, W = 8.0, 0.05, 0.3


def _rk4_reference(s, ctx, gs, dt):
    """Classical RK4 on Eq. 6, A(t) from the closed-form pulse, SCC shift at every stage."""
    n = int(round(T_END / dt))
    A = inputs.pulse_field(2 * n, dt / 2, E0, W, duration=T_END)

    def rhs(D, j):
        _, _, _, eps_orb = O.observables(ctx, D, A[j])
        return [O.ddot(D[ik], O.hamiltonian(ctx["H0"][ik], ctx["S"][ik], ctx["P"][ik], A[j], eps_orb),
                       ctx["Sinv"][ik]) for ik in range(len(D))]

    D = [d.copy() for d in gs["D"]]
    for m in range(n):
        k1 = rhs(D, 2 * m)
        k2 = rhs([d + 0.5 * dt * k for d, k in zip(D, k1)], 2 * m + 1)
        k3 = rhs([d + 0.5 * dt * k for d, k in zip(D, k2)], 2 * m + 1)
        k4 = rhs([d + dt * k for d, k in zip(D, k3)], 2 * m + 2)
        D = [d + dt / 6.0 * (a + 2 * b + 2 * c + e) for d, a, b, c, e in zip(D, k1, k2, k3, k4)]
    return D


def cn_errors(s, ctx, gs, D_ref, dts=(0.2, 0.1, 0.05)):
    errs = []
    for dt in dts:
        sd = dict(s)
        sd["dt"] = dt
        n = int(round(T_END / dt))
        A = inputs.pulse_field(n, dt, E0, W, duration=T_END)
        r = cn.propagate_cn(sd, A, n, gs["C"], ctx=ctx)
        D = cn.density(r["C"])
        errs.append(np.sqrt(sum(np.linalg.norm(a - b) ** 2 for a, b in zip(D, D_ref))))
    return errs


@pytest.fixture(scope="module")
def rk4_ref(si8d):
    s, ctx, gs = si8d
    return _rk4_reference(s, ctx, gs, 0.0125)


def test_cn4_second_order(si8d, rk4_ref):
    s, ctx, gs = si8d
    e = cn_errors(s, ctx, gs, rk4_ref)
    assert 3.5 <= e[0] / e[1] <= 4.5 and 3.5 <= e[1] / e[2] <= 4.5, e
