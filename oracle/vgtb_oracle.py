"""Plain FP64 CPU oracle for velocity-gauge real-time TDDFTB propagation.

TEST INFRASTRUCTURE ONLY.  This module is imported by the test-suite, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
library's propagation path never imports, links or calls it.  It shares no code
with the CUDA path: it reads the same input dictionaries (system blocks, A(t)
tables) and restates the paper's equations with dense complex128 numpy
matrices, in the order the paper gives them.

Equations (Xu et al., "Velocity-gauge real-time TDDFTB", Sec. 2):
  Eq. 3   A(t) = -c int_0^t E            (input tables; see tests for pins)
  Eq. 6   i dD_k/dt = S_k^-1 H_k D_k - D_k H_k S_k^-1
  Eq. 7   S_k = sum_L exp(-i k.L) S(L)
  Eq. 8   H_k = sum_L exp(-i k.L) H(L)
  Eq. 9   H(L) = H0(L) + H2(L) + Hext(L)
  Eq. 10  H2^{mu nu}(L) = 1/2 S^{mu nu}(L) sum_K (gamma_IK + gamma_JK) dq_K,
          q_I = (1/N_k) sum_k sum_{mu in I} [D_k S_k]^{mu mu}, dq = q - Z
  Eq. 12  Hext(L) = (1/c) A.<phi^L_mu|p|phi^0_nu> + |A|^2/(2c^2) S(L),
          <phi^L_mu|p|phi^0_nu> = i d S(L)/d R_J
  Eq. 13  D(t+dt) = D(t-dt) + 2 dt dD/dt(t)             (leapfrog)
  Eq. 14  J(t) = -(1/(Omega N_k)) sum_k Tr[D_k Pi_k],
          Pi_k = sum_L exp(-i k.L) <phi^L|p|phi^0> + (1/c) A S_k

Readings where the paper is silent (also listed in the design notes):
  * the leapfrog start is one forward-Euler step, D(dt) = D(0) + dt D'(0);
  * D_k carries the occupation numbers f_n in {0, 2}, so Tr(D_k S_k) = N_el;
  * k-weights w_k (equal, 1/N_k) replace 1/N_k;
  * traces and Mulliken diagonals take the real part (the "+ c.c." of Eq. 10
    and Eq. 14);
  * the SCC shift at t_n is computed from D(t_n);
  * energy E = sum_k w_k Re Tr[D_k (H0_k + (A/c).P_k + |A|^2/(2c^2) S_k)]
    + 1/2 dq^T gamma dq (second-order SCC-DFTB energy without repulsion);
  * the ground state occupies the lowest N_el/2 generalized eigenstates of
    H_k C = S_k C eps at every k with f = 2, iterated to charge
    self-consistency with Anderson mixing of dq.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

C_LIGHT = 137.035999084


# ----------------------------------------------------------------------------
# Real-space blocks -> k-space matrices (Eqs. 7, 8, 12)
# ----------------------------------------------------------------------------
def _block_views(sysd):
    """Yield (I, J, n, h0_blk, s_blk, ds_blk[3]) for every real-space block."""
    off = np.asarray(sysd["orb_offset"])
    ijl = np.asarray(sysd["blk_ijl"])
    h0, s, ds = sysd["h0"], sysd["s"], sysd["ds"]
    pos = 0
    for row in ijl:
        i, j = int(row[0]), int(row[1])
        ni, nj = off[i + 1] - off[i], off[j + 1] - off[j]
        sz = ni * nj
        yield (i, j, row[2:5].astype(float),
               h0[pos:pos + sz].reshape(ni, nj),
               s[pos:pos + sz].reshape(ni, nj),
               ds[:, pos:pos + sz].reshape(3, ni, nj))
        pos += sz


def bloch_matrices(sysd, kred):
    """Return S_k, H0_k and the momentum matrices P_k[3] at reduced k.

    Eq. 7 / Eq. 8: X_k^{mu nu} = sum_L exp(-i k.L) X^{mu nu}(L) with
    k.L = 2 pi k_red . n for L = n1 a1 + n2 a2 + n3 a3; block (I, J, L) goes to
    rows of atom I and columns of atom J.  Eq. 12: the momentum block is
    <phi^L_mu|p|phi^0_nu> = i dS^{mu nu}(L)/dR_J.
    """
    off = np.asarray(sysd["orb_offset"])
    n = int(off[-1])
    S = np.zeros((n, n), complex)
    H0 = np.zeros((n, n), complex)
    P = np.zeros((3, n, n), complex)
    kred = np.asarray(kred, float)
    for i, j, nvec, h0b, sb, dsb in _block_views(sysd):
        ph = np.exp(-2j * np.pi * float(kred @ nvec))
        r = slice(off[i], off[i + 1])
        c = slice(off[j], off[j + 1])
        S[r, c] += ph * sb
        H0[r, c] += ph * h0b
        P[:, r, c] += ph * 1j * dsb
    return S, H0, P


def orbital_atom(sysd):
    """Atom index of every orbital (the map mu -> I of mu = (I, l, m))."""
    off = np.asarray(sysd["orb_offset"])
    return np.repeat(np.arange(len(off) - 1), np.diff(off))


# ----------------------------------------------------------------------------
# Charges and the SCC shift (Eq. 10)
# ----------------------------------------------------------------------------
def mulliken(D_list, S_list, wk, atom_of):
    """q_I = sum_k w_k sum_{mu in I} Re [D_k S_k]^{mu mu} (Eq. 10 text)."""
    nat = int(atom_of.max()) + 1
    q = np.zeros(nat)
    for D, S, w in zip(D_list, S_list, wk):
        diag = np.real(np.einsum("ij,ji->i", D, S))
        q += w * np.bincount(atom_of, weights=diag, minlength=nat)
    return q


def scc_shift(gamma, dq):
    """eps_I = sum_K gamma_IK dq_K, so that H2 = 1/2 S (eps_I + eps_J) (Eq. 10)."""
    return gamma @ dq


def hamiltonian(H0, S, P, A, eps_orb):
    """H_k(t) by Eqs. 9, 10, 12 for one k.

    H = H0 + 1/2 (diag(eps) S + S diag(eps)) + (1/c) A.P + |A|^2/(2c^2) S.
    """
    A = np.asarray(A, float)
    H = H0 + 0.5 * (eps_orb[:, None] * S + S * eps_orb[None, :])
    H = H + (A[0] * P[0] + A[1] * P[1] + A[2] * P[2]) / C_LIGHT
    H = H + (A @ A) / (2.0 * C_LIGHT ** 2) * S
    return H


# ----------------------------------------------------------------------------
# Equation of motion and integrator (Eqs. 6, 13)
# ----------------------------------------------------------------------------
def ddot(D, H, Sinv):
    """dD/dt = -i (S^-1 H D - D H S^-1) (Eq. 6)."""
    return -1j * (Sinv @ H @ D - D @ H @ Sinv)


# ----------------------------------------------------------------------------
# Observables (Eq. 14 and the energy reading)
# ----------------------------------------------------------------------------
def current(D_list, P_list, S_list, A, omega, wk):
    """J_a = -(1/Omega) sum_k w_k Re Tr[D_k Pi_k^a], Pi^a = P^a + (A_a/c) S (Eq. 14)."""
    J = np.zeros(3)
    for D, P, S, w in zip(D_list, P_list, S_list, wk):
        for a in range(3):
            Pi = P[a] + (A[a] / C_LIGHT) * S
            J[a] += w * np.real(np.sum(D * Pi.T))       # Tr[D Pi]
    return -J / omega


def energy(D_list, H0_list, P_list, S_list, A, wk, gamma, dq):
    """E = sum_k w_k Re Tr[D_k(H0 + (A/c).P + |A|^2/(2c^2) S)] + 1/2 dq.gamma.dq."""
    A = np.asarray(A, float)
    e = 0.0
    for D, H0, P, S, w in zip(D_list, H0_list, P_list, S_list, wk):
        Hn = H0 + (A[0] * P[0] + A[1] * P[1] + A[2] * P[2]) / C_LIGHT \
            + (A @ A) / (2.0 * C_LIGHT ** 2) * S
        e += w * np.real(np.sum(D * Hn.T))              # Tr[D Hn]
    return e + 0.5 * dq @ gamma @ dq


def cell_volume(sysd):
    """Omega = |det(a1, a2, a3)| (Eq. 14)."""
    return abs(float(np.linalg.det(np.asarray(sysd["lattice"], float))))


# ----------------------------------------------------------------------------
# Setup: k-space matrices, inverse overlap, ground state
# ----------------------------------------------------------------------------
def setup(sysd):
    """Bloch matrices and S_k^-1 (Cholesky based) for every k-point."""
    out = {"S": [], "H0": [], "P": [], "Sinv": []}
    for k in np.asarray(sysd["kpt"], float):
        S, H0, P = bloch_matrices(sysd, k)
        cf = sla.cho_factor(S, lower=True)
        Sinv = sla.cho_solve(cf, np.eye(S.shape[0], dtype=complex))
        Sinv = 0.5 * (Sinv + Sinv.conj().T)
        out["S"].append(S)
        out["H0"].append(H0)
        out["P"].append(P)
        out["Sinv"].append(Sinv)
    out["atom_of"] = orbital_atom(sysd)
    out["omega"] = cell_volume(sysd)
    out["wk"] = np.asarray(sysd["wk"], float)
    out["gamma"] = np.asarray(sysd["gamma"], float)
    out["z"] = np.asarray(sysd["z_ref"], float)
    return out


def occupied_states(H, S, n_occ):
    """Lowest n_occ solutions of H C = S C eps (Eq. 5 at rest); returns (C_occ, eps)."""
    e, C = sla.eigh(H, S)
    return C[:, :n_occ], e


def density_from_hamiltonian(H, S, n_occ):
    """D = sum_{n < n_occ} 2 C_n C_n^dagger from H C = S C eps; returns (D, eps)."""
    Co, e = occupied_states(H, S, n_occ)
    return 2.0 * (Co @ Co.conj().T), e


def ground_state(sysd, tol=1e-12, max_iter=200, mix=0.2, history=8, ctx=None):
    """SCC ground state at A = 0 (Sec. 3.1): returns dict(D, C, dq, eps, gap, iters).

    Each iteration diagonalises H_k[dq] at every k, occupies the lowest
    N_el/2 states twice and recomputes dq; dq is mixed with Anderson mixing
    (linear mixing `mix` for the first step) until max |dq_out - dq_in| < tol.
    """
    ctx = setup(sysd) if ctx is None else ctx
    nel = float(sysd["n_electrons"])
    n_occ = int(round(nel / 2))
    atom_of = ctx["atom_of"]
    gamma = ctx["gamma"]
    z = ctx["z"]
    dq = np.zeros(len(z))
    xs, fs = [], []
    gap = np.inf
    for it in range(1, max_iter + 1):
        eps_orb = scc_shift(gamma, dq)[atom_of]
        D_list, C_list = [], []
        gap = np.inf
        for S, H0, P in zip(ctx["S"], ctx["H0"], ctx["P"]):
            H = hamiltonian(H0, S, P, np.zeros(3), eps_orb)
            Co, e = occupied_states(H, S, n_occ)
            C_list.append(Co)
            D_list.append(2.0 * (Co @ Co.conj().T))
            gap = min(gap, e[n_occ] - e[n_occ - 1])
        dq_out = mulliken(D_list, ctx["S"], ctx["wk"], atom_of) - z
        res = dq_out - dq
        if np.max(np.abs(res)) < tol or not np.any(gamma):
            return {"D": D_list, "C": C_list, "dq": dq_out, "eps": scc_shift(gamma, dq_out),
                    "gap": gap, "iters": it, "residual": float(np.max(np.abs(res)))}
        xs.append(dq.copy())
        fs.append(res.copy())
        xs, fs = xs[-history:], fs[-history:]
        if len(fs) == 1:
            dq = dq + mix * res
        else:
            dF = np.array([fs[i + 1] - fs[i] for i in range(len(fs) - 1)]).T
            dX = np.array([xs[i + 1] - xs[i] for i in range(len(xs) - 1)]).T
            coef, *_ = np.linalg.lstsq(dF, res, rcond=None)
            dq = dq + mix * res - (dX + mix * dF) @ coef
    raise RuntimeError("SCC ground state did not converge")


# ----------------------------------------------------------------------------
# Propagation (Eqs. 6, 10, 13, 14)
# ----------------------------------------------------------------------------
def observables(ctx, D_list, A):
    """(J, E, q, eps_orb) at one time level from D_k(t) and A(t)."""
    q = mulliken(D_list, ctx["S"], ctx["wk"], ctx["atom_of"])
    dq = q - ctx["z"]
    eps = scc_shift(ctx["gamma"], dq)
    J = current(D_list, ctx["P"], ctx["S"], A, ctx["omega"], ctx["wk"])
    E = energy(D_list, ctx["H0"], ctx["P"], ctx["S"], A, ctx["wk"], ctx["gamma"], dq)
    return J, E, q, eps[ctx["atom_of"]]


def propagate(sysd, A_table, nsteps, D0_list, ctx=None, D_prev_list=None, n0=0, eps_fixed=None):
    """Leapfrog propagation of D_k for `nsteps` steps from time level n0.

    At every level t_n (n = n0 .. n0+nsteps) the charges, SCC shift, current
    and energy are evaluated from D(t_n); for n < n0+nsteps, dD/dt(t_n) follows
    Eq. 6 with H_k(t_n) and D(t_{n+1}) follows Eq. 13 (forward Euler when no
    earlier level is given).  With eps_fixed (atom-resolved shifts eps_I), the
    H2 term of Eq. 10 uses those shifts at every level instead of gamma dq(t_n)
    (the SCC shift frozen: a non-self-consistent propagation); the charges and
    the energy are still evaluated from D(t_n).  Returns dict(J, E, q, D,
    D_prev) where D is D(t_{n0+nsteps}) and D_prev is D(t_{n0+nsteps-1}).
    """
    ctx = setup(sysd) if ctx is None else ctx
    dt = float(sysd["dt"])
    A_table = np.asarray(A_table, float)
    D = [np.array(d, dtype=complex) for d in D0_list]
    Dp = None if D_prev_list is None else [np.array(d, dtype=complex) for d in D_prev_list]
    Js, Es, qs = [], [], []
    for n in range(n0, n0 + nsteps + 1):
        A = A_table[n]
        J, E, q, eps_orb = observables(ctx, D, A)
        if eps_fixed is not None:
            eps_orb = np.asarray(eps_fixed, float)[ctx["atom_of"]]
        Js.append(J)
        Es.append(E)
        qs.append(q)
        if n == n0 + nsteps:
            break
        Dn = []
        for ik in range(len(D)):
            H = hamiltonian(ctx["H0"][ik], ctx["S"][ik], ctx["P"][ik], A, eps_orb)
            Dd = ddot(D[ik], H, ctx["Sinv"][ik])
            if Dp is None:
                Dn.append(D[ik] + dt * Dd)           # start: forward Euler
            else:
                Dn.append(Dp[ik] + 2.0 * dt * Dd)    # Eq. 13
        Dp, D = D, Dn
    return {"J": np.array(Js), "E": np.array(Es), "q": np.array(qs),
            "D": D, "D_prev": Dp}
