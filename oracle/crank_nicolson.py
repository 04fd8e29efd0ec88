"""Crank-Nicolson propagation of the coefficient vectors (Eq. 5).

TEST INFRASTRUCTURE ONLY (see oracle/vgtb_oracle.py): imported by the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``.

Eq. 5 is i dC_nk/dt = S_k^-1 H_k C_nk.  Sec. 2 names the unitary Crank-Nicolson
scheme as the alternative to the leapfrog of Eq. 13 without giving its form;
the form used here is the standard one (Crank and Nicolson 1947; Castro et al.
2004):

  (S_k + i (dt/2) H_k(t_{n+1/2})) C(t_{n+1}) = (S_k - i (dt/2) H_k(t_{n+1/2})) C(t_n)

which keeps C^dagger S_k C constant when H_k is Hermitian.  Readings where the
paper is silent (listed in the design notes):
  * the density and all observables at t_n come from D_k = sum_n f_n C C^dagger
    with f_n = 2 on the lowest N_el/2 states (the occupation of the leapfrog
    path), through the same Mulliken charge, current and energy as there;
  * H_k(t_{n+1/2}) takes A at the midpoint, (A_n + A_{n+1})/2, and the SCC
    shift extrapolated linearly from the two latest levels,
    eps_{n+1/2} = (3 eps_n - eps_{n-1})/2 (eps_{-1} = eps_0 at the first step);
  * the |A|^2/(2c^2) S term of Eq. 12 is left out of H_k: the remark after
    Eq. 3 says it only multiplies the wavefunction by an overall phase.
"""
import numpy as np

from . import vgtb_oracle as _o


def cn_hamiltonian(H0, S, P, A, eps_orb):
    """H_k of Eqs. 9, 10, 12 without the |A|^2 S term (remark after Eq. 3)."""
    A = np.asarray(A, float)
    return _o.hamiltonian(H0, S, P, A, eps_orb) - (A @ A) / (2.0 * _o.C_LIGHT ** 2) * S


def cn_step(S, H, C, theta):
    """One Crank-Nicolson step: solve (S + i theta H) C_new = (S - i theta H) C, theta = dt/2."""
    return np.linalg.solve(S + 1j * theta * H, (S - 1j * theta * H) @ C)


def cn_midpoint(A_table, n, eps_n, eps_prev):
    """(A, SCC shift per atom) at t_{n+1/2}: midpoint A, linearly extrapolated shift."""
    A_mid = 0.5 * (np.asarray(A_table[n], float) + np.asarray(A_table[n + 1], float))
    e_prev = eps_n if eps_prev is None else eps_prev
    return A_mid, 1.5 * eps_n - 0.5 * e_prev


def density(C_list, occ=2.0):
    """D_k = occ C_k C_k^dagger (columns of C_k are the occupied states)."""
    return [occ * (C @ C.conj().T) for C in C_list]


def propagate_cn(sysd, A_table, nsteps, C0_list, ctx=None, occ=2.0, eps_prev=None, n0=0):
    """Crank-Nicolson propagation of the occupied coefficient vectors.

    At every level t_n (n = n0 .. n0+nsteps) the observables come from
    D_k(t_n) = occ C_k C_k^dagger exactly as on the leapfrog path; for
    n < n0+nsteps, C_k(t_{n+1}) follows one Crank-Nicolson step with
    H_k(t_{n+1/2}).  `eps_prev` is the per-atom SCC shift at t_{n0-1} (None
    at the start of a run).  Returns dict(J, E, q, C, eps, eps_prev): the
    final coefficients and the shifts at the last two levels.
    """
    ctx = _o.setup(sysd) if ctx is None else ctx
    theta = 0.5 * float(sysd["dt"])
    A_table = np.asarray(A_table, float)
    gamma, atom_of = ctx["gamma"], ctx["atom_of"]
    C = [np.array(c, dtype=complex) for c in C0_list]
    Js, Es, qs = [], [], []
    eps_n = None
    for n in range(n0, n0 + nsteps + 1):
        D = density(C, occ)
        J, E, q, _ = _o.observables(ctx, D, A_table[n])
        Js.append(J)
        Es.append(E)
        qs.append(q)
        eps_n = _o.scc_shift(gamma, q - ctx["z"])
        if n == n0 + nsteps:
            break
        A_mid, eps_mid = cn_midpoint(A_table, n, eps_n, eps_prev)
        Cn = []
        for ik in range(len(C)):
            H = cn_hamiltonian(ctx["H0"][ik], ctx["S"][ik], ctx["P"][ik], A_mid, eps_mid[atom_of])
            Cn.append(cn_step(ctx["S"][ik], H, C[ik], theta))
        C = Cn
        eps_prev = eps_n
    return {"J": np.array(Js), "E": np.array(Es), "q": np.array(qs), "C": C,
            "eps": eps_n, "eps_prev": eps_prev}
