"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test targets a plausible mistake: a dropped term, a wrong sign or index,
a transposed operand, a wrong phase convention, a wrong integrator start.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2308_09782_gb300 import inputs
from tests import _brute


def _fro_rel(a_list, b_list):
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(a_list, b_list))
    den = sum(np.linalg.norm(b) ** 2 for b in b_list)
    return np.sqrt(num / den)


@pytest.fixture(scope="module")
def si8():
    s, A, n = inputs.config("si8_pulse")
    ctx = O.setup(s)
    gs = O.ground_state(s, ctx=ctx)
    return s, A, n, ctx, gs


@pytest.fixture(scope="module")
def si8_run(si8):
    s, A, n, ctx, gs = si8
    return O.propagate(s, A, n, gs["D"], ctx=ctx)


def test_bloch_matrices_hermitian_and_overlap_positive(si8):
    s, A, n, ctx, gs = si8
    for S, H0, P in zip(ctx["S"], ctx["H0"], ctx["P"]):
        np.testing.assert_allclose(S, S.conj().T, atol=1e-15)
        np.testing.assert_allclose(H0, H0.conj().T, atol=1e-15)
        for a in range(3):
            np.testing.assert_allclose(P[a], P[a].conj().T, atol=1e-15)
        assert np.linalg.eigvalsh(S).min() > 0.05


def test_gen_acceptance_gap_and_stability():
    """The synthetic systems have a gap at N_el/2 and dt*(spread of S^-1H) < 0.5."""
    for cfg in ("si8_pulse", "si64_pulse"):
        s, A, n = inputs.config(cfg)
        ctx = O.setup(s)
        nocc = int(s["n_electrons"] / 2)
        for S, H0 in zip(ctx["S"], ctx["H0"]):
            e = sla.eigh(H0, S, eigvals_only=True)
            assert e[nocc] - e[nocc - 1] > 0.05
            assert s["dt"] * (e[-1] - e[0]) < 0.5


def test_p1_hermiticity_preserved_exactly(si8_run):
    """P-1: D' of Eq. 6 is Hermitian, so Eq. 13 keeps D_k Hermitian to rounding."""
    for D in si8_run["D"]:
        assert np.abs(D - D.conj().T).max() <= 1e-13 * np.abs(D).max()


def test_p2_electron_count_conserved(si8, si8_run):
    """P-2: Tr(D_k S_k) = N_el for every k and every step; sum dq = 0."""
    s, A, n, ctx, gs = si8
    for D, S in zip(si8_run["D"], ctx["S"]):
        assert abs(np.trace(D @ S).real - s["n_electrons"]) < 1e-11
    np.testing.assert_allclose(si8_run["q"].sum(1), s["n_electrons"], atol=1e-11)


def test_p3_ground_state_stationary_without_field():
    """P-3: at A = 0 the SCC ground state does not move (displaced 64-atom cell)."""
    s = inputs.diamond_si(2, 0.05, seed=64, kgrid="gamma")
    ctx = O.setup(s)
    gs = O.ground_state(s, ctx=ctx, tol=1e-13)
    n = 60
    r = O.propagate(s, np.zeros((n + 1, 3)), n, gs["D"], ctx=ctx)
    assert _fro_rel(r["D"], gs["D"]) < 1e-11
    assert np.abs(r["J"]).max() < 1e-14
    assert np.ptp(r["E"]) < 1e-11
    assert np.abs(r["q"] - r["q"][0]).max() < 1e-11


def test_p4_a_squared_term_is_a_pure_phase(si8):
    """P-4: with P = 0 only |A|^2/(2c^2) S remains: D stays put, E shifts by alpha*N_el."""
    s, A, n, ctx, gs = si8
    s0 = dict(s)
    s0["ds"] = np.zeros_like(s["ds"])
    a0 = 40.0
    nst = 50
    At = np.tile([a0, -0.3 * a0, 0.5 * a0], (nst + 1, 1))
    ctx0 = O.setup(s0)
    r = O.propagate(s0, At, nst, gs["D"], ctx=ctx0)
    r0 = O.propagate(s0, np.zeros_like(At), 0, gs["D"], ctx=ctx0)
    assert _fro_rel(r["D"], gs["D"]) < 1e-12
    alpha = (At[0] @ At[0]) / (2 * O.C_LIGHT ** 2)
    np.testing.assert_allclose(r["E"] - r0["E"][0], alpha * s["n_electrons"], rtol=1e-12)


def test_p6_leapfrog_closed_form_constant_hamiltonian():
    """P-6: for constant H each generalized-eigenbasis element follows
    x_{n+1} = x_{n-1} - 2 i w dt x_n with the Euler start x_1 = (1 - i w dt) x_0."""
    s = inputs.diamond_si(1, 0.1, seed=5, kgrid="mp2", gamma_scale=0.0)
    ctx = O.setup(s)
    gs = O.ground_state(s, ctx=ctx)
    n = 300
    A = inputs.kick_field(n, 2.0, pol=(1.0, 0.5, -0.2))
    r = O.propagate(s, A, n, gs["D"], ctx=ctx)
    dt = s["dt"]
    for ik in (0, 3):
        H = O.hamiltonian(ctx["H0"][ik], ctx["S"][ik], ctx["P"][ik], A[0],
                          np.zeros(ctx["S"][ik].shape[0]))
        M = ctx["Sinv"][ik] @ H
        lam, V = sla.eig(M)
        lam = lam.real
        Vi = np.linalg.inv(V)
        X0 = Vi @ gs["D"][ik] @ Vi.conj().T
        w = lam[:, None] - lam[None, :]
        rp = -1j * w * dt + np.sqrt(1 - (w * dt) ** 2)
        rm = -1j * w * dt - np.sqrt(1 - (w * dt) ** 2)
        x1 = (1 - 1j * w * dt) * X0
        a = (x1 - rm * X0) / (rp - rm)
        b = X0 - a
        Xn = a * rp ** n + b * rm ** n
        Dn = V @ Xn @ V.conj().T
        assert np.linalg.norm(Dn - r["D"][ik]) / np.linalg.norm(Dn) < 1e-11


def test_p6b_frozen_shift_is_the_closed_form_of_its_constant_hamiltonian():
    """P-6 with the SCC shift frozen (eps_fixed): with gamma != 0 and a kick, H_k
    = H0 + (eps0_I + eps0_J) S / 2 + (A/c).P + |A|^2/(2c^2) S is constant in time,
    so the leapfrog from the SCC ground state equals the closed form of P-6 for
    that H, while the self-consistent run (shift following dq(t)) does not."""
    s = inputs.diamond_si(1, 0.1, seed=5, kgrid="mp2")
    ctx = O.setup(s)
    gs = O.ground_state(s, ctx=ctx)
    n = 300
    A = inputs.kick_field(n, 2.0, pol=(1.0, 0.5, -0.2))
    r = O.propagate(s, A, n, gs["D"], ctx=ctx, eps_fixed=gs["eps"])
    r_scc = O.propagate(s, A, n, gs["D"], ctx=ctx)
    dt = s["dt"]
    eps_orb = gs["eps"][ctx["atom_of"]]
    assert np.abs(gs["eps"]).max() > 1e-3
    for ik in (0, 3):
        H = O.hamiltonian(ctx["H0"][ik], ctx["S"][ik], ctx["P"][ik], A[0], eps_orb)
        lam, V = sla.eig(ctx["Sinv"][ik] @ H)
        lam = lam.real
        Vi = np.linalg.inv(V)
        X0 = Vi @ gs["D"][ik] @ Vi.conj().T
        w = lam[:, None] - lam[None, :]
        rp = -1j * w * dt + np.sqrt(1 - (w * dt) ** 2)
        rm = -1j * w * dt - np.sqrt(1 - (w * dt) ** 2)
        x1 = (1 - 1j * w * dt) * X0
        a = (x1 - rm * X0) / (rp - rm)
        Dn = V @ (a * rp ** n + (X0 - a) * rm ** n) @ V.conj().T
        assert np.linalg.norm(Dn - r["D"][ik]) / np.linalg.norm(Dn) < 1e-11
        assert np.linalg.norm(Dn - r_scc["D"][ik]) / np.linalg.norm(Dn) > 1e-6


def test_p7_band_folding_supercell_equals_kgrid(si8):
    """P-7: 64-atom Gamma supercell == 8-atom cell on the Gamma-centred 2x2x2 grid."""
    s8 = inputs.diamond_si(1, 0.0, seed=8, kgrid="gc2")
    s64 = inputs.diamond_si(2, 0.0, seed=8, kgrid="gamma")
    n = 40
    A = inputs.pulse_field(n, 0.2, 0.02, 0.15, pol=(1.0, 0.3, 0.1), duration=12.0)
    g8 = O.ground_state(s8)
    g64 = O.ground_state(s64)
    r8 = O.propagate(s8, A, n, g8["D"])
    r64 = O.propagate(s64, A, n, g64["D"])
    np.testing.assert_allclose(r64["J"], r8["J"], rtol=0, atol=1e-11 * np.abs(r8["J"]).max())
    np.testing.assert_allclose(r64["E"], 8 * r8["E"], rtol=1e-12)
    np.testing.assert_allclose(r64["q"][:, :8], r8["q"], atol=1e-11)
    assert np.abs(r8["J"]).max() > 1e-6


def test_p8_work_theorem_second_order(si8):
    """P-8: dE/dt = Omega E_field . J; the discrete mismatch shrinks as dt^2."""
    s, _, _, ctx, gs = si8
    err = []
    for dt in (0.2, 0.1):
        sd = dict(s)
        sd["dt"] = dt
        T = 60.0
        n = int(round(T / dt))
        A = inputs.pulse_field(n, dt, 0.02, 0.1)
        r = O.propagate(sd, A, n, gs["D"], ctx=ctx)
        t = np.arange(n + 1) * dt
        ef = 0.02 * np.sin(np.pi * t / T) ** 2 * np.cos(0.1 * t)    # E_x(t)
        power = ctx["omega"] * r["J"][:, 0] * ef
        work = np.concatenate([[0.0], np.cumsum(0.5 * (power[1:] + power[:-1]) * dt)])
        err.append(np.abs((r["E"] - r["E"][0]) - work).max())
        assert np.abs(r["E"] - r["E"][0]).max() > 10 * err[-1]
    assert 3.0 < err[0] / err[1] < 5.0


def test_p9_two_level_rabi():
    """P-9: two-level system driven at resonance through the A.p term."""
    delta, p, dt = 0.5, 1.0, 0.05
    a0 = 0.01 * O.C_LIGHT / p       # Rabi frequency A0 p / c = 0.01
    sysd = {
        "lattice": np.eye(3) * 1000.0, "pos": np.array([[0., 0, 0], [1.0, 0, 0]]),
        "orb_offset": np.array([0, 1, 2], np.int32), "z_ref": np.array([1.0, 0.0]),
        "blk_ijl": np.array([[0, 0, 0, 0, 0], [1, 1, 0, 0, 0], [0, 1, 0, 0, 0], [1, 0, 0, 0, 0]], np.int32),
        "h0": np.array([-delta / 2, delta / 2, 0.0, 0.0]), "s": np.array([1.0, 1.0, 0.0, 0.0]),
        "ds": np.array([[0.0, 0.0, p, -p], [0.0] * 4, [0.0] * 4]),
        "gamma": np.zeros((2, 2)), "kpt": np.zeros((1, 3)), "wk": np.ones(1),
        "n_electrons": 1.0, "dt": dt,
    }
    omega_r = a0 * p / O.C_LIGHT
    T = np.pi / omega_r                         # half a Rabi period: full inversion
    n = int(round(T / dt))
    t = np.arange(n + 1) * dt
    A = np.zeros((n + 1, 3))
    A[:, 0] = a0 * np.cos(delta * t)
    D0 = np.diag([1.0, 0.0]).astype(complex)
    ctx = O.setup(sysd)
    # excited population along the run against the rotating-wave formula
    pe = []
    D, Dp = [D0], None
    for m in range(0, n, 200):
        step = min(200, n - m)
        r = O.propagate(sysd, A, step, D, ctx=ctx, D_prev_list=Dp, n0=m)
        D, Dp = r["D"], r["D_prev"]
        pe.append((t[m + step], D[0][1, 1].real))
    for tt, pp in pe:
        assert abs(pp - np.sin(omega_r * tt / 2) ** 2) < 0.03
    # and against a brute-force midpoint exponential at dt/100: error O(dt^2)
    def exact(nsteps, h_dt):
        U = np.eye(2, dtype=complex)
        h = h_dt / 100
        for j in range(100 * nsteps):
            tm = (j + 0.5) * h
            a = a0 * np.cos(delta * tm)
            H = np.array([[-delta / 2, 1j * p * a / O.C_LIGHT], [-1j * p * a / O.C_LIGHT, delta / 2]])
            U = sla.expm(-1j * H * h) @ U
        return U @ D0 @ U.conj().T
    errs = []
    nshort = 200
    for h_dt in (dt, dt / 2):
        sd = dict(sysd)
        sd["dt"] = h_dt
        ns = int(round(nshort * dt / h_dt))
        tt = np.arange(ns + 1) * h_dt
        Ah = np.zeros((ns + 1, 3))
        Ah[:, 0] = a0 * np.cos(delta * tt)
        r = O.propagate(sd, Ah, ns, [D0])
        errs.append(np.abs(r["D"][0] - exact(ns, h_dt)).max())
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_p10_density_matrix_eom_equals_coefficient_eom():
    """P-10: Eq. 6 for D = sum f C C^dagger agrees with Eq. 5 for C to O(dt^2)."""
    s = inputs.diamond_si(1, 0.1, seed=11, kgrid="gamma")
    ctx = O.setup(s)
    gs = O.ground_state(s, ctx=ctx)
    S, H0, P, Si = ctx["S"][0], ctx["H0"][0], ctx["P"][0], ctx["Sinv"][0]
    nocc = int(s["n_electrons"] / 2)
    Hg = O.hamiltonian(H0, S, P, np.zeros(3), O.scc_shift(ctx["gamma"], gs["dq"])[ctx["atom_of"]])
    _, Cg = sla.eigh(Hg, S)
    Cg = Cg[:, :nocc]
    T = 8.0
    errs = []
    for dt in (0.1, 0.05):
        sd = dict(s)
        sd["dt"] = dt
        n = int(round(T / dt))
        A = inputs.pulse_field(n, dt, 0.05, 0.2, duration=T)
        r = O.propagate(sd, A, n, gs["D"], ctx=ctx)
        # Eq. 5 with SCC: C(t+h) = exp(-i S^-1 H(t+h/2) h) C, fine steps h = dt/20
        Cc = Cg.copy()
        h = dt / 20
        tt = 0.0
        for j in range(20 * n):
            Dm = 2 * Cc @ Cc.conj().T
            q = O.mulliken([Dm], [S], [1.0], ctx["atom_of"])
            eps = O.scc_shift(ctx["gamma"], q - ctx["z"])[ctx["atom_of"]]
            tm = tt + 0.5 * h
            Am = inputs.pulse_field(1, tm, 0.05, 0.2, duration=T)[1]
            Cp = sla.expm(-1j * Si @ O.hamiltonian(H0, S, P, Am, eps) * (h / 2)) @ Cc
            Dm = 2 * Cp @ Cp.conj().T
            q = O.mulliken([Dm], [S], [1.0], ctx["atom_of"])
            eps = O.scc_shift(ctx["gamma"], q - ctx["z"])[ctx["atom_of"]]
            Cc = sla.expm(-1j * Si @ O.hamiltonian(H0, S, P, Am, eps) * h) @ Cc
            tt += h
        Dc = 2 * Cc @ Cc.conj().T
        errs.append(np.linalg.norm(r["D"][0] - Dc) / np.linalg.norm(Dc))
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_p11_inversion_and_time_reversal(si8):
    """P-11: centrosymmetric crystal: J[-A] = -J[A]; at A = 0: D_{-k} = conj(D_k)."""
    s, _, _, ctx, gs = si8
    kp = s["kpt"]
    for i, k in enumerate(kp):
        j = int(np.argmin(np.abs(kp + k).sum(1)))
        np.testing.assert_allclose(gs["D"][j], gs["D"][i].conj(), atol=1e-12)
    n = 60
    A = inputs.pulse_field(n, s["dt"], 0.02, 0.1, pol=(1.0, 0.2, 0.0))
    rp = O.propagate(s, A, n, gs["D"], ctx=ctx)
    rm = O.propagate(s, -A, n, gs["D"], ctx=ctx)
    np.testing.assert_allclose(rm["J"], -rp["J"], atol=1e-12 * np.abs(rp["J"]).max())
    assert np.abs(rp["J"]).max() > 1e-6


def test_p12_linear_response_limit(si8):
    """P-12: J(2 A0) / J(A0) -> 2 for a weak kick (odd response, error O(A0^2))."""
    s, _, _, ctx, gs = si8
    n = 80
    j1 = O.propagate(s, inputs.kick_field(n, 1e-3), n, gs["D"], ctx=ctx)["J"][:, 0]
    j2 = O.propagate(s, inputs.kick_field(n, 2e-3), n, gs["D"], ctx=ctx)["J"][:, 0]
    big = np.abs(j1) > 0.1 * np.abs(j1).max()
    np.testing.assert_allclose(j2[big] / j1[big], 2.0, rtol=1e-5)


def test_p14_brute_force_loops_gamma():
    """P-14: the oracle equals an element-by-element loop implementation (10 steps)."""
    s = inputs.diamond_si(1, 0.15, seed=14, kgrid="gamma")
    ctx = O.setup(s)
    gs = O.ground_state(s, ctx=ctx, tol=1e-10)
    n = 10
    A = inputs.pulse_field(n, s["dt"], 0.5, 0.3, pol=(0.3, 1.0, 0.2), duration=2.0)
    r = O.propagate(s, A, n, gs["D"], ctx=ctx)
    Jb, Db = _brute.propagate_gamma(s, A, n, gs["D"][0])
    np.testing.assert_allclose(r["J"], np.array(Jb), rtol=1e-10, atol=1e-15)
    assert np.abs(r["D"][0] - np.array(Db)).max() < 1e-12


def test_ground_state_properties(si8):
    """The ground state has Tr(DS) = N_el per k, D S D = 2 D (idempotent up to f = 2)."""
    s, _, _, ctx, gs = si8
    for D, S in zip(gs["D"], ctx["S"]):
        assert abs(np.trace(D @ S).real - s["n_electrons"]) < 1e-11
        np.testing.assert_allclose(D @ S @ D, 2 * D, atol=1e-11)


def test_p13_constant_a_is_a_gauge_transformation_to_first_order():
    """P-13: orthonormal ring with P = i[H0, X]: H(A) = U H0 U^dagger + O(A^2) with
    U = exp(-i A.X / c), so D' = U D0 U^dagger is stationary under a constant A up to
    O(A^2); a wrong sign of the (1/c) A.P term of Eq. 12 would make it drift at O(A)."""
    nat = 6
    rng = np.random.default_rng(13)
    ang = 2 * np.pi * np.arange(nat) / nat
    pos = np.stack([5.0 * np.cos(ang), 5.0 * np.sin(ang), np.zeros(nat)], 1) + rng.normal(0, 0.1, (nat, 3))
    H0 = np.zeros((nat, nat))
    for i in range(nat):
        H0[i, i] = -0.3 + 0.05 * rng.normal()
        j = (i + 1) % nat
        H0[i, j] = H0[j, i] = -0.1 * (1 + 0.1 * rng.normal())
    ijl, h0, s, ds = [], [], [], []
    for i in range(nat):
        for j in range(nat):
            if i == j or H0[i, j] != 0.0:
                ijl.append((i, j, 0, 0, 0))
                h0.append(H0[i, j])
                s.append(1.0 if i == j else 0.0)
                # dS/dR_J such that P = i dS = i [H0, X]:  [H0, X]_ij = H0_ij (x_j - x_i)
                ds.append(H0[i, j] * (pos[j] - pos[i]))
    sysd = {"lattice": np.eye(3) * 1000.0, "pos": pos, "orb_offset": np.arange(nat + 1, dtype=np.int32),
            "z_ref": np.ones(nat), "blk_ijl": np.array(ijl, np.int32), "h0": np.array(h0), "s": np.array(s),
            "ds": np.array(ds).T.copy(), "gamma": np.zeros((nat, nat)), "kpt": np.zeros((1, 3)),
            "wk": np.ones(1), "n_electrons": float(nat), "dt": 0.1}
    ctx = O.setup(sysd)
    gs = O.ground_state(sysd, ctx=ctx)
    n = 400
    devs = []
    for a0 in (4.0, 2.0):
        A = np.tile([a0, 0.5 * a0, 0.0], (n + 1, 1))
        U = np.diag(np.exp(-1j * (pos @ A[0]) / O.C_LIGHT))
        Dg = U @ gs["D"][0] @ U.conj().T
        r = O.propagate(sysd, A, n, [Dg], ctx=ctx)
        devs.append(np.linalg.norm(r["D"][0] - Dg))
        # a first-order (wrong-sign) error would show up as drift of size O(A)
        Dw = U.conj().T @ gs["D"][0] @ U
        rw = O.propagate(sysd, A, n, [Dw], ctx=ctx)
        assert np.linalg.norm(rw["D"][0] - Dw) > 5 * devs[-1]
    assert 3.5 < devs[0] / devs[1] < 4.5
