"""Seeded synthetic inputs for velocity-gauge rt-TDDFTB propagation.

This module builds the *inputs* of the propagation problem and nothing else:
silicon-like diamond supercells, Slater-Koster-like real-space two-centre
blocks (overlap S(L), Hamiltonian H0(L) and the overlap gradient dS/dR_J that
defines the momentum blocks of Eq. 12), a Klopman-Ohno gamma matrix, k-point
sets and vector-potential tables A(t_n).  It performs none of the method's
arithmetic (no Bloch sums, charges, commutators or time stepping); both the
CUDA library and the CPU oracle consume the dictionaries it returns.

The paper's Slater-Koster files and structures are not available, so these
synthetic systems stand in for its c-Si / a-Si workloads (Sec. 3.1):

* diamond cubic Si, a = 10.26 bohr, 8 atoms per cubic cell, sp3 basis
  (4 orbitals per atom, orbital order s, px, py, pz), 4 valence electrons per
  atom (Z_I = 4);
* supercells n x n x n with Gaussian atomic displacements of width sigma;
* radial functions c_X * exp(-r / 1.5 bohr) for X in {ss sigma, sp sigma,
  pp sigma, pp pi}, combined with the textbook s/p direction-cosine rules,
  cut off at 10 bohr; prefactors are perturbed by up to +-10 % from the seed;
* gamma_IJ = the Klopman-Ohno kernel 1/sqrt(r^2 + U^-2) (U = 0.25 Ha, equal
  Hubbard parameters) summed over ALL periodic images, evaluated in reciprocal
  space like the Ewald treatment of the long-range part (Sec. 2, after
  Eq. 11): gamma_IJ = (1/Omega) sum_{G != 0} g(G) cos(G.(R_I - R_J)) with
  g(G) = 4 pi a K1(a G) / G, a = 1/U.  The dropped G = 0 term adds the same
  constant to every gamma_IJ and multiplies sum_K dq_K = 0.  A sum truncated
  at 10 bohr is not positive on neutral charge vectors and makes the SCC loop
  diverge, so it is not used;
* Monkhorst-Pack 2x2x2 (k_red in {+-1/4}^3), Gamma-centred 2x2x2
  (k_red in {0, 1/2}^3) or Gamma-only k sets, equal weights;
* A(t) tables: a sin^2-envelope pulse E(t) = E0 sin^2(pi t/T) cos(w t) for
  0 <= t <= T integrated in closed form into A(t) = -c int_0^t E (Eq. 3), or a
  delta kick, A(t_n) = A0 for every n >= 0.

Block convention (Eq. 7): block (I, J, L) holds <phi_mu(r - R_I - L) | . |
phi_nu(r - R_J)> for mu on atom I, nu on atom J, with L = n1 a1 + n2 a2 + n3 a3.
Its distance vector is d = R_J - R_I - L.  For every block (I, J, L) the mirror
block (J, I, -L) is present.  ds[c] is the derivative of the overlap block with
respect to R_J,c (the c-th component of d).
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 137.035999084  # speed of light in atomic units

A_SI = 10.26          # bohr, cubic lattice constant used by all configs
R_CUT = 10.0          # bohr, two-centre cutoff
R_DECAY = 1.5         # bohr, radial decay length of the synthetic integrals
U_HUBBARD = 0.25      # Ha, Klopman-Ohno hardness
ONSITE_S = -0.40      # Ha, s orbital energy
ONSITE_P = -0.15      # Ha, p orbital energy

# Base prefactors of c * exp(-r/R_DECAY) for (ss sigma, sp sigma, pp sigma, pp pi).
# Overlaps follow the usual sign pattern of real s/p orbitals (S_ss > 0,
# S_sp < 0, S_pp sigma < 0, S_pp pi > 0); Hamiltonian integrals carry the
# opposite signs, as for bonding orbitals with negative on-site energies.
BASE_S = np.array([3.2, -3.6, -4.0, 1.9])
BASE_H = np.array([-2.6, 3.0, 3.6, -1.2])

_FRAC_DIAMOND = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])


def _sk_block(d: np.ndarray, v: np.ndarray, onsite: np.ndarray | None):
    """Return (block, grad) for an sp3 pair at distance vector d.

    block[mu, nu] is the two-centre integral of orbital mu (bra, on the atom at
    the origin) with orbital nu (ket, on the atom at d); grad[c] is its
    derivative with respect to d_c.  v holds the four prefactors.  For d = 0
    the on-site block is returned (onsite diagonal, zero gradient).
    """
    blk = np.zeros((4, 4))
    grad = np.zeros((3, 4, 4))
    r = float(np.sqrt(d @ d))
    if r == 0.0:
        if onsite is None:
            blk[:] = np.eye(4)
        else:
            blk[:] = np.diag(onsite)
        return blk, grad
    n = d / r
    f = v * np.exp(-r / R_DECAY)          # radial values
    fp = -f / R_DECAY                      # radial derivatives
    vss, vsp, vpps, vppp = f
    dss, dsp, dpps, dppp = fp
    eye = np.eye(3)
    dn = (eye - np.outer(n, n)) / r        # dn[a, c] = d n_a / d d_c
    # s-s
    blk[0, 0] = vss
    grad[:, 0, 0] = dss * n
    for a in range(3):
        # s - p_a  (bra s at origin, ket p_a at d) and the mirrored p_a - s
        blk[0, 1 + a] = n[a] * vsp
        blk[1 + a, 0] = -n[a] * vsp
        g = dn[a, :] * vsp + n[a] * dsp * n
        grad[:, 0, 1 + a] = g
        grad[:, 1 + a, 0] = -g
        for b in range(3):
            blk[1 + a, 1 + b] = n[a] * n[b] * (vpps - vppp) + eye[a, b] * vppp
            grad[:, 1 + a, 1 + b] = ((dn[a, :] * n[b] + n[a] * dn[b, :]) * (vpps - vppp)
                                     + n[a] * n[b] * (dpps - dppp) * n
                                     + eye[a, b] * dppp * n)
    return blk, grad


def diamond_si(n_cells: int = 1, sigma: float = 0.0, seed: int = 0,
               kgrid: str = "mp2", dt: float = 0.2, a: float = A_SI,
               r_cut: float = R_CUT, hubbard: float = U_HUBBARD,
               gamma_scale: float = 1.0) -> dict:
    """Return a synthetic diamond-Si system as a dict of numpy arrays.

    Keys mirror the C struct ``vgtb_system``: lattice (3,3) rows a1..a3 in
    bohr; pos (n_atoms,3); orb_offset (n_atoms+1,) int32; z_ref (n_atoms,);
    blk_ijl (n_blocks,5) int32 rows (I, J, n1, n2, n3); h0, s flat float64
    (row-major n_I x n_J blocks concatenated); ds (3, total) float64;
    gamma (n_atoms, n_atoms); kpt (n_k,3) reduced; wk (n_k,); n_electrons; dt.
    gamma_scale multiplies gamma (0 turns the charge self-consistency off).
    """
    rng = np.random.default_rng(seed)
    vs = BASE_S * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, 4))
    vh = BASE_H * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, 4))
    lat = np.eye(3) * a * n_cells
    cells = np.array([[i, j, k] for i in range(n_cells) for j in range(n_cells)
                      for k in range(n_cells)], dtype=float)
    frac = (cells[:, None, :] + _FRAC_DIAMOND[None, :, :]).reshape(-1, 3) / n_cells
    pos = frac @ lat
    if sigma > 0.0:
        pos = pos + rng.normal(0.0, sigma, pos.shape)
    nat = pos.shape[0]
    lmax = int(np.ceil(r_cut / (a * n_cells))) + 1
    rng_l = np.arange(-lmax, lmax + 1)
    shifts = np.array([[i, j, k] for i in rng_l for j in rng_l for k in rng_l])
    lvec = shifts @ lat                                     # (n_L, 3)
    ijl, h0, s, ds = [], [], [], []
    onsite = np.array([ONSITE_S, ONSITE_P, ONSITE_P, ONSITE_P])
    for i in range(nat):
        dvec = pos[None, :, :] - pos[i][None, None, :] - lvec[:, None, :]  # (n_L, nat, 3)
        dist = np.sqrt((dvec ** 2).sum(-1))
        li, jj = np.nonzero(dist <= r_cut)
        order = np.lexsort((li, jj))
        for t in order:
            l_idx, j = li[t], jj[t]
            d = dvec[l_idx, j]
            sb, sg = _sk_block(d, vs, None)
            hb, _ = _sk_block(d, vh, onsite)
            ijl.append((i, j, *shifts[l_idx]))
            s.append(sb.ravel())
            h0.append(hb.ravel())
            ds.append(sg.reshape(3, 16))
    kpt, wk = kpoints(kgrid)
    return {
        "lattice": lat,
        "pos": pos,
        "orb_offset": np.arange(0, 4 * nat + 1, 4, dtype=np.int32),
        "z_ref": np.full(nat, 4.0),
        "blk_ijl": np.array(ijl, dtype=np.int32),
        "h0": np.concatenate(h0),
        "s": np.concatenate(s),
        "ds": np.concatenate(ds, axis=1),
        "gamma": gamma_scale * periodic_klopman_ohno(lat, pos, hubbard),
        "kpt": kpt,
        "wk": wk,
        "n_electrons": 4.0 * nat,
        "dt": float(dt),
    }


def periodic_klopman_ohno(lat, pos, hubbard, a_gmax: float = 36.0,
                          chunk: int = 32768) -> np.ndarray:
    """gamma_IJ = (1/Omega) sum_{G != 0} 4 pi a K1(aG)/G cos(G.(R_I - R_J)), a = 1/U.

    This is the lattice sum over all images of 1/sqrt(r^2 + a^2), whose Fourier
    transform is 4 pi a K1(a G)/G > 0, without its G = 0 term.  Terms with
    a|G| > a_gmax (relative size < exp(-a_gmax)) are dropped.  Computed as
    gamma = sum_G w_G [c_G c_G^T + s_G s_G^T] over half of the G sphere.
    """
    from scipy.special import k1
    a = 1.0 / hubbard
    lat = np.asarray(lat, float)
    omega = abs(np.linalg.det(lat))
    rec = 2.0 * np.pi * np.linalg.inv(lat).T            # rows b_i, b_i.a_j = 2 pi delta
    gmax = a_gmax / a
    m = [int(np.ceil(gmax / np.linalg.norm(rec[i]) * 1.0)) + 1 for i in range(3)]
    m0 = np.arange(-m[0], m[0] + 1)
    m1 = np.arange(-m[1], m[1] + 1)
    m2 = np.arange(-m[2], m[2] + 1)
    grid = np.stack(np.meshgrid(m0, m1, m2, indexing="ij"), -1).reshape(-1, 3)
    # half space: first nonzero integer coordinate positive
    first = np.where(grid[:, 0] != 0, grid[:, 0], np.where(grid[:, 1] != 0, grid[:, 1], grid[:, 2]))
    grid = grid[first > 0]
    gvec = grid @ rec
    gn = np.sqrt((gvec ** 2).sum(1))
    keep = gn <= gmax
    gvec, gn = gvec[keep], gn[keep]
    w = 2.0 * (4.0 * np.pi * a * k1(a * gn) / gn) / omega   # factor 2: +-G pair
    nat = pos.shape[0]
    gam = np.zeros((nat, nat))
    for s0 in range(0, len(gn), chunk):
        ph = pos @ gvec[s0:s0 + chunk].T
        sw = np.sqrt(w[s0:s0 + chunk])
        c = np.cos(ph) * sw
        s = np.sin(ph) * sw
        gam += c @ c.T + s @ s.T
    return 0.5 * (gam + gam.T)


def kpoints(kind: str):
    """k-point sets in reduced coordinates with equal weights summing to one."""
    if kind == "gamma":
        k = np.zeros((1, 3))
    elif kind == "mp2":          # Monkhorst-Pack 2x2x2, shifted off Gamma
        v = np.array([-0.25, 0.25])
        k = np.array([[x, y, z] for x in v for y in v for z in v])
    elif kind == "gc2":          # Gamma-centred 2x2x2
        v = np.array([0.0, 0.5])
        k = np.array([[x, y, z] for x in v for y in v for z in v])
    else:
        raise ValueError(f"unknown k grid {kind!r}")
    return k, np.full(k.shape[0], 1.0 / k.shape[0])


def pulse_field(nsteps: int, dt: float, e0: float, omega: float,
                pol=(1.0, 0.0, 0.0), duration: float | None = None) -> np.ndarray:
    """A(t_n), n = 0..nsteps, for E(t) = e0 sin^2(pi t/T) cos(omega t) pol.

    A(t) = -c int_0^t E(tau) dtau (Eq. 3), integrated in closed form; the
    envelope lasts T = duration (default nsteps*dt) and A stays constant after.
    """
    T = nsteps * dt if duration is None else duration
    t = np.minimum(np.arange(nsteps + 1) * dt, T)
    w1 = 2.0 * np.pi / T
    # sin^2(pi t/T) cos(w t) = cos(w t)/2 - [cos((w-w1)t) + cos((w+w1)t)]/4
    def sinc_int(w):
        return t.copy() if w == 0.0 else np.sin(w * t) / w
    integral = 0.5 * sinc_int(omega) - 0.25 * (sinc_int(omega - w1) + sinc_int(omega + w1))
    pol = np.asarray(pol, dtype=float)
    pol = pol / np.linalg.norm(pol)
    return (-C_LIGHT * e0 * integral)[:, None] * pol[None, :]


def kick_field(nsteps: int, a0: float, pol=(1.0, 0.0, 0.0)) -> np.ndarray:
    """A(t_n) = a0 * pol for every n >= 0 (a delta kick applied at t = 0)."""
    pol = np.asarray(pol, dtype=float)
    pol = pol / np.linalg.norm(pol)
    return np.tile(a0 * pol, (nsteps + 1, 1))


BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
HARTREE_EV = 27.211386245988
AU_TIME_FS = 0.0241888432658


def coordination_numbers(sysd: dict, r_bond: float = 2.85 * BOHR_PER_ANGSTROM) -> np.ndarray:
    """Neighbours of each atom within r_bond (bohr; 2.85 A is the bond-length cut-off
    of the a-Si coordination analysis in Sec. 3.3), over all periodic images."""
    lat = np.asarray(sysd["lattice"], float)
    pos = np.asarray(sysd["pos"], float)
    n = len(pos)
    inv = np.linalg.inv(lat)
    cn = np.zeros(n, dtype=np.int64)
    reach = [int(np.ceil(r_bond * np.linalg.norm(inv[:, i]))) for i in range(3)]
    shifts = np.array([(a, b, c) for a in range(-reach[0], reach[0] + 1)
                       for b in range(-reach[1], reach[1] + 1)
                       for c in range(-reach[2], reach[2] + 1)], float) @ lat
    for i in range(n):
        d = pos[None, :, :] + shifts[:, None, :] - pos[i][None, None, :]
        r = np.linalg.norm(d, axis=2)
        cn[i] = int(np.sum((r > 1e-8) & (r <= r_bond)))
    return cn


def laser_sweep(dt: float = 0.2, e0: float = 0.00534, energies_ev=(2.3, 3.9, 6.0), duration_fs: float = 20.0,
                pol=(1.0, 0.0, 0.0)):
    """Fields of the laser experiment of Sec. 3.3: a sin^2-enveloped pulse of 20 fs
    (centred at 10 fs) at each photon energy, E0 = 0.00534 au (10^12 W/cm^2, about
    0.274 eV/A) along x.  Returns (list of A tables, nsteps)."""
    T = duration_fs / AU_TIME_FS
    n = int(round(T / dt))
    return [pulse_field(n, dt, e0, w / HARTREE_EV, pol=pol, duration=T) for w in energies_ev], n


def config(name: str):
    """Named workloads: returns (system, A table, nsteps).

    si8_pulse   : 8-atom cell, MP 2x2x2, pulse E0=0.01, w=0.1 Ha, 1000 steps.
    si64_pulse  : 64-atom cell, sigma=0.05, MP 2x2x2, same pulse, 2000 steps.
    si512_kick  : 512-atom cell, sigma=0.3, Gamma, kick A_x=0.001, 5000 steps.
    si512k8_kick: as si512_kick on the MP 2x2x2 grid.
    """
    if name == "si8_pulse":
        sysd = diamond_si(1, 0.0, seed=8, kgrid="mp2")
        n = 1000
        return sysd, pulse_field(n, sysd["dt"], 0.01, 0.1), n
    if name == "si64_pulse":
        sysd = diamond_si(2, 0.05, seed=64, kgrid="mp2")
        n = 2000
        return sysd, pulse_field(n, sysd["dt"], 0.01, 0.1), n
    if name == "si512_kick":
        sysd = diamond_si(4, 0.3, seed=512, kgrid="gamma")
        n = 5000
        return sysd, kick_field(n, 0.001), n
    if name == "si512k8_kick":
        sysd = diamond_si(4, 0.3, seed=512, kgrid="mp2")
        n = 5000
        return sysd, kick_field(n, 0.001), n
    raise ValueError(f"unknown config {name!r}")
