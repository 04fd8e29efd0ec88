"""Checks of the seeded synthetic inputs (no GPU, no oracle arithmetic)."""
import numpy as np
import pytest
from scipy.integrate import quad

from paper_2308_09782_gb300 import inputs


def test_sk_gradient_matches_finite_difference():
    rng = np.random.default_rng(1)
    v = np.array([3.0, -3.3, -4.1, 2.0])
    for _ in range(5):
        d = rng.normal(0, 3.0, 3)
        _, g = inputs._sk_block(d, v, None)
        h = 1e-6
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            fd = (inputs._sk_block(d + e, v, None)[0] - inputs._sk_block(d - e, v, None)[0]) / (2 * h)
            np.testing.assert_allclose(g[c], fd, atol=1e-8, rtol=1e-6)


def test_mirror_blocks_consistent():
    """Block (J,I,-L) is the transpose of (I,J,L); its gradient the negated transpose."""
    s = inputs.diamond_si(1, 0.1, seed=3, kgrid="gamma")
    ijl = s["blk_ijl"]
    key = {tuple(r): b for b, r in enumerate(ijl)}
    for b, r in enumerate(ijl):
        i, j, n1, n2, n3 = r
        m = key[(j, i, -n1, -n2, -n3)]
        np.testing.assert_array_equal(s["s"][16 * m:16 * m + 16].reshape(4, 4),
                                      s["s"][16 * b:16 * b + 16].reshape(4, 4).T)
        np.testing.assert_array_equal(s["h0"][16 * m:16 * m + 16].reshape(4, 4),
                                      s["h0"][16 * b:16 * b + 16].reshape(4, 4).T)
        np.testing.assert_array_equal(s["ds"][:, 16 * m:16 * m + 16].reshape(3, 4, 4),
                                      -s["ds"][:, 16 * b:16 * b + 16].reshape(3, 4, 4).transpose(0, 2, 1))


def test_neighbour_count_diamond():
    """Undistorted diamond within 10 bohr: 1 + 4 + 12 + 12 = 29 partners per atom."""
    s = inputs.diamond_si(2, 0.0, seed=0, kgrid="gamma")
    counts = np.bincount(s["blk_ijl"][:, 0])
    assert np.all(counts == 29)


def test_pulse_is_minus_c_integral_of_field():
    """Eq. 3: A(t) = -c int_0^t E(tau) dtau for the sin^2 pulse."""
    n, dt, e0, w = 400, 0.2, 0.01, 0.1
    A = inputs.pulse_field(n, dt, e0, w)
    T = n * dt

    def field(t):
        return e0 * np.sin(np.pi * t / T) ** 2 * np.cos(w * t)
    for step in (0, 37, 200, 399, 400):
        t = step * dt
        ref = -inputs.C_LIGHT * quad(field, 0.0, t, limit=200)[0]
        assert abs(A[step, 0] - ref) < 1e-10
        assert A[step, 1] == 0.0 and A[step, 2] == 0.0


def test_gamma_positive_on_neutral_charges_and_symmetric():
    s = inputs.diamond_si(2, 0.05, seed=64, kgrid="gamma")
    g = s["gamma"]
    np.testing.assert_array_equal(g, g.T)
    nat = g.shape[0]
    proj = np.eye(nat) - np.ones((nat, nat)) / nat
    ev = np.linalg.eigvalsh(proj @ g @ proj)
    assert np.sort(ev)[1] > 0.0  # one zero eigenvalue (the uniform vector), the rest > 0


def test_gamma_matches_independent_ewald_split():
    """gamma_IJ - gamma_IK against an Ewald-split evaluation of the same lattice sum:
    sum_L [KO - 1/r] in real space (r^-3 tail) + the Coulomb part by standard Ewald
    (erfc real-space sum + Gaussian-damped reciprocal sum).  Constants cancel in
    the differences; the truncated r^-3 tail limits agreement to ~2e-4, far below
    the ~1e-2 size of the differences (a factor or sign error would show)."""
    from scipy.special import erfc
    s = inputs.diamond_si(1, 0.07, seed=2, kgrid="gamma")
    lat, pos = s["lattice"], s["pos"]
    omega = abs(np.linalg.det(lat))
    a = 1.0 / inputs.U_HUBBARD
    alpha = 0.35
    rc = 150.0
    m = int(np.ceil(rc / lat[0, 0])) + 1
    r = np.arange(-m, m + 1)
    L = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3) @ lat
    rec = 2 * np.pi * np.linalg.inv(lat).T
    mg = 12
    rg = np.arange(-mg, mg + 1)
    G = np.stack(np.meshgrid(rg, rg, rg, indexing="ij"), -1).reshape(-1, 3) @ rec
    G2 = (G ** 2).sum(1)
    G, G2 = G[G2 > 0], G2[G2 > 0]

    def lattice_sum(d):
        x = np.sqrt(((d[None, :] + L) ** 2).sum(1))
        short = np.sum(1.0 / np.sqrt(x[x <= rc] ** 2 + a * a) - 1.0 / x[x <= rc])
        real = np.sum(erfc(alpha * x[x <= 40.0]) / x[x <= 40.0])
        recip = 4 * np.pi / omega * np.sum(np.exp(-G2 / (4 * alpha ** 2)) / G2 * np.cos(G @ d))
        return short + real + recip
    g = s["gamma"]
    ref = [lattice_sum(pos[j] - pos[0]) for j in (1, 4, 6)]
    for (j, k), (rj, rk) in zip([(1, 4), (4, 6)], [(ref[0], ref[1]), (ref[1], ref[2])]):
        assert abs((g[0, j] - g[0, k]) - (rj - rk)) < 5e-4
    assert abs(g[0, 1] - g[0, 4]) > 5e-3


def test_config_shapes():
    s, A, n = inputs.config("si8_pulse")
    assert s["orb_offset"][-1] == 32 and s["kpt"].shape == (8, 3) and A.shape == (n + 1, 3)
    assert abs(s["wk"].sum() - 1.0) < 1e-15
    assert s["blk_ijl"].dtype == np.int32


@pytest.mark.parametrize("kind,nk", [("gamma", 1), ("mp2", 8), ("gc2", 8)])
def test_kpoint_sets(kind, nk):
    k, w = inputs.kpoints(kind)
    assert k.shape == (nk, 3)
    np.testing.assert_allclose(w.sum(), 1.0)
    # every set is closed under k -> -k modulo reciprocal lattice vectors
    for kk in k:
        assert np.any(np.all(np.abs(((k + kk + 0.5) % 1.0) - 0.5) < 1e-12, axis=1))


def test_coordination_numbers():
    """Diamond: 4 nearest neighbours at a sqrt(3)/4 = 4.44 bohr, the next shell at
    a/sqrt(2) = 7.26 bohr, so every atom is 4-coordinated with the 2.85 A (5.39 bohr) cut-off,
    in the cell and in a supercell (periodic images counted).  Pulling one atom 2 bohr away
    from one neighbour along their bond makes both 3-coordinated."""
    for n in (1, 2):
        s = inputs.diamond_si(n, 0.0, seed=0, kgrid="gamma")
        assert np.all(inputs.coordination_numbers(s) == 4)
    s = inputs.diamond_si(2, 0.0, seed=0, kgrid="gamma")
    pos = np.array(s["pos"], float)
    lat = np.asarray(s["lattice"], float)
    d = pos - pos[0]
    d -= np.round(d @ np.linalg.inv(lat)) @ lat
    r = np.linalg.norm(d, axis=1)
    j = int(np.argmin(np.where(r > 1e-8, r, np.inf)))
    pos[0] -= 2.0 * d[j] / r[j]
    s2 = dict(s)
    s2["pos"] = pos
    cn = inputs.coordination_numbers(s2)
    assert cn[0] == 3 and cn[j] == 3
    assert np.sum(cn == 4) == len(cn) - 2


def test_laser_sweep_fields():
    """Sec. 3.3: 20 fs sin^2 pulses at 2.3 / 3.9 / 6.0 eV, 10^12 W/cm^2 (E0 = 0.00534 au) along x."""
    fields, n = inputs.laser_sweep(0.2)
    assert n == round(20.0 / 0.0241888432658 / 0.2)
    assert len(fields) == 3
    for f, ev in zip(fields, (2.3, 3.9, 6.0)):
        w = ev / 27.211386245988
        ref = inputs.pulse_field(n, 0.2, 0.00534, w, duration=20.0 / 0.0241888432658)
        assert np.allclose(f, ref, rtol=0, atol=1e-12)
        assert np.all(f[:, 1:] == 0.0)
    # the field's intensity: I = (c / 8 pi) E0^2 in atomic units -> W/cm^2
    e0_au = 0.00534
    i_wcm2 = 3.50944758e16 * e0_au ** 2
    assert abs(i_wcm2 / 1e12 - 1.0) < 0.01
