"""Pins of the spectrum oracle (Eqs. 15, 16) against closed forms."""
import numpy as np

from oracle import spectrum


def _exact(w, w0, G, T):
    """int_0^T e^{i w t} cos(w0 t) e^{-G t} dt in closed form."""
    out = 0.0
    for s in (1.0, -1.0):
        z = 1j * (w + s * w0) - G
        out = out + 0.5 * (np.exp(z * T) - 1.0) / z
    return out


def test_damped_cosine_has_the_analytic_lorentzian():
    """J(t) = cos(w0 t) e^{-g t}: int_0^T e^{iwt} J e^{-t/tau0} dt has a closed form
    (a pair of Lorentzians 1/2 [1/(G - i(w + w0)) + 1/(G - i(w - w0))], G = g + 1/tau0,
    plus the e^{-G T} truncation term)."""
    dt, T, w0, g, tau0, E0 = 0.01, 400.0, 0.3, 0.01, 200.0, 2.5
    t = np.arange(int(T / dt) + 1) * dt
    J = np.stack([np.cos(w0 * t) * np.exp(-g * t), np.zeros_like(t), -2 * np.cos(w0 * t) * np.exp(-g * t)], 1)
    w = np.linspace(0.05, 0.8, 31)
    s = spectrum.conductivity(J, dt, E0, w, tau0)
    G = g + 1.0 / tau0
    ref = _exact(w, w0, G, t[-1]) / E0
    np.testing.assert_allclose(s[:, 0], ref, rtol=1e-5, atol=1e-6)
    lor = 0.5 * (1 / (G - 1j * (w + w0)) + 1 / (G - 1j * (w - w0))) / E0
    assert np.abs(s[:, 0] - lor).max() < 0.05 * np.abs(lor).max()
    np.testing.assert_allclose(s[:, 2], -2 * ref, rtol=1e-5, atol=1e-6)
    assert np.all(s[:, 1] == 0)


def test_trapezoid_is_second_order():
    w0, g, tau0 = 0.5, 0.0, 50.0
    errs = []
    for dt in (0.2, 0.1):
        t = np.arange(int(300 / dt) + 1) * dt
        J = np.cos(w0 * t)[:, None] * np.ones((1, 3))
        s = spectrum.conductivity(J, dt, 1.0, np.array([0.4]), tau0)[0, 0]
        G = g + 1.0 / tau0
        errs.append(abs(s - _exact(0.4, w0, G, t[-1])))
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_dielectric_definition():
    sig = np.array([[1.0 + 2.0j, 0, 0], [0.5j, 0, 0]])
    w = np.array([0.5, 2.0])
    e = spectrum.dielectric(sig, w)
    np.testing.assert_allclose(e[0, 0], 1 + 4j * np.pi * (1 + 2j) / 0.5)
    np.testing.assert_allclose(e[1, 0], 1 + 4j * np.pi * 0.5j / 2.0)
    np.testing.assert_allclose(e[:, 1], 1.0)
