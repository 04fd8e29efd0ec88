"""Conductivity and dielectric function from the current of a kick (Eqs. 15, 16).

TEST INFRASTRUCTURE ONLY (see oracle/vgtb_oracle.py).

  sigma_ij(w) = (1/E0_j) int_0^T e^{i w t} J_i(t) f(t) dt,  f(t) = exp(-t / tau0)   (Eq. 15)
  eps_ij(w)   = 1 + 4 pi i sigma_ij(w) / w                                          (Eq. 16)

The paper does not state the quadrature; J is known at t_n = n dt, and the
integral is taken with the trapezoid rule over n = 0..N (a reading listed in
the design notes).  tau0 = 200 a.u. in the paper.
"""
import numpy as np


def conductivity(J, dt, E0, omegas, tau0=200.0):
    """sigma[w, i] for J[n, i] sampled at t_n = n dt (Eq. 15, trapezoid rule)."""
    J = np.asarray(J, float)
    t = np.arange(J.shape[0]) * dt
    wts = np.full(J.shape[0], dt)
    wts[0] = wts[-1] = 0.5 * dt
    kern = np.exp(1j * np.outer(np.asarray(omegas, float), t)) * (wts * np.exp(-t / tau0))[None, :]
    return kern @ J / E0


def dielectric(sigma, omegas):
    """eps[w, i] = 1 + 4 pi i sigma[w, i] / w (Eq. 16)."""
    return 1.0 + 4j * np.pi * sigma / np.asarray(omegas, float)[:, None]
