"""Backscatter radar cross section (oracle; test infrastructure only).

The paper defers the RCS formula to its reference on cavity-backed apertures
(Sec. 7).  It is derived here from (EGa2): in the far field
grad_y g(x, y) -> -i kappa0 x_hat g, and only the curl of the identity part of
G0 survives, so

    E^s(x) ~ (i kappa0 exp(i kappa0 r) / (2 pi r)) x_hat x L,
    L = int_Gamma (z x E)(y) exp(-i kappa0 x_hat . y) dy,   z x E = (-E2, E1, 0),

and sigma = lim 4 pi r^2 |E^s|^2 / |E^inc|^2 = (kappa0^2 / pi) |e . (x_hat x L)|^2.
For backscatter x_hat = -d; theta-theta uses e = theta_hat, phi-phi e = phi_hat.
L is separable per mode: the 1-D integrals int_0^a cos(m pi y/a) exp(-i g y) dy
and the sine counterpart have closed forms.
"""

import numpy as np

from .geometry import Cavity


def _ef(s, a):
    """int_0^a exp(-i s y) dy."""
    s = np.asarray(s, dtype=float)
    safe = np.where(s == 0, 1.0, s)
    return np.where(s == 0, a + 0j, (1.0 - np.exp(-1j * safe * a)) / (1j * safe))


def cos_int(ms, g, a):
    k = np.asarray(ms) * np.pi / a
    return 0.5 * (_ef(g - k, a) + _ef(g + k, a))


def sin_int(ms, g, a):
    k = np.asarray(ms) * np.pi / a
    return (_ef(g - k, a) - _ef(g + k, a)) / 2j


def far_vector(cav: Cavity, x, theta, phi):
    """L of the aperture field x for the observation direction (theta, phi)."""
    e1, e2, _ = cav.split(x)
    xh = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    g1, g2 = cav.kappa0 * xh[0], cav.kappa0 * xh[1]
    M, N = cav.M, cav.N
    C1x = cos_int(np.arange(0, M + 1), g1, cav.a)
    S1y = sin_int(np.arange(1, N + 1), g2, cav.b)
    S2x = sin_int(np.arange(1, M + 1), g1, cav.a)
    C2y = cos_int(np.arange(0, N + 1), g2, cav.b)
    I1 = C1x @ e1 @ S1y          # int E1
    I2 = S2x @ e2 @ C2y          # int E2
    return np.array([-I2, I1, 0.0 + 0j])


def backscatter(cav: Cavity, x, theta, phi, pol='theta'):
    """sigma for backscatter at (theta, phi): pol 'theta' -> e = theta_hat."""
    L = far_vector(cav, x, theta, phi)
    xh = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    if pol == 'theta':
        e = np.array([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)])
    else:
        e = np.array([-np.sin(phi), np.cos(phi), 0.0])
    v = np.dot(e, np.cross(xh, L))
    return cav.kappa0 ** 2 / np.pi * abs(v) ** 2
