"""Incident plane wave and the aperture data g1, g2 (oracle; test infrastructure
only).

Sec. 7 parametrises the incident field as
    E^inc = (cos(alpha) theta_hat + sin(alpha) phi_hat) exp(i kappa0 d . x),
    d = -(sin t cos f, sin t sin f, cos t),
so in the notation of Sec. 2, q = kappa0 d = (alpha1, alpha2, -beta) and
p = cos(alpha) theta_hat + sin(alpha) phi_hat.  With the reflected wave of Sec. 2
the TBC data is  z x curl(E^inc + E^ref) = (2i(alpha1 p3 + beta p1),
2i(alpha2 p3 + beta p2)) exp(i(alpha1 x1 + alpha2 x2))  on the aperture.

Galerkin testing with cos*sin (row 1, (c1mn)) and sin*cos (row 2, Appendix A)
and the scaling h/q^{(m,n)}, h/c^{(m,n)} give g1, g2 (Sec. 3 and Appendix A).
The test integrals g~ of (nosig) are taken with the same trapezoid rule on the
aperture nodes that Sec. 5.2 prescribes for the outer integrals of the TBC, so
the Galerkin rows use one quadrature throughout (reading recorded in the design
notes; T9 pins its O(h^2) distance from the closed form).
"""

import numpy as np

from .geometry import Cavity
from .tbc import trap_matrix


def incident(kappa0, theta, phi, alpha):
    """(alpha1, alpha2, beta, p) of the plane wave arriving from (theta, phi)."""
    st, ct = np.sin(theta), np.cos(theta)
    sf, cf = np.sin(phi), np.cos(phi)
    a1 = -kappa0 * st * cf
    a2 = -kappa0 * st * sf
    beta = kappa0 * ct
    th_hat = np.array([ct * cf, ct * sf, -st])
    ph_hat = np.array([-sf, cf, 0.0])
    p = np.cos(alpha) * th_hat + np.sin(alpha) * ph_hat
    return a1, a2, beta, p


def g_tilde(cav: Cavity, a1, a2):
    """Trapezoid values of (nosig) for row 1 (cos x1 sin x2, over N1) and its
    row-2 counterpart (sin x1 cos x2, over N2)."""
    M, N = cav.M, cav.N
    x = np.arange(cav.nx + 1) * cav.a / cav.nx
    y = np.arange(cav.ny + 1) * cav.b / cav.ny
    ex = np.exp(1j * a1 * x)
    ey = np.exp(1j * a2 * y)
    cx = trap_matrix('c', np.arange(0, M + 1), cav.nx, cav.a) @ ex
    sx = trap_matrix('s', np.arange(1, M + 1), cav.nx, cav.a) @ ex
    cy = trap_matrix('c', np.arange(0, N + 1), cav.ny, cav.b) @ ey
    sy = trap_matrix('s', np.arange(1, N + 1), cav.ny, cav.b) @ ey
    return np.outer(cx, sy), np.outer(sx, cy)


def q_norm(cav: Cavity):
    """q^{(m,n)} of (c1mn) over N1 (depends on m only) and c^{(m,n)} of Appendix
    A over N2 (depends on n only)."""
    ab = cav.a * cav.b
    q = np.full(cav.M + 1, ab / 4.0)
    q[0] = ab / 2.0
    cn = np.full(cav.N + 1, ab / 4.0)
    cn[0] = ab / 2.0
    return q, cn


def rhs(cav: Cavity, theta, phi, alpha):
    """Right-hand side [g1; g2; 0] of (EJ1) / (uT1) for one incident direction."""
    a1, a2, beta, p = incident(cav.kappa0, theta, phi, alpha)
    gt1, gt2 = g_tilde(cav, a1, a2)
    q, cn = q_norm(cav)
    h = cav.h
    g1 = (h / q)[:, None] * 2j * (a1 * p[2] + beta * p[0]) * gt1
    g2 = (h / cn)[None, :] * 2j * (a2 * p[2] + beta * p[1]) * gt2
    g3 = np.zeros((cav.M, cav.N), dtype=complex)
    return cav.join(g1, g2, g3)
