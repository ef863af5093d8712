"""Fourier transform of the truncated free-space Green's function (oracle; test
infrastructure only).

Sec. 5.2 replaces g(x, y) = exp(i kappa0 |x-y|) / (4 pi |x-y|) on the aperture by
G = g * 1_{|x-y| <= R}, R = sqrt(2) max(a, b), and needs its 2-D Fourier
transform at frequency xi = (xi1, xi2), which depends on rho = |xi| only:

    F(G)(rho) = int_0^R int_0^{2 pi} exp(-2 pi i rho r cos t) exp(i kappa0 r)/(4 pi) dt dr
              = 1/2 int_0^R J0(2 pi rho r) exp(i kappa0 r) dr .

The paper prints the prefactor 1/(4 pi) in front of the radial integral; the
angular integral contributes 2 pi J0, so the prefactor is 1/2 (reading recorded
in the design notes).  The integrand is entire in r, so composite Gauss-Legendre
quadrature on panels no wider than pi / (2 pi rho + kappa0) converges
geometrically; 16 nodes per panel leave an error far below 1e-14 relative.  The
paper's own large-frequency scheme (Hankel asymptotics + Fresnel integrals) is
an approximation and is not what this oracle computes.
"""

import numpy as np
from scipy.special import j0

_NODES = 16


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def khat(rho, kappa0, R, nodes=_NODES):
    """1/2 int_0^R J0(2 pi rho r) exp(i kappa0 r) dr for an array of rho >= 0."""
    rho = np.asarray(rho, dtype=float)
    flat = rho.ravel()
    out = np.zeros(flat.shape, dtype=complex)
    x, w = _gl(nodes)
    omega = 2.0 * np.pi * flat + abs(kappa0)
    npan = np.maximum(1, np.ceil(omega * R / np.pi)).astype(int)
    for npv in np.unique(npan):
        sel = np.nonzero(npan == npv)[0]
        width = R / npv
        # node positions for all panels: (npv * nodes,)
        starts = np.arange(npv) * width
        r = (starts[:, None] + 0.5 * width * (x[None, :] + 1.0)).ravel()
        wt = np.tile(0.5 * width * w, npv)
        ez = np.exp(1j * kappa0 * r) * wt           # (nr,)
        # chunk over rho to bound memory
        chunk = max(1, int(4_000_000 // r.size))
        for s in range(0, sel.size, chunk):
            idx = sel[s:s + chunk]
            vals = j0(2.0 * np.pi * flat[idx, None] * r[None, :])
            out[idx] = 0.5 * (vals @ ez)
    return out.reshape(rho.shape)


def khat_zero(kappa0, R):
    """Closed form at rho = 0: 1/2 int_0^R exp(i kappa0 r) dr."""
    if kappa0 == 0:
        return 0.5 * R
    return (np.exp(1j * kappa0 * R) - 1.0) / (2j * kappa0)
