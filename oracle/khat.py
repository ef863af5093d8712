"""Fourier transform of the truncated free-space Green's function (oracle; test
infrastructure only).

Sec. 5.2 replaces g(x, y) = exp(i kappa0 |x-y|) / (4 pi |x-y|) on the aperture by
G = g * 1_{|x-y| <= R}, R = sqrt(2) max(a, b), and needs its 2-D Fourier
transform at frequency xi = (xi1, xi2), which depends on rho = |xi| only:

    F(G)(rho) = int_0^R int_0^{2 pi} exp(-2 pi i rho r cos t) exp(i kappa0 r)/(4 pi) dt dr
              = 1/2 int_0^R J0(2 pi rho r) exp(i kappa0 r) dr .

The paper prints the prefactor 1/(4 pi) in front of the radial integral; the
angular integral contributes 2 pi J0, so the prefactor is 1/2.  The integrand is
entire in r, so composite Gauss-Legendre quadrature on panels no wider than
pi / (2 pi rho + kappa0) converges geometrically (16 nodes per panel).  What
is left is the conditioning of the sum: the rounding of the arguments c r
(c = 2 pi rho) shifts every oscillation coherently, a relative error of about
c R * 1e-16 (1.4e-13 at c R = 1440, measured against a 30-digit evaluation):
`khat` is the reference table to that accuracy.

`khat_paper` is the paper's own scheme of Sec. 5.2, an approximation, kept as a
measured variant: quadrature for small frequencies and, for large c = 2 pi rho,
    int_0^R J0(c r) e^{i k r} dr = int_0^inf - int_R^inf,
with the first term in closed form and the tail from the two-term asymptotic
form of J0 and the Fresnel integrals with their two-term asymptotic
expansions.  Corrections to the printed formulas (the printed ones are
dimensionally inconsistent or garbled):
  int_0^inf J0(c r) e^{i k r} dr = 1/sqrt(c^2 - k^2) (c > k), i/sqrt(k^2 - c^2)
      (c < k)  [printed: 1/(c^2 - k^2)];
  int_Z^inf e^{i p z} z^{-1/2} dz = sqrt(pi/(2p)) (1 + i - 2 C(T) - 2i S(T)),
      T = sqrt(2 p Z / pi), p > 0  [printed prefactor: sqrt(pi)/(2p)]; p < 0 by
      complex conjugation;
  sin(z - pi/4) = (e^{i(z - pi/4)} - e^{-i(z - pi/4)}) / (2i)  [printed with
      the same exponential twice].
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
    jobs = []
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
        jobs.extend((sel[s:s + chunk], r, ez) for s in range(0, sel.size, chunk))

    def one(job):
        idx, r, ez = job
        vals = j0(2.0 * np.pi * flat[idx, None] * r[None, :])
        out[idx] = 0.5 * (vals @ ez)
    # chunks are independent (disjoint entries of out); J0 releases the GIL,
    # so large tables are shared out over threads
    if len(jobs) > 1 and flat.size > 100_000:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(one, jobs))
    else:
        for job in jobs:
            one(job)
    return out.reshape(rho.shape)


def _threads():
    try:
        import os
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:
        return 1


def khat_zero(kappa0, R):
    """Closed form at rho = 0: 1/2 int_0^R exp(i kappa0 r) dr."""
    if kappa0 == 0:
        return 0.5 * R
    return (np.exp(1j * kappa0 * R) - 1.0) / (2j * kappa0)


# ------------------------------------------------------------------ Sec. 5.2 scheme
# frequencies with c R below this use the quadrature (the paper's "small
# frequency" case; its threshold max|j| <= 10 expressed in c R)
PAPER_CASE1_CR = 20.0 * np.pi * np.sqrt(2.0)


def integral_to_infinity(c, k):
    """int_0^inf J0(c r) e^{i k r} dr: the limit eps -> 0+ of the Laplace
    transform 1/sqrt(c^2 + (eps - i k)^2), i.e. 1/sqrt(c^2 - k^2) for c > k and
    i/sqrt(k^2 - c^2) for c < k (infinite at c = k)."""
    c = np.asarray(c, dtype=float)
    d = c * c - k * k
    with np.errstate(divide='ignore'):
        return np.where(d > 0, 1.0 / np.sqrt(np.abs(d)) + 0j, 1j / np.sqrt(np.abs(d)))


def _fresnel_asym(T):
    """Fresnel C(T), S(T) from the two-term asymptotic expansions of Sec. 5.2
    (valid for T >> 1)."""
    u = np.pi * T * T
    f = (1.0 - 3.0 / (u * u)) / (np.pi * T)
    g = (1.0 - 15.0 / (u * u)) / (np.pi ** 2 * T ** 3)
    ph = 0.5 * u
    C = 0.5 + f * np.sin(ph) - g * np.cos(ph)
    S = 0.5 - f * np.cos(ph) - g * np.sin(ph)
    return C, S


def _tail_half(p, Z):
    """A(p) = int_Z^inf e^{i p z} z^{-1/2} dz, by the Fresnel form."""
    ap = abs(p)
    T = np.sqrt(2.0 * ap * Z / np.pi)
    C, S = _fresnel_asym(T)
    v = np.sqrt(np.pi / (2.0 * ap)) * (1.0 + 1j - 2.0 * C - 2j * S)
    return np.where(p > 0, v, np.conj(v))


def _tail_three_halves(p, Z):
    """B(p) = int_Z^inf e^{i p z} z^{-3/2} dz = 2 e^{i p Z}/sqrt(Z) + 2 i p A(p)."""
    return 2.0 * np.exp(1j * p * Z) / np.sqrt(Z) + 2j * p * _tail_half(p, Z)


def khat_paper(rho, kappa0, R, case1_cr=PAPER_CASE1_CR):
    """The Sec. 5.2 scheme for 1/2 int_0^R J0(2 pi rho r) exp(i kappa0 r) dr:
    quadrature where c R <= case1_cr, otherwise
      I = I_inf - (1/c) sqrt(2/pi) int_{cR}^inf [cos(z - pi/4) z^{-1/2}
                + sin(z - pi/4) z^{-3/2} / 8] e^{i kappa0 z / c} dz,
    each term expanded in e^{+-i(z - pi/4)} and integrated by _tail_half /
    _tail_three_halves with p = kappa0/c +- 1."""
    rho = np.asarray(rho, dtype=float)
    flat = rho.ravel()
    out = np.zeros(flat.shape, dtype=complex)
    c = 2.0 * np.pi * flat
    small = c * R <= case1_cr
    if np.any(small):
        out[small] = khat(flat[small], kappa0, R)
    big = ~small
    if np.any(big):
        cb = c[big]
        k = kappa0
        Z = cb * R
        inf = integral_to_infinity(cb, k)
        pp, pm = k / cb + 1.0, k / cb - 1.0
        e4 = np.exp(-0.25j * np.pi)
        # cos(z - pi/4) = (e^{-i pi/4} e^{iz} + e^{i pi/4} e^{-iz}) / 2
        cos_part = 0.5 * (e4 * _tail_half(pp, Z) + np.conj(e4) * _tail_half(pm, Z))
        # sin(z - pi/4) = (e^{-i pi/4} e^{iz} - e^{i pi/4} e^{-iz}) / (2i)
        sin_part = (e4 * _tail_three_halves(pp, Z) - np.conj(e4) * _tail_three_halves(pm, Z)) / 2j
        tail = np.sqrt(2.0 / np.pi) / cb * (cos_part + sin_part / 8.0)
        out[big] = 0.5 * (inf - tail)
    return out.reshape(rho.shape)
