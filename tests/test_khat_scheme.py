"""Pins of the oracle's restatement of the Sec. 5.2 large-frequency scheme for
F(G) (`khat_paper`, a measured variant of the kernel table), against
quadrature and special-function values that do not use its formulas."""

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import fresnel, j0

from oracle.khat import (_fresnel_asym, _tail_half, _tail_three_halves, integral_to_infinity,
                         khat, khat_paper)


def test_integral_to_infinity_is_the_laplace_limit():
    """int_0^inf J0(c r) e^{-(eps - i k) r} dr by quadrature equals
    1/sqrt(c^2 + (eps - i k)^2); its eps -> 0 limit is the closed form used."""
    for c, k in ((7.0, 3.0), (2.0, 5.0)):
        eps = 0.4
        re = quad(lambda r: j0(c * r) * np.exp(-eps * r) * np.cos(k * r), 0, 120, limit=2000)[0]
        im = quad(lambda r: j0(c * r) * np.exp(-eps * r) * np.sin(k * r), 0, 120, limit=2000)[0]
        assert abs(re + 1j * im - 1 / np.sqrt(c * c + (eps - 1j * k) ** 2)) < 1e-8
        lim = 1 / np.sqrt(c * c + (1e-12 - 1j * k) ** 2)
        assert abs(integral_to_infinity(c, k) - lim) < 1e-9 * abs(lim)


def test_fresnel_tail_matches_fourier_quadrature():
    """A(p) = int_Z^inf e^{ipz} z^{-1/2} dz: the corrected Fresnel form with
    SciPy's exact C, S equals QUADPACK's Fourier-integral value, for p of both
    signs; the z^{-3/2} integral by parts likewise."""
    for p, Z in ((0.7, 40.0), (-0.4, 60.0), (1.9, 150.0)):
        ref = quad(lambda z: z ** -0.5, Z, np.inf, weight='cos', wvar=p)[0] + \
            1j * quad(lambda z: z ** -0.5, Z, np.inf, weight='sin', wvar=p)[0]
        T = np.sqrt(2 * abs(p) * Z / np.pi)
        S, C = fresnel(T)
        v = np.sqrt(np.pi / (2 * abs(p))) * (1 + 1j - 2 * C - 2j * S)
        exact = v if p > 0 else np.conj(v)
        assert abs(exact - ref) < 1e-9 * abs(ref)
        # the module's version uses the asymptotic C, S: close for large T
        assert abs(_tail_half(np.array(p), Z) - ref) < 1e-4 * abs(ref)
        ref3 = quad(lambda z: z ** -1.5, Z, np.inf, weight='cos', wvar=p)[0] + \
            1j * quad(lambda z: z ** -1.5, Z, np.inf, weight='sin', wvar=p)[0]
        assert abs(2 * np.exp(1j * p * Z) / np.sqrt(Z) + 2j * p * exact - ref3) < 1e-8 * abs(ref3)


def test_fresnel_asymptotics_order():
    """The two-term expansions of C and S: error O(T^-9) against SciPy."""
    errs = []
    for T in (4.0, 8.0, 16.0):
        S, C = fresnel(T)
        Ca, Sa = _fresnel_asym(T)
        errs.append(max(abs(Ca - C), abs(Sa - S)))
    assert errs[0] < 1e-5 and errs[2] < 1e-9
    assert errs[0] / errs[1] > 100 and errs[1] / errs[2] > 100


def test_paper_scheme_converges_to_quadrature_away_from_the_ridge():
    """Away from 2 pi rho = kappa0 the scheme's error falls with c R like the
    dropped O(z^-2) terms of the asymptotic J0; near the ridge it fails (the
    reason it is a variant and not the default)."""
    k, R = 2 * np.pi * 25.6, np.sqrt(2.0)
    rho = np.array([50.0, 100.0, 200.0, 400.0])
    err = np.abs(khat_paper(rho, k, R) - khat(rho, k, R)) / np.abs(khat(rho, k, R))
    assert np.all(err[1:] < 1e-8)
    assert np.all(err[:-1] / err[1:] > 3.0)
    small = np.array([0.0, 3.0, 9.0])            # c R below the case-1 threshold
    assert np.allclose(khat_paper(small, k, R), khat(small, k, R), rtol=0, atol=1e-16)
    ridge = np.array([k / (2 * np.pi) + 0.05])
    assert abs(khat_paper(ridge, k, R) - khat(ridge, k, R))[0] > 1e-3 * abs(khat(ridge, k, R))[0]
