"""Interior back-substitution and field synthesis (oracle; test infrastructure
only).

(EInter) recovers the interior levels from the aperture values; with the
per-mode profiles of `zsystem` this is  E_{l,j}^{mn} = P_{l,j}^{mn} E_l^{mn}
(+ Q_{l,j}^{mn} E_3^{mn} for l = 1, 2 in a layered fill).  The field follows from
the truncated series (E123F) evaluated on the grid, written here as explicit
cos/sin matrices:

  E1(x1_p, x2_q, x3_j), p = 0..Nx, q = 1..Ny-1   (cos x1, sin x2)
  E2(x1_p, x2_q, x3_j), p = 1..Nx-1, q = 0..Ny   (sin x1, cos x2)
  E3(x1_p, x2_q, x3_j), p = 1..Nx-1, q = 1..Ny-1 (sin x1, sin x2)

for levels j = 1..Nz (the aperture included; the bottom level is fixed by the
wall conditions).  At an interface level E3 is the upper layer's value.
The flat output of one direction is, level by level, [E1 | E2 | E3] row-major.
"""

import numpy as np

from .geometry import Cavity
from .zsystem import Profiles


def synth_mats(cav: Cavity):
    M, N = cav.M, cav.N
    px = np.arange(cav.nx + 1)
    py = np.arange(cav.ny + 1)
    cosx = np.cos(np.pi * np.outer(px, np.arange(0, M + 1)) / cav.nx)
    sinx = np.sin(np.pi * np.outer(px[1:-1], np.arange(1, M + 1)) / cav.nx)
    cosy = np.cos(np.pi * np.outer(py, np.arange(0, N + 1)) / cav.ny)
    siny = np.sin(np.pi * np.outer(py[1:-1], np.arange(1, N + 1)) / cav.ny)
    return cosx, sinx, cosy, siny


def level_coeffs(cav: Cavity, prof: Profiles, x, j):
    """Modal coefficients of the three components at level j (EInter)."""
    e1, e2, e3 = cav.split(x)
    c1 = prof.P1[:, :, j] * e1
    c1[1:, :] += prof.Q1[1:, :, j] * e3
    c2 = prof.P2[:, :, j] * e2
    c2[:, 1:] += prof.Q2[:, 1:, j] * e3
    c3 = prof.P3[:, :, j] * e3
    return c1, c2, c3


def samples_per_level(cav: Cavity):
    nx, ny = cav.nx, cav.ny
    return (nx + 1) * (ny - 1) + (nx - 1) * (ny + 1) + (nx - 1) * (ny - 1)


def field_level(cav: Cavity, prof: Profiles, x, j, mats=None):
    cosx, sinx, cosy, siny = mats if mats is not None else synth_mats(cav)
    c1, c2, c3 = level_coeffs(cav, prof, x, j)
    f1 = cosx @ c1 @ siny.T
    f2 = sinx @ c2 @ cosy.T
    f3 = sinx @ c3 @ siny.T
    return np.concatenate([f1.ravel(), f2.ravel(), f3.ravel()])


def field(cav: Cavity, prof: Profiles, x, levels=None):
    """Field samples of one direction for the given levels (default 1..Nz),
    shape (len(levels), samples_per_level)."""
    if levels is None:
        levels = range(1, cav.nz + 1)
    mats = synth_mats(cav)
    return np.stack([field_level(cav, prof, x, j, mats) for j in levels])


def field_point(cav: Cavity, prof: Profiles, x, comp, j, p, q):
    """One field sample computed on its own (for sampled parity checks at sizes
    where the full field is too large): component comp in {1,2,3}, level j,
    node (p, q)."""
    c = level_coeffs(cav, prof, x, j)[comp - 1]
    M, N = cav.M, cav.N
    if comp == 1:
        bx = np.cos(np.pi * p * np.arange(0, M + 1) / cav.nx)
        by = np.sin(np.pi * q * np.arange(1, N + 1) / cav.ny)
    elif comp == 2:
        bx = np.sin(np.pi * p * np.arange(1, M + 1) / cav.nx)
        by = np.cos(np.pi * q * np.arange(0, N + 1) / cav.ny)
    else:
        bx = np.sin(np.pi * p * np.arange(1, M + 1) / cav.nx)
        by = np.sin(np.pi * q * np.arange(1, N + 1) / cav.ny)
    return bx @ c @ by
