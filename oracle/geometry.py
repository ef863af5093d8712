"""Cavity geometry, Fourier index sets and the vertical grid (oracle; test
infrastructure only).

Index sets (Sec. 3, after (ode3x3)):
    N1 = {0..M} x {1..N}   coefficients of E1 (cos x1, sin x2)
    N2 = {1..M} x {0..N}   coefficients of E2 (sin x1, cos x2)
    N3 = {1..M} x {1..N}   coefficients of E3 (sin x1, sin x2)
ordered m-major as in Appendix A.  The aperture vector is [E1; E2; E3] with
n_ap = 3MN + M + N entries.

Horizontal grid: x1_p = p a / Nx (p = 0..Nx), x2_q = q b / Ny, with M = Nx - 1 and
N = Ny - 1 modes (the reading that the Fourier truncation matches the grid).

Vertical grid (Sec. 3): x3^j = -c + j h, j = 0..Nz, h = c / Nz; level Nz is the
aperture (the paper's J + 1), levels 1..Nz-1 are the interior unknowns.
Layers (Sec. 4 and the closing remark of Sec. 4) are listed top to bottom by the
number of grid steps they span; the level shared by two layers is an interface
level where the continuity conditions (con12)-(con63) hold.
"""

from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass(frozen=True)
class Layer:
    """One horizontal slab of the cavity fill: `nlev` grid steps of height h and
    relative permittivity `eps` (complex)."""
    nlev: int
    eps: complex


@dataclass
class Cavity:
    """Geometry, discretisation and medium of one cavity problem.

    a, b, c   aperture [0,a] x [0,b], depth c (Sec. 2)
    nx, ny    horizontal grid intervals (M = nx-1, N = ny-1 Fourier modes)
    nz        vertical grid steps; h = c/nz; aperture at level nz
    kappa0    free-space wavenumber (Sec. 2)
    layers    top-to-bottom list of Layer; default one layer with eps = 1
    pad       period of the frequency-domain convolution in units of the
              aperture side (Lx = pad * a); part of the discrete TBC operator
    pad_y     the same along x2 (Ly = pad_y * b); 0 = pad.  A period must
              exceed the side plus the kernel's truncation radius, so a long
              narrow aperture needs a longer period along its short side
    """
    a: float
    b: float
    c: float
    nx: int
    ny: int
    nz: int
    kappa0: float
    layers: List[Layer] = field(default_factory=list)
    pad: int = 4
    pad_y: int = 0

    def __post_init__(self):
        if not self.pad_y:
            self.pad_y = self.pad
        if not self.layers:
            self.layers = [Layer(self.nz, 1.0 + 0j)]
        self.layers = [Layer(int(l.nlev), complex(l.eps)) for l in self.layers]
        if sum(l.nlev for l in self.layers) != self.nz:
            raise ValueError("layer level counts must sum to nz")
        if any(l.nlev < 2 for l in self.layers):
            raise ValueError("every layer must span at least two grid steps")
        if self.nx < 2 or self.ny < 2 or self.nz < 2:
            raise ValueError("grid too small")

    # -- sizes -------------------------------------------------------------
    @property
    def M(self):
        return self.nx - 1

    @property
    def N(self):
        return self.ny - 1

    @property
    def h(self):
        return self.c / self.nz

    @property
    def n1(self):
        return (self.M + 1) * self.N

    @property
    def n2(self):
        return self.M * (self.N + 1)

    @property
    def n3(self):
        return self.M * self.N

    @property
    def n_ap(self):
        return self.n1 + self.n2 + self.n3

    # -- layers on the level grid -----------------------------------------
    def level_layer(self):
        """For each level j = 0..nz the index (top-to-bottom) of the layer whose
        interior contains it, or -1 at interface levels, the bottom (j = 0) and
        the aperture (j = nz)."""
        out = np.full(self.nz + 1, -1, dtype=int)
        top = self.nz
        for li, lay in enumerate(self.layers):
            bot = top - lay.nlev
            out[bot + 1:top] = li
            top = bot
        return out

    def interfaces(self):
        """List of (level, upper_layer_index, lower_layer_index) for every
        interface level, from the top down."""
        res = []
        top = self.nz
        for li in range(len(self.layers) - 1):
            top -= self.layers[li].nlev
            res.append((top, li, li + 1))
        return res

    def sigma(self, layer_index, lam):
        """h^2 (kappa_l^2 - lambda_mn), the diagonal shift of (dfE1M)/(dfE3M)
        in layer l, with kappa_l^2 = kappa0^2 eps_l (Sec. 4; reading: the
        homogeneous algorithm of Sec. 3 uses kappa0^2 eps_r in D)."""
        k2 = self.kappa0 ** 2 * self.layers[layer_index].eps
        return self.h ** 2 * (k2 - lam)

    # -- modes -------------------------------------------------------------
    def lam(self, m, n):
        """(m pi / a)^2 + (n pi / b)^2 (ode1x3)."""
        return (m * np.pi / self.a) ** 2 + (n * np.pi / self.b) ** 2

    def modes1(self):
        M, N = self.M, self.N
        return [(m, n) for m in range(0, M + 1) for n in range(1, N + 1)]

    def modes2(self):
        M, N = self.M, self.N
        return [(m, n) for m in range(1, M + 1) for n in range(0, N + 1)]

    def modes3(self):
        M, N = self.M, self.N
        return [(m, n) for m in range(1, M + 1) for n in range(1, N + 1)]

    def split(self, x):
        """Split an aperture vector [E1; E2; E3] (last axis) into the three 2-D
        coefficient arrays E1[m, n-1], E2[m-1, n], E3[m-1, n-1]."""
        M, N = self.M, self.N
        x = np.asarray(x)
        e1 = x[..., :self.n1].reshape(x.shape[:-1] + (M + 1, N))
        e2 = x[..., self.n1:self.n1 + self.n2].reshape(x.shape[:-1] + (M, N + 1))
        e3 = x[..., self.n1 + self.n2:].reshape(x.shape[:-1] + (M, N))
        return e1, e2, e3

    def join(self, e1, e2, e3):
        lead = e1.shape[:-2]
        return np.concatenate([e1.reshape(lead + (-1,)), e2.reshape(lead + (-1,)),
                               e3.reshape(lead + (-1,))], axis=-1)
