"""Singular integrals of the transparent boundary condition by the FFT route of
Sec. 5 (oracle; test infrastructure only).

Sec. 5.1 reduces every coefficient of (sig1)-(sig3) and their Appendix A
counterparts to three integrals over the aperture Gamma = [0,a] x [0,b]:

    I1^{mn}_k = <cs_mn, G * cs_k>,  I2^{mn}_k = <sc_mn, G * sc_k>,
    I3^{mn}_k = <cc_mn, G * cc_k>,

with cs_k(y) = cos(k1 pi y1/a) sin(k2 pi y2/b) etc. and the weakly singular kernel
g(x, y) = exp(i kappa0 |x-y|)/(4 pi |x-y|).  Sec. 5.2 evaluates the inner
integral I_k(x) = int F(y) G(x-y) dy as F^{-1}(F(F) F(G)) and the outer integral
by the trapezoid rule.  The discrete rule written out here (and binding for the
CUDA path) is:

  * the convolution is periodised with period Lx = pad*a, Ly = pad_y*b; for
    x, y in Gamma and the truncation radius R = sqrt(2) max(a,b) no image
    contributes while pad*a > a + R and pad_y*b > b + R (pad_y = pad = 4 for
    apertures up to about 2:1; a 4:1 aperture needs pad_y = 8 along its short
    side);
  * the inverse transform is the Fourier series on that torus truncated to the
    symmetric box |j1| <= Px/2 - 1, |j2| <= Py/2 - 1 with Px = pad*Nx,
    Py = pad_y*Ny (so the torus grid of spacing a/Nx, b/Ny contains the
    aperture nodes):
    I_k(x) = (Lx Ly)^{-1} sum_j F(F)(j/L) F(G)(|j/L|) exp(2 pi i j.x/L);
  * F(F) is the exact transform of the truncated basis function, separable into
    1-D factors  f^c_k(xi) = [E(xi - k/2a) + E(xi + k/2a)]/2 and
    f^s_k(xi) = [E(xi - k/2a) - E(xi + k/2a)]/(2i) with
    E(nu) = int_0^a exp(-2 pi i nu y) dy = (1 - exp(-2 pi i nu a))/(2 pi i nu),
    E(0) = a  (the paper's closed form for F(F), with the missing factor i
    restored);
  * F(G) is the radial integral of `khat`;
  * the outer integral is the trapezoid rule on x1_p = p a/Nx, x2_q = q b/Ny.

Each step is a dense matrix here (numpy matmul as the only library step).

Variant outer='parseval' (the symmetric form of the next rows of the plan,
not used by the CUDA path): the outer integral is taken exactly as well, by
Parseval's identity on the torus, <phi_m, I_k> = (Lx Ly)^{-1} sum_j
conj(F(phi_m))(j/L) F(G)(|j/L|) F(phi_k)(j/L): the same frequency box and
kernel table, with the test functions transformed exactly like the trial
functions, so each block is Phi^H diag(F(G)) Phi, complex symmetric, and a
dense contraction.
"""

import numpy as np

from .geometry import Cavity
from .khat import khat, khat_paper


def freq_index(P):
    """Symmetric frequency box -(P/2-1) .. (P/2-1) (the Nyquist line is left out
    so that the box, and with it every mirror symmetry of the problem, is
    symmetric)."""
    h = P // 2 - 1
    return np.arange(-h, h + 1)


def _E(D, a, pad):
    """E(nu) at nu = D / (2 pad a) for integer D."""
    D = np.asarray(D, dtype=float)
    nu = D / (2.0 * pad * a)
    safe = np.where(D == 0, 1.0, nu)
    val = (1.0 - np.exp(-2j * np.pi * safe * a)) / (2j * np.pi * safe)
    return np.where(D == 0, a + 0j, val)


def phi_matrix(kind, ks, js, a, pad):
    """Phi[j, k] = exact 1-D Fourier transform at xi = j / (pad a) of
    cos(k pi y / a) 1_[0,a](y)  (kind 'c')  or  sin(k pi y / a) 1_[0,a](y) ('s')."""
    js = np.asarray(js)[:, None]
    ks = np.asarray(ks)[None, :]
    em = _E(2 * js - pad * ks, a, pad)
    ep = _E(2 * js + pad * ks, a, pad)
    if kind == 'c':
        return 0.5 * (em + ep)
    return (em - ep) / 2j


def idft_matrix(nodes, js, P):
    """X[p, j] = exp(2 pi i j p / P): the torus Fourier series at x_p = p a/Nx."""
    return np.exp(2j * np.pi * np.outer(nodes, js) / P)


def trap_matrix(kind, ms, n_int, a):
    """T[m, p] = w_p cos(m pi p / n_int) or w_p sin(...), trapezoid weights
    w_p = (a / n_int) (1/2 at p = 0 and p = n_int)."""
    p = np.arange(n_int + 1)
    w = np.full(n_int + 1, a / n_int)
    w[0] *= 0.5
    w[-1] *= 0.5
    arg = np.pi * np.outer(ms, p) / n_int
    base = np.cos(arg) if kind == 'c' else np.sin(arg)
    return base * w[None, :]


class TBCOperator:
    """The three convolution-projection maps of a cavity, as dense factors.

    apply(kind, C):  C[k1, k2] (coefficients of the basis of type `kind`,
    'cs', 'sc' or 'cc', over the full ranges k1 = 0..M or 1..M etc.) ->
    out[m, n] = sum_k I^{mn}_k C[k] over the same index ranges.
    """

    def __init__(self, cav: Cavity, kh=None, scheme='quadrature', outer='trapezoid'):
        """scheme: 'quadrature' (the reference F(G)) or 'paper' (the
        approximate large-frequency scheme of Sec. 5.2, `khat_paper`).
        outer: 'trapezoid' (rule D) or 'parseval' (exact outer integral)."""
        if outer not in ('trapezoid', 'parseval'):
            raise ValueError("outer must be 'trapezoid' or 'parseval'")
        self.outer = outer
        self.cav = cav
        self._khat = khat if scheme == 'quadrature' else khat_paper
        a, b, nx, ny = cav.a, cav.b, cav.nx, cav.ny
        padx, pady = cav.pad, cav.pad_y
        self.Px, self.Py = padx * nx, pady * ny
        self.jx, self.jy = freq_index(self.Px), freq_index(self.Py)
        self.Lx, self.Ly = padx * a, pady * b
        R = np.sqrt(2.0) * max(a, b)
        if padx * a <= a + R or pady * b <= b + R:
            raise ValueError("period too short for the truncated kernel")
        if kh is None:
            kh = self._kernel_table(R)
        self.Kh = kh
        M, N = cav.M, cav.N
        rng = {'c': (np.arange(0, M + 1), np.arange(0, N + 1)),
               's': (np.arange(1, M + 1), np.arange(1, N + 1))}
        self._fx, self._fy = {}, {}
        self._tx, self._ty = {}, {}
        for kind in 'cs':
            kx = rng[kind][0]
            ky = rng[kind][1]
            self._fx[kind] = phi_matrix(kind, kx, self.jx, a, padx)
            self._fy[kind] = phi_matrix(kind, ky, self.jy, b, pady)
            self._tx[kind] = trap_matrix(kind, kx, nx, a)
            self._ty[kind] = trap_matrix(kind, ky, ny, b)
        self._ex = idft_matrix(np.arange(nx + 1), self.jx, self.Px) / self.Lx
        self._ey = idft_matrix(np.arange(ny + 1), self.jy, self.Py) / self.Ly

    def _kernel_table(self, R):
        """F(G) on the frequency box, evaluated once per distinct radius: the
        table is even in j1 and in j2 (and depends on j1^2 + j2^2 only when the
        two periods agree)."""
        ax, ay = np.abs(self.jx), np.abs(self.jy)
        if self.Lx == self.Ly:
            key = ax[:, None] ** 2 + ay[None, :] ** 2
            uniq, inv = np.unique(key, return_inverse=True)
            vals = self._khat(np.sqrt(uniq) / self.Lx, self.cav.kappa0, R)
            return vals[inv].reshape(key.shape)
        ux, ix = np.unique(ax, return_inverse=True)
        uy, iy = np.unique(ay, return_inverse=True)
        rho = np.sqrt((ux[:, None] / self.Lx) ** 2 + (uy[None, :] / self.Ly) ** 2)
        q = self._khat(rho, self.cav.kappa0, R)
        return q[ix][:, iy]

    def factors(self, kind):
        """X[m, j1] (projection after inverse DFT) and Phi[j1, k1] per axis."""
        kx, ky = kind[0], kind[1]
        if self.outer == 'parseval':
            Xx = self._fx[kx].conj().T / self.Lx
            Xy = self._fy[ky].conj().T / self.Ly
        else:
            Xx = self._tx[kx] @ self._ex
            Xy = self._ty[ky] @ self._ey
        return (Xx, self._fx[kx]), (Xy, self._fy[ky])

    def apply(self, kind, C):
        """Matrix-free I C for one coefficient array (or a batch, leading axes)."""
        kx, ky = kind[0], kind[1]
        V = self._fx[kx] @ C @ self._fy[ky].T           # frequency box
        V = V * self.Kh
        if self.outer == 'parseval':                       # exact outer integral
            return (self._fx[kx].conj().T / self.Lx) @ V @ (self._fy[ky].conj() / self.Ly)
        U = self._ex @ V @ self._ey.T                      # aperture nodes
        return self._tx[kx] @ U @ self._ty[ky].T           # trapezoid projection

    def diag(self, kind):
        """The diagonal I^{mn}_{mn} over the full index ranges of `kind`:
        sum_j X(m,j1) Phi(j1,m) Kh(j1,j2) Y(n,j2) Psi(j2,n)."""
        (Xx, Fx), (Xy, Fy) = self.factors(kind)
        return (Xx * Fx.T) @ self.Kh @ (Xy * Fy.T).T

    def dense(self, kind, mm=None, nn=None):
        """I[m, n, k1, k2] for the full index ranges of `kind` (small grids),
        or, with mm, nn, for the modes m, k1 <= mm and n, k2 <= nn only (the
        factor rows and columns of those modes; the rest of each range is
        cut off)."""
        (Xx, Fx), (Xy, Fy) = self.factors(kind)
        if mm is not None:
            cx = mm + 1 if kind[0] == 'c' else mm      # 'c' ranges start at 0, 's' at 1
            cy = nn + 1 if kind[1] == 'c' else nn
            Xx, Fx, Xy, Fy = Xx[:cx], Fx[:, :cx], Xy[:cy], Fy[:, :cy]
        T1 = np.einsum('mj,jl,jk->mkl', Xx, self.Kh, Fx, optimize=True)
        return np.einsum('nl,mkl,lq->mnkq', Xy, T1, Fy, optimize=True)
