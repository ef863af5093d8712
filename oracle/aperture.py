"""The reduced aperture system (EJ1) / (uT1) (oracle; test infrastructure only).

Unknowns x = [E1; E2; E3] at the aperture level (Appendix A ordering).  Rows:

 row 1, (m,n) in N1 (ENU14 with E_{1,Nz-1} eliminated by the top relation):
   (-1 + tau1) E1 + (m pi h / a + vs1) E3[m,n] (m >= 1)
     + (h/q) [ 2 kappa0^2 <cs_mn, G*u1>  -  (2 n pi / b) <cc_mn, G*w> ]  = g1
 row 2, (m,n) in N2 (ENU24):
   (-1 + tau2) E2 + (n pi h / b + vs2) E3[m,n] (n >= 1)
     + (h/c) [ 2 kappa0^2 <sc_mn, G*u2>  +  (2 m pi / a) <cc_mn, G*w> ]  = g2
 row 3, (m,n) in N3 (ENU34, with the factor h on both coupling terms):
   (m pi h / a) E1 + (n pi h / b) E2 + (-1 + tau3) E3 = 0

where u1 = sum_k E1^k cs_k, u2 = sum_k E2^k sc_k and
w = sum_{N1} (k2 pi/b) E1^k cc_k - sum_{N2} (k1 pi/a) E2^k cc_k = div_Gamma(z x E).
The bracketed terms are the F1 + H1 and G1 (resp. H2 and F2 + G2) blocks of
Sec. 3 and Appendix A after the integration by parts of Sec. 5.1
(G~1 = H~1 = -(n pi/b) I3,  G~2 = H~2 = -(m pi/a) I3).
tau_l = -1/r_JJ (EJJ1) or -1/r_II (uTT1); vs_l = s_l / r_II is the layered
coupling of (uT1) column 3 (zero for a homogeneous fill).

Sign of the TBC operator (reading).  Taking the curl of (EGa2) gives
curl E^s = +2 kappa0^2 int (z x E) . G0 ds (curl curl of g M is
grad div (g M) + kappa0^2 g M off the aperture); (ENU) prints -2 kappa0^2.  With
the printed sign the operator T of (ENU1) equals, for every evanescent Fourier
component, the interior value of d1 E3 - d3 E1 itself, so the reduced system is
singular in the continuum limit and the aperture absorbs instead of radiates.
The rows above therefore carry F, G, H with the sign that follows from (EGa2):
T(E) is the half-space exterior admittance z x curl E^s.  The printed sign of
the data g (z x curl of incident plus reflected wave) is unaffected.
"""

import numpy as np
import scipy.linalg as sla
from scipy.sparse.linalg import LinearOperator, gmres

from .geometry import Cavity
from .excitation import q_norm
from .tbc import TBCOperator
from .zsystem import Profiles


class ApertureSystem:
    def __init__(self, cav: Cavity, prof: Profiles = None, tbc: TBCOperator = None):
        self.cav = cav
        self.prof = prof if prof is not None else Profiles(cav)
        self.tbc = tbc if tbc is not None else TBCOperator(cav)
        M, N = cav.M, cav.N
        self.q, self.cn = q_norm(cav)
        self.mx = np.arange(0, M + 1) * np.pi / cav.a      # m pi / a, m = 0..M
        self.ny = np.arange(0, N + 1) * np.pi / cav.b      # n pi / b, n = 0..N

    # -- pieces --------------------------------------------------------------
    def w_coeffs(self, e1, e2):
        """cc-coefficients of w = div_Gamma(z x E), k1 = 0..M, k2 = 0..N."""
        M, N = self.cav.M, self.cav.N
        wc = np.zeros(e1.shape[:-2] + (M + 1, N + 1), dtype=complex)
        wc[..., :, 1:] += self.ny[None, 1:] * e1
        wc[..., 1:, :] -= self.mx[1:, None] * e2
        return wc

    def local(self, e1, e2, e3):
        """The cavity (non-TBC) part of (EJ1)/(uT1)."""
        p, h = self.prof, self.cav.h
        y1 = (-1.0 + p.tau1) * e1
        y1[..., 1:, :] += (self.mx[1:, None] * h + p.vs1[1:, :]) * e3
        y2 = (-1.0 + p.tau2) * e2
        y2[..., :, 1:] += (self.ny[None, 1:] * h + p.vs2[:, 1:]) * e3
        y3 = (self.mx[1:, None] * h) * e1[..., 1:, :] \
            + (self.ny[None, 1:] * h) * e2[..., :, 1:] + (-1.0 + p.tau3) * e3
        return y1, y2, y3

    def apply(self, x):
        cav = self.cav
        e1, e2, e3 = cav.split(x)
        y1, y2, y3 = self.local(e1, e2, e3)
        k2 = 2.0 * cav.kappa0 ** 2
        h = cav.h
        U1 = self.tbc.apply('cs', e1)
        U2 = self.tbc.apply('sc', e2)
        W = self.tbc.apply('cc', self.w_coeffs(e1, e2))
        y1 = y1 + (h / self.q)[:, None] * (k2 * U1 - 2.0 * self.ny[None, 1:] * W[:, 1:])
        y2 = y2 + (h / self.cn)[None, :] * (k2 * U2 + 2.0 * self.mx[1:, None] * W[1:, :])
        return cav.join(y1, y2, y3)

    def dense(self):
        """Assemble the full n_ap x n_ap matrix (small grids only)."""
        cav = self.cav
        eye = np.eye(cav.n_ap, dtype=complex)
        e1, e2, e3 = cav.split(eye)
        y1, y2, y3 = self.local(e1, e2, e3)
        return cav.join(y1, y2, y3).T + self.dense_tbc()

    def dense_tbc(self):
        """The TBC part alone (F, G, H blocks of (ENUGa)) as a dense matrix."""
        cav = self.cav
        n1, n2 = cav.n1, cav.n2
        nap = cav.n_ap
        A = np.zeros((nap, nap), dtype=complex)
        k2 = 2.0 * cav.kappa0 ** 2
        h = cav.h
        I1 = self.tbc.dense('cs')            # [m, n, k1, k2] over (M+1, N) x (M+1, N)
        I2 = self.tbc.dense('sc')            # (M, N+1) x (M, N+1)
        I3 = self.tbc.dense('cc')            # (M+1, N+1) x (M+1, N+1)
        s1 = (h / self.q)[:, None]
        s2 = (h / self.cn)[None, :]
        # row 1 <- E1 via I1 and via w (k2 pi / b) I3
        B11 = k2 * s1[:, :, None, None] * I1
        B11 -= (s1 * 2.0 * self.ny[None, 1:])[:, :, None, None] * \
            I3[:, 1:, :, 1:] * self.ny[None, None, None, 1:]
        # row 1 <- E2 via w: -(k1 pi/a) I3
        B12 = (s1 * 2.0 * self.ny[None, 1:])[:, :, None, None] * \
            I3[:, 1:, 1:, :] * self.mx[None, None, 1:, None]
        # row 2 <- E1 via w
        B21 = (s2 * 2.0 * self.mx[1:, None])[:, :, None, None] * \
            I3[1:, :, :, 1:] * self.ny[None, None, None, 1:]
        # row 2 <- E2 via I2 and w
        B22 = k2 * s2[:, :, None, None] * I2
        B22 -= (s2 * 2.0 * self.mx[1:, None])[:, :, None, None] * \
            I3[1:, :, 1:, :] * self.mx[None, None, 1:, None]
        A[:n1, :n1] += B11.reshape(n1, n1)
        A[:n1, n1:n1 + n2] += B12.reshape(n1, n2)
        A[n1:n1 + n2, :n1] += B21.reshape(n2, n1)
        A[n1:n1 + n2, n1:n1 + n2] += B22.reshape(n2, n2)
        return A

    def block_diagonal(self):
        """The 3x3 (2x2 / 1x1 at m = 0 or n = 0) diagonal blocks of the reduced
        matrix that couple E1, E2, E3 of one mode (m, n); B[m, n, r, c] with
        component order (E1, E2, E3) and absent components left as identity."""
        cav = self.cav
        M, N, h = cav.M, cav.N, cav.h
        k2 = 2.0 * cav.kappa0 ** 2
        p = self.prof
        d1 = self.tbc.diag('cs')       # (M+1, N)   n = 1..N
        d2 = self.tbc.diag('sc')       # (M, N+1)   m = 1..M
        d3 = self.tbc.diag('cc')       # (M+1, N+1)
        B = np.zeros((M + 1, N + 1, 3, 3), dtype=complex)
        for r in range(3):
            B[:, :, r, r] = 1.0
        mx = self.mx[:, None]
        ny = self.ny[None, :]
        sq = (h / self.q)[:, None]
        sc = (h / self.cn)[None, :]
        # E1 row (n >= 1)
        B[:, 1:, 0, 0] = (-1.0 + p.tau1) + sq * (k2 * d1 - 2.0 * ny[:, 1:] ** 2 * d3[:, 1:])
        B[1:, 1:, 0, 1] = (sq * 2.0 * ny * mx * d3)[1:, 1:]
        B[1:, 1:, 0, 2] = mx[1:] * h + p.vs1[1:, :]
        # E2 row (m >= 1)
        B[1:, 1:, 1, 0] = (sc * 2.0 * mx * ny * d3)[1:, 1:]
        B[1:, :, 1, 1] = (-1.0 + p.tau2) + sc * (k2 * d2 - 2.0 * mx[1:] ** 2 * d3[1:, :])
        B[1:, 1:, 1, 2] = ny[:, 1:] * h + p.vs2[:, 1:]
        # E3 row
        B[1:, 1:, 2, 0] = (mx * h)[1:] + 0 * ny[:, 1:]
        B[1:, 1:, 2, 1] = (ny * h)[:, 1:] + 0 * mx[1:]
        B[1:, 1:, 2, 2] = -1.0 + p.tau3
        return B

    def preconditioner(self):
        """x -> (block diagonal)^{-1} x, used only to speed up GMRES."""
        cav = self.cav
        Binv = np.linalg.inv(self.block_diagonal())

        def apply(v):
            e1, e2, e3 = cav.split(v)
            M, N = cav.M, cav.N
            V = np.zeros((M + 1, N + 1, 3), dtype=complex)
            V[:, 1:, 0] = e1
            V[1:, :, 1] = e2
            V[1:, 1:, 2] = e3
            Y = np.einsum('mnrc,mnc->mnr', Binv, V)
            return cav.join(Y[:, 1:, 0], Y[1:, :, 1], Y[1:, 1:, 2])
        return apply

    # -- solves --------------------------------------------------------------
    def solve_dense(self, b):
        A = self.dense()
        return sla.solve(A, np.asarray(b).T).T

    def kept_modes(self, mm, nn):
        """Unknowns of the modes (m, n) with m <= mm and n <= nn: the truncated
        aperture expansion of the paper's runs (Sec. 7, Table 2 keeps
        M ~ 2a/lambda modes).  Boolean mask in Appendix A order."""
        M, N = self.cav.M, self.cav.N
        def keep(m0, n0):
            m, n = np.meshgrid(np.arange(m0, M + 1), np.arange(n0, N + 1), indexing='ij')
            return ((m <= mm) & (n <= nn)).ravel()
        return np.concatenate([keep(0, 1), keep(1, 0), keep(1, 1)])

    def solve_truncated(self, b, mm, nn):
        """Galerkin restriction of (EJ1)/(uT1) to the kept modes: the rows and
        columns of the dropped modes removed, a dense solve of the rest, zeros
        for the dropped unknowns."""
        A = self.dense()
        k = self.kept_modes(mm, nn)
        b = np.atleast_2d(b)
        X = np.zeros(b.shape, dtype=complex)
        X[:, k] = sla.solve(A[np.ix_(k, k)], b[:, k].T).T
        return X

    def dense_kept(self, mm, nn):
        """The kept block A[k][:, k] of dense() for the modes m <= mm, n <= nn,
        assembled from restricted pieces: the cavity part couples the three
        components of one mode only, and each TBC integral is a product of
        per-axis factors, so the block needs the factor rows and columns of the
        kept modes alone (TBCOperator.dense with mm, nn).  Rows and columns in
        the order of kept_modes: E1 (m = 0..mm, n = 1..nn), E2 (m = 1..mm,
        n = 0..nn), E3 (m = 1..mm, n = 1..nn), m-major."""
        cav = self.cav
        h = cav.h
        k2 = 2.0 * cav.kappa0 ** 2
        p = self.prof
        n1, n2, n3 = (mm + 1) * nn, mm * (nn + 1), mm * nn
        nk = n1 + n2 + n3
        mx, ny = self.mx[:mm + 1], self.ny[:nn + 1]
        I1 = self.tbc.dense('cs', mm, nn)            # m, k1 = 0..mm;  n, k2 = 1..nn
        I2 = self.tbc.dense('sc', mm, nn)            # m, k1 = 1..mm;  n, k2 = 0..nn
        I3 = self.tbc.dense('cc', mm, nn)            # m, k1 = 0..mm;  n, k2 = 0..nn
        s1 = (h / self.q[:mm + 1])[:, None]
        s2 = (h / self.cn[:nn + 1])[None, :]
        A = np.zeros((nk, nk), dtype=complex)
        # TBC blocks (the F, G, H blocks of (ENUGa) with w = div_Gamma(z x E))
        B11 = k2 * s1[:, :, None, None] * I1
        B11 -= (s1 * 2.0 * ny[None, 1:])[:, :, None, None] * \
            I3[:, 1:, :, 1:] * ny[None, None, None, 1:]
        B12 = (s1 * 2.0 * ny[None, 1:])[:, :, None, None] * \
            I3[:, 1:, 1:, :] * mx[None, None, 1:, None]
        B21 = (s2 * 2.0 * mx[1:, None])[:, :, None, None] * \
            I3[1:, :, :, 1:] * ny[None, None, None, 1:]
        B22 = k2 * s2[:, :, None, None] * I2
        B22 -= (s2 * 2.0 * mx[1:, None])[:, :, None, None] * \
            I3[1:, :, 1:, :] * mx[None, None, 1:, None]
        A[:n1, :n1] = B11.reshape(n1, n1)
        A[:n1, n1:n1 + n2] = B12.reshape(n1, n2)
        A[n1:n1 + n2, :n1] = B21.reshape(n2, n1)
        A[n1:n1 + n2, n1:n1 + n2] = B22.reshape(n2, n2)
        # cavity part, mode by mode (the rows of local())
        m1, q1 = np.meshgrid(np.arange(0, mm + 1), np.arange(1, nn + 1), indexing='ij')
        m2, q2 = np.meshgrid(np.arange(1, mm + 1), np.arange(0, nn + 1), indexing='ij')
        m3, q3 = np.meshgrid(np.arange(1, mm + 1), np.arange(1, nn + 1), indexing='ij')
        i1 = (m1 * nn + q1 - 1).ravel()
        i2 = (n1 + (m2 - 1) * (nn + 1) + q2).ravel()
        i3 = (n1 + n2 + (m3 - 1) * nn + q3 - 1).ravel()
        A[i1, i1] += (-1.0 + p.tau1[m1, q1 - 1]).ravel()
        A[i2, i2] += (-1.0 + p.tau2[m2 - 1, q2]).ravel()
        A[i3, i3] += (-1.0 + p.tau3[m3 - 1, q3 - 1]).ravel()
        # E3 columns of rows 1 and 2, and row 3
        j1 = (m3 * nn + q3 - 1).ravel()                    # E1 unknown of mode (m, n), m, n >= 1
        j2 = (n1 + (m3 - 1) * (nn + 1) + q3).ravel()       # E2 unknown of the same mode
        A[j1, i3] += (m3 * np.pi / cav.a * h + p.vs1[m3, q3 - 1]).ravel()
        A[j2, i3] += (q3 * np.pi / cav.b * h + p.vs2[m3 - 1, q3]).ravel()
        A[i3, j1] += (m3 * np.pi / cav.a * h).ravel()
        A[i3, j2] += (q3 * np.pi / cav.b * h).ravel()
        return A

    def solve_kept(self, b, mm, nn):
        """solve_truncated with the kept block assembled by dense_kept (the
        same system; feasible where the full dense matrix is not)."""
        A = self.dense_kept(mm, nn)
        k = self.kept_modes(mm, nn)
        b = np.atleast_2d(b)
        X = np.zeros(b.shape, dtype=complex)
        X[:, k] = sla.solve(A, b[:, k].T).T
        return X

    def solve_gmres(self, b, rtol=1e-13, restart=200, maxiter=200):
        """Restarted GMRES (SciPy) on the matrix-free operator with the block
        diagonal as preconditioner; the true residual is recomputed afterwards.
        Returns (x, relative residuals)."""
        nap = self.cav.n_ap
        op = LinearOperator((nap, nap), matvec=self.apply, dtype=complex)
        pre = LinearOperator((nap, nap), matvec=self.preconditioner(), dtype=complex)
        b = np.atleast_2d(b)
        xs, res = [], []
        for bi in b:
            x, info = gmres(op, bi, rtol=rtol, atol=0.0, restart=restart,
                            maxiter=maxiter, M=pre)
            r = np.linalg.norm(self.apply(x) - bi) / np.linalg.norm(bi)
            xs.append(x)
            res.append(r)
        return np.array(xs), np.array(res)
