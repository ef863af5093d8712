"""Per-mode finite-difference systems along x3 (oracle; test infrastructure only).

For every Fourier mode (m, n) the paper reduces Maxwell's equations to 1-D
Helmholtz problems in x3 (ode1x3)/(ode3x3), discretised by the second-order
scheme (dfE1M)/(dfE3M) on the levels j = 1..Nz-1 with the aperture value
E_{l,Nz} (the paper's E_{l,J+1}) as data.  In a layered fill (Sec. 4) the
levels shared by two layers carry the discrete continuity conditions
(con12), (con22), (con32), (con42-1), (con42-2), their E2 analogue from
(con51), and (con61) with a forward difference above and a backward difference
below the interface.  The closing remark of Sec. 4 extends this to more than
two layers by repeating the interface step; that is what is assembled here.

Each per-mode system is assembled in full and solved directly with banded LU
with partial pivoting (Algorithm I/II, Step 2) -- no ratio recurrence, no
determinant formulas.  Solving for unit aperture data gives the profiles

    E_{l,j} = P_{l,j} E_{l,Nz} + Q_{l,j} E_{3,Nz}     (l = 1, 2)
    E_{3,j} = P_{3,j} E_{3,Nz}

(Q = 0 in a homogeneous cavity) and the top relations used by (EJ1)/(uT1):
    E_{l,Nz-1} = tau_l E_{l,Nz} + varsigma_l E_{3,Nz}.
In the notation of (EJJ1) and (uTT1): tau = -1/r_JJ (or -1/r_II), and
varsigma_l = s_l / r_II.  At an interface level E3 is double valued
(eps_U u3 = eps_D v3, (con32)); the profile stores the value of the upper layer.
"""

import numpy as np
from scipy.linalg import solve_banded

from .geometry import Cavity


def _band_set(ab, u, i, j, v):
    ab[u + i - j, j] += v


def e3_profile(cav: Cavity, m: int, n: int):
    """Solve the E3 system of mode (m, n) in N3 for unit aperture value.

    Unknowns, bottom-up: one value per ordinary level, and (D, U) -- the values
    of the lower and upper layer -- at each interface level.
    Rows:
      ordinary level j of layer l: E_{j-1} + (sigma_l - 2) E_j + E_{j+1} = 0,
        neighbours taken on layer l's side; at j = 1 the Neumann condition
        E_{3,0} = E_{3,1} of (dfE3M) gives (sigma_l - 1) E_1 + E_2 = 0;
      interface level j: (E_{j+1} - U_j) - (D_j - E_{j-1}) = 0   (con61)
                         eps_U U_j - eps_D D_j = 0                (con32)
    Returns (P, D_at_interfaces): P has length Nz+1 with P[0] the value at the
    bottom level (equal to P[1] by the Neumann condition), P[Nz] = 1, and the
    upper-layer value at interface levels; D maps interface level -> lower value.
    """
    nz = cav.nz
    lay_of = cav.level_layer()
    ifaces = {lev: (up, lo) for lev, up, lo in cav.interfaces()}
    lam = cav.lam(m, n)
    # variable indexing
    var = {}
    k = 0
    for j in range(1, nz):
        if j in ifaces:
            var[(j, 'D')] = k
            var[(j, 'U')] = k + 1
            k += 2
        else:
            var[(j, 'x')] = k
            k += 1
    nvar = k

    def vid(j, layer):
        """index of the unknown at level j as seen from layer `layer`"""
        if j in ifaces:
            up, lo = ifaces[j]
            return var[(j, 'U')] if layer == up else var[(j, 'D')]
        return var[(j, 'x')]

    L = U = 2
    ab = np.zeros((L + U + 1, nvar), dtype=complex)
    rhs = np.zeros(nvar, dtype=complex)
    for j in range(1, nz):
        if j in ifaces:
            up, lo = ifaces[j]
            ia, ib = var[(j, 'D')], var[(j, 'U')]
            # (con61): (E_{j+1} - U_j) - (D_j - E_{j-1}) = 0
            if j + 1 == nz:
                rhs[ia] -= 1.0
            else:
                _band_set(ab, U, ia, vid(j + 1, up), 1.0)
            _band_set(ab, U, ia, ib, -1.0)
            _band_set(ab, U, ia, ia, -1.0)
            _band_set(ab, U, ia, vid(j - 1, lo), 1.0)
            # (con32): eps_U U_j - eps_D D_j = 0
            _band_set(ab, U, ib, ib, cav.layers[up].eps)
            _band_set(ab, U, ib, ia, -cav.layers[lo].eps)
        else:
            li = lay_of[j]
            i = var[(j, 'x')]
            s = cav.sigma(li, lam)
            diag = s - 2.0
            if j == 1:
                diag += 1.0          # Neumann: E_{3,0} = E_{3,1}
            else:
                _band_set(ab, U, i, vid(j - 1, li), 1.0)
            _band_set(ab, U, i, i, diag)
            if j + 1 == nz:
                rhs[i] -= 1.0
            else:
                _band_set(ab, U, i, vid(j + 1, li), 1.0)
    sol = solve_banded((L, U), ab, rhs)
    P = np.zeros(nz + 1, dtype=complex)
    D = {}
    for j in range(1, nz):
        if j in ifaces:
            P[j] = sol[var[(j, 'U')]]
            D[j] = sol[var[(j, 'D')]]
        else:
            P[j] = sol[var[(j, 'x')]]
    P[0] = P[1]
    P[nz] = 1.0
    return P, D


def tangential_profiles(cav: Cavity, m: int, n: int, mu: float, p3=None):
    """Solve the E1 (mu = m pi / a) or E2 (mu = n pi / b) system of mode (m, n).

    Unknowns T_1..T_{Nz-1} (T_0 = 0 by (E12D), T_Nz = aperture value).
    Rows:
      ordinary level j of layer l: T_{j-1} + (sigma_l - 2) T_j + T_{j+1} = 0
      interface level j (upper U, lower D), from (con42-2) / the (con51)
      analogue with (con12), (con22), (con32):
          T_{j-1} - 2 T_j + T_{j+1} = mu h (1 - eps_U / eps_D) u3_j
      where u3_j is the upper-layer E3 value at the interface.
    `p3` is the E3 profile of the same (m, n) for unit E3 aperture value (None
    when the mode has no E3 partner or the cavity has no interface).
    Returns (P, Q), each of length Nz+1 (P[0] = Q[0] = 0, P[Nz] = 1, Q[Nz] = 0).
    """
    nz = cav.nz
    lay_of = cav.level_layer()[1:nz]                 # levels 1..Nz-1
    lam = cav.lam(m, n)
    k2 = cav.kappa0 ** 2 * np.array([l.eps for l in cav.layers])
    sig = cav.h ** 2 * (k2 - lam)
    diag = np.where(lay_of >= 0, sig[np.maximum(lay_of, 0)] - 2.0, -2.0 + 0j)
    ab = np.zeros((3, nz - 1), dtype=complex)
    ab[0, 1:] = 1.0
    ab[1, :] = diag
    ab[2, :-1] = 1.0
    rhs = np.zeros((nz - 1, 2), dtype=complex)
    rhs[-1, 0] = -1.0
    if p3 is not None:
        for lev, up, lo in cav.interfaces():
            coef = mu * cav.h * (1.0 - cav.layers[up].eps / cav.layers[lo].eps)
            rhs[lev - 1, 1] += coef * p3[lev]
    sol = solve_banded((1, 1), ab, rhs)
    P = np.zeros(nz + 1, dtype=complex)
    Q = np.zeros(nz + 1, dtype=complex)
    P[1:nz] = sol[:, 0]
    Q[1:nz] = sol[:, 1]
    P[nz] = 1.0
    return P, Q


def _e3_profile_homogeneous(cav: Cavity, m: int, n: int):
    """E3 system of (dfE3M) without interfaces: tridiagonal A2 + D."""
    nz = cav.nz
    s = cav.sigma(0, cav.lam(m, n))
    ab = np.zeros((3, nz - 1), dtype=complex)
    ab[0, 1:] = 1.0
    ab[1, :] = s - 2.0
    ab[1, 0] = s - 1.0                       # E_{3,0} = E_{3,1}
    ab[2, :-1] = 1.0
    rhs = np.zeros(nz - 1, dtype=complex)
    rhs[-1] = -1.0
    P = np.zeros(nz + 1, dtype=complex)
    P[1:nz] = solve_banded((1, 1), ab, rhs)
    P[0] = P[1]
    P[nz] = 1.0
    return P


def _profile_rows(cav: Cavity, ms):
    """Profiles of every mode in the rows m in `ms` (P3, then P1/Q1 and P2/Q2,
    which use P3 of the same (m, n) in a layered fill)."""
    N, nz = cav.N, cav.nz
    layered = len(cav.layers) > 1
    out = []
    for m in ms:
        p3 = np.zeros((N, nz + 1), dtype=complex) if m >= 1 else None
        if m >= 1:
            for n in range(1, N + 1):
                if layered:
                    p3[n - 1], _ = e3_profile(cav, m, n)
                else:
                    p3[n - 1] = _e3_profile_homogeneous(cav, m, n)
        p1 = np.zeros((N, nz + 1), dtype=complex)
        q1 = np.zeros_like(p1)
        for n in range(1, N + 1):
            d3 = p3[n - 1] if (layered and m >= 1) else None
            p1[n - 1], q1[n - 1] = tangential_profiles(cav, m, n, m * np.pi / cav.a, d3)
        p2 = q2 = None
        if m >= 1:
            p2 = np.zeros((N + 1, nz + 1), dtype=complex)
            q2 = np.zeros_like(p2)
            for n in range(0, N + 1):
                d3 = p3[n - 1] if (layered and n >= 1) else None
                p2[n], q2[n] = tangential_profiles(cav, m, n, n * np.pi / cav.b, d3)
        out.append((m, p3, p1, q1, p2, q2))
    return out


def _profile_rows_job(args):
    return _profile_rows(*args)


def _workers(cav: Cavity, workers):
    """Processes for the per-mode solves: one for small grids (where starting
    a pool costs more than it saves), else every core of this process."""
    if workers is not None:
        return max(1, int(workers))
    if cav.M * cav.N < 128 * 128:
        return 1
    try:
        import os
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:
        return 1


class Profiles:
    """All per-mode profiles of a cavity.

    P1[m, n-1, j], Q1[m, n-1, j]   E1 over N1, levels j = 0..Nz
    P2[m-1, n, j], Q2[m-1, n, j]   E2 over N2
    P3[m-1, n-1, j]                E3 over N3 (upper value at interfaces)
    tau1, tau2, tau3, vs1, vs2     top relations (level Nz-1) as 2-D arrays

    Every mode's system is solved on its own (the per-mode problems are
    independent); on large grids the rows m are shared out over a pool of
    processes (started with `spawn`), each solving whole rows exactly as a
    single process would.
    """

    def __init__(self, cav: Cavity, workers=None):
        M, N, nz = cav.M, cav.N, cav.nz
        self.P3 = np.zeros((M, N, nz + 1), dtype=complex)
        self.P1 = np.zeros((M + 1, N, nz + 1), dtype=complex)
        self.Q1 = np.zeros_like(self.P1)
        self.P2 = np.zeros((M, N + 1, nz + 1), dtype=complex)
        self.Q2 = np.zeros_like(self.P2)
        nw = _workers(cav, workers)
        rows = list(range(0, M + 1))
        parts = None
        if nw > 1:
            # a spawned worker re-imports the main script, so a script that
            # builds large profiles needs the usual `if __name__ == "__main__"`
            # guard; without it the pool fails and the rows are solved here
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            chunks = [rows[k::4 * nw] for k in range(4 * nw)]
            try:
                with ProcessPoolExecutor(nw, mp_context=mp.get_context("spawn")) as ex:
                    parts = list(ex.map(_profile_rows_job, [(cav, c) for c in chunks if c]))
            except Exception:
                parts = None
        if parts is None:
            parts = [_profile_rows(cav, rows)]
        for part in parts:
            for m, p3, p1, q1, p2, q2 in part:
                self.P1[m], self.Q1[m] = p1, q1
                if m >= 1:
                    self.P3[m - 1] = p3
                    self.P2[m - 1], self.Q2[m - 1] = p2, q2
        j = nz - 1
        self.tau1 = self.P1[:, :, j]
        self.tau2 = self.P2[:, :, j]
        self.tau3 = self.P3[:, :, j]
        self.vs1 = self.Q1[:, :, j]
        self.vs2 = self.Q2[:, :, j]
