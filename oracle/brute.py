"""The full, unreduced discrete system on tiny grids (oracle; test
infrastructure only).

All levels of all modes are unknowns at once: the finite-difference rows
(dfE1M)/(dfE3M) per mode and level, the interface rows (con12)-(con63) of a
layered fill, and the aperture rows (ENU14), (ENU24), (ENU34) in their
unreduced form, i.e. with E_{l,Nz-1} still an unknown (the (ENUGa) system for a
homogeneous fill, (uNUGa) for a layered one).  Solving it densely checks the
Gaussian-elimination reduction to the aperture, (EJ1)/(uT1), and the
back-substitution (EInter) independently of `zsystem`: this module assembles
its own rows and never calls the per-mode solver.
"""

import numpy as np

from .geometry import Cavity


def solve_unreduced(cav: Cavity, tbc_dense, rhs):
    """Solve the global system.  `tbc_dense` is the TBC part of the aperture
    rows (n_ap x n_ap, acting on the aperture values), `rhs` the aperture data
    [g1; g2; 0].  Returns a dict comp -> array [mode, level j = 1..Nz] with the
    upper-layer value of E3 at interface levels."""
    nz, h = cav.nz, cav.h
    lay_of = cav.level_layer()
    ifaces = {lev: (up, lo) for lev, up, lo in cav.interfaces()}
    nI = len(ifaces)
    modes = {1: cav.modes1(), 2: cav.modes2(), 3: cav.modes3()}
    # unknown numbering
    idx = {}
    k = 0
    for comp in (1, 2, 3):
        for mi, _ in enumerate(modes[comp]):
            for j in range(1, nz + 1):
                if comp == 3 and j in ifaces:
                    idx[(comp, mi, j, 'D')] = k
                    idx[(comp, mi, j, 'U')] = k + 1
                    k += 2
                else:
                    idx[(comp, mi, j, 'x')] = k
                    k += 1
    nvar = k
    A = np.zeros((nvar, nvar), dtype=complex)
    b = np.zeros(nvar, dtype=complex)
    e3_of = {mn: i for i, mn in enumerate(modes[3])}

    def var(comp, mi, j, layer):
        if comp == 3 and j in ifaces:
            up, lo = ifaces[j]
            return idx[(comp, mi, j, 'U' if layer == up else 'D')]
        return idx[(comp, mi, j, 'x')]

    row = 0
    for comp in (1, 2, 3):
        for mi, (m, n) in enumerate(modes[comp]):
            lam = cav.lam(m, n)
            mu = m * np.pi / cav.a if comp == 1 else n * np.pi / cav.b
            for j in range(1, nz):
                if j in ifaces:
                    up, lo = ifaces[j]
                    if comp == 3:
                        # (con61) forward difference above, backward below
                        A[row, var(3, mi, j + 1, up)] += 1.0
                        A[row, var(3, mi, j, up)] -= 1.0
                        A[row, var(3, mi, j, lo)] -= 1.0
                        A[row, var(3, mi, j - 1, lo)] += 1.0
                        row += 1
                        # (con32)
                        A[row, var(3, mi, j, up)] += cav.layers[up].eps
                        A[row, var(3, mi, j, lo)] -= cav.layers[lo].eps
                        row += 1
                    else:
                        # (con42-1)/(con42-2) or the (con51) analogue, with
                        # (con12)/(con22) and (con32) substituted
                        A[row, var(comp, mi, j - 1, None)] += 1.0
                        A[row, var(comp, mi, j, None)] -= 2.0
                        A[row, var(comp, mi, j + 1, None)] += 1.0
                        if mu != 0.0 and m >= 1 and n >= 1:
                            coef = mu * h * (1.0 - cav.layers[up].eps / cav.layers[lo].eps)
                            A[row, var(3, e3_of[(m, n)], j, up)] -= coef
                        row += 1
                else:
                    li = lay_of[j]
                    s = h * h * (cav.kappa0 ** 2 * cav.layers[li].eps - lam)
                    if j == 1:
                        # bottom: E_{1,0} = E_{2,0} = 0;  E_{3,0} = E_{3,1}
                        A[row, var(comp, mi, 1, li)] += s - 2.0 + (1.0 if comp == 3 else 0.0)
                    else:
                        A[row, var(comp, mi, j - 1, li)] += 1.0
                        A[row, var(comp, mi, j, li)] += s - 2.0
                    A[row, var(comp, mi, j + 1, li)] += 1.0
                    row += 1
    # aperture rows (ENU14), (ENU24), (ENU34) -- unreduced
    top = cav.nz
    n1, n2 = cav.n1, cav.n2
    ap_var = [var(1, i, top, 0) for i in range(n1)] + \
             [var(2, i, top, 0) for i in range(n2)] + \
             [var(3, i, top, 0) for i in range(cav.n3)]
    below = [var(1, i, top - 1, 0) for i in range(n1)] + \
            [var(2, i, top - 1, 0) for i in range(n2)] + \
            [var(3, i, top - 1, 0) for i in range(cav.n3)]
    r0 = row
    for i in range(cav.n_ap):
        A[r0 + i, below[i]] += 1.0           # I^_l E_{l,J}
        A[r0 + i, ap_var[i]] -= 1.0          # -I^_l E_{l,J+1}
    for i, (m, n) in enumerate(modes[1]):    # I1 E3
        if m >= 1:
            A[r0 + i, ap_var[n1 + n2 + e3_of[(m, n)]]] += m * np.pi * h / cav.a
    for i, (m, n) in enumerate(modes[2]):    # I2 E3
        if n >= 1:
            A[r0 + n1 + i, ap_var[n1 + n2 + e3_of[(m, n)]]] += n * np.pi * h / cav.b
    e1_of = {mn: i for i, mn in enumerate(modes[1])}
    e2_of = {mn: i for i, mn in enumerate(modes[2])}
    for i, (m, n) in enumerate(modes[3]):    # F3 E1 + G3 E2
        A[r0 + n1 + n2 + i, ap_var[e1_of[(m, n)]]] += m * np.pi * h / cav.a
        A[r0 + n1 + n2 + i, ap_var[n1 + e2_of[(m, n)]]] += n * np.pi * h / cav.b
    for i in range(cav.n_ap):
        A[r0 + i, ap_var] += tbc_dense[i]
    b[r0:r0 + cav.n_ap] = rhs
    assert r0 + cav.n_ap == nvar
    sol = np.linalg.solve(A, b)
    out = {}
    for comp in (1, 2, 3):
        arr = np.zeros((len(modes[comp]), nz), dtype=complex)
        for mi in range(len(modes[comp])):
            for j in range(1, nz + 1):
                arr[mi, j - 1] = sol[var(comp, mi, j, 0 if j not in ifaces else ifaces[j][0])]
        out[comp] = arr
    return out
