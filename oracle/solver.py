"""End-to-end oracle driver (test infrastructure only).

Algorithm I / II of Sec. 6 in the paper's order:
  Step 1  the TBC coefficients (I1, I2, I3 by the FFT route) and g1, g2,
  Step 2  the per-mode eliminations in x3 (profiles, top relations),
  Step 3  the aperture system (EJ1)/(uT1): dense LU when small, else GMRES,
then (EInter) and the field synthesis (E123F).
"""

import time

import numpy as np

from .aperture import ApertureSystem
from .excitation import rhs
from .field import field
from .geometry import Cavity
from .tbc import TBCOperator
from .zsystem import Profiles

DENSE_LIMIT = 6000


class OracleSolution:
    def __init__(self, cav, system, x, resid, timings):
        self.cav = cav
        self.system = system
        self.x = x                      # (ndir, n_ap) aperture coefficients
        self.resid = resid
        self.timings = timings

    @property
    def prof(self):
        return self.system.prof

    def field(self, d, levels=None):
        return field(self.cav, self.prof, self.x[d], levels)


def solve(cav: Cavity, thetas, phis, alphas, method='auto', gmres_rtol=1e-13):
    t0 = time.perf_counter()
    tbc = TBCOperator(cav)
    t1 = time.perf_counter()
    prof = Profiles(cav)
    t2 = time.perf_counter()
    sysm = ApertureSystem(cav, prof, tbc)
    B = np.array([rhs(cav, t, p, a) for t, p, a in zip(thetas, phis, alphas)])
    if method == 'auto':
        method = 'dense' if cav.n_ap <= DENSE_LIMIT else 'gmres'
    if method == 'dense':
        A = sysm.dense()
        t3 = time.perf_counter()
        x = np.linalg.solve(A, B.T).T
        resid = np.linalg.norm(x @ A.T - B, axis=1) / np.linalg.norm(B, axis=1)
    else:
        t3 = time.perf_counter()
        x, resid = sysm.solve_gmres(B, rtol=gmres_rtol)
    t4 = time.perf_counter()
    timings = dict(singular=t1 - t0, eliminate=t2 - t1, assemble=t3 - t2, solve=t4 - t3)
    return OracleSolution(cav, sysm, x, resid, timings)
