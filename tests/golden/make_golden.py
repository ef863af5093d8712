"""Writes the oracle regression fixtures of tests/golden/ (run from the
repository root: python tests/golden/make_golden.py).

The paper prints no solution values of a worked example: its tables give
operation counts (Table 1) and timings (Tables 2-5), and its RCS curves are
figures.  So the stored values here are the oracle's own, written by this
script, which calls only oracle/ and the input lists of workloads.py.  They
are regression values, not pins (the pins are in tests/test_oracle_pins.py):
tests/test_golden.py checks that the oracle still reproduces them, so a change
of the oracle's arithmetic shows up as a changed fixture in the same commit.

Cases:
  small       32 x 32 x 32, eps = 1, kappa0 = 8 pi, normal incidence (the
              homogeneous fill of Sec. 3), dense solve of (EJ1)
  layered16   the four-layer fill of Sec. 4 at 16 x 16 x 16 (same points
              per wavelength in the densest layer as the 512^2 workload),
              one seeded oblique direction, dense solve of (uT1)
  small_kept10
              the small case with the aperture expansion truncated to the
              modes m, n <= 10 (the few-mode runs of Sec. 7, Table 2): the
              kept block assembled from its restricted pieces and solved
              densely (residual of the kept rows)
  layered16_parseval
              the layered16 case with the outer integral of Sec. 5.2 taken
              exactly (the Parseval form), dense solve
Each case stores n_ap, the solve residual, the backscatter RCS in both
polarisations, the 2-norm of the aperture vector, aperture coefficients at
12 seeded indices among those above 1e-6 of the largest, and field samples
at 12 seeded (component, level, p, q) nodes, all to 17 significant digits.
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads  # noqa: E402
from oracle.aperture import ApertureSystem  # noqa: E402
from oracle.excitation import rhs  # noqa: E402
from oracle.field import field_point  # noqa: E402
from oracle.geometry import Cavity, Layer  # noqa: E402
from oracle.rcs import backscatter  # noqa: E402
from oracle.solver import solve  # noqa: E402
from oracle.tbc import TBCOperator  # noqa: E402

KEPT = 10   # modes kept per axis in small_kept10


def case_inputs(name):
    if name.startswith('small'):
        w = workloads.workload('small')
    else:
        w = workloads.scaled('layered4', 16, ndir=1)
    return w


def sample_nodes(cav, rng, n=12):
    """Seeded (component, level, p, q) nodes inside each component's grid."""
    out = []
    for _ in range(n):
        comp = int(rng.integers(1, 4))
        j = int(rng.integers(1, cav.nz + 1))
        if comp == 1:
            p, q = int(rng.integers(0, cav.nx + 1)), int(rng.integers(1, cav.ny))
        elif comp == 2:
            p, q = int(rng.integers(1, cav.nx)), int(rng.integers(0, cav.ny + 1))
        else:
            p, q = int(rng.integers(1, cav.nx)), int(rng.integers(1, cav.ny))
        out.append((comp, j, p, q))
    return out


def compute(name):
    w = case_inputs(name)
    cav = Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], w['kappa0'],
                 layers=[Layer(n, e) for n, e in w['layers']])
    th, ph, al = w['theta'][:1], w['phi'][:1], w['alpha'][:1]
    if name == 'small_kept10':
        sysm = ApertureSystem(cav)
        b = rhs(cav, th[0], ph[0], al[0])
        k = sysm.kept_modes(KEPT, KEPT)
        x = sysm.solve_kept(b, KEPT, KEPT)[0]
        A = sysm.dense_kept(KEPT, KEPT)
        resid = np.linalg.norm(A @ x[k] - b[k]) / np.linalg.norm(b[k])
        prof = sysm.prof
    elif name == 'layered16_parseval':
        sysm = ApertureSystem(cav, tbc=TBCOperator(cav, outer='parseval'))
        b = rhs(cav, th[0], ph[0], al[0])
        A = sysm.dense()
        x = np.linalg.solve(A, b)
        resid = np.linalg.norm(A @ x - b) / np.linalg.norm(b)
        prof = sysm.prof
    else:
        sol = solve(cav, th, ph, al, method='dense')
        x, resid, prof = sol.x[0], sol.resid[0], sol.prof
    rng = np.random.Generator(np.random.PCG64(77))
    # coefficients that the selection rules of normal incidence do not zero
    # (entries at rounding level would make the fixture machine-dependent)
    live = np.flatnonzero(np.abs(x) >= 1e-6 * np.abs(x).max())
    idx = sorted(int(i) for i in rng.choice(live, min(12, live.size), replace=False))
    nodes = sample_nodes(cav, rng)
    vals = dict(
        n_ap=cav.n_ap,
        resid=float(resid),
        rcs_theta=float(backscatter(cav, x, th[0], ph[0], 'theta')),
        rcs_phi=float(backscatter(cav, x, th[0], ph[0], 'phi')),
        norm=float(np.linalg.norm(x)),
        aperture=[(i, complex(x[i])) for i in idx],
        field=[(c, j, p, q, complex(field_point(cav, prof, x, c, j, p, q)))
               for c, j, p, q in nodes],
    )
    return vals


def write(name, vals, path):
    with open(path, 'w') as f:
        f.write('# oracle regression values, case %s; written by tests/golden/make_golden.py\n' % name)
        f.write('# from oracle/ only (the paper prints no solution values to pin against)\n')
        f.write('n_ap %d\n' % vals['n_ap'])
        f.write('resid %.17g\n' % vals['resid'])
        f.write('rcs_theta %.17g\n' % vals['rcs_theta'])
        f.write('rcs_phi %.17g\n' % vals['rcs_phi'])
        f.write('norm %.17g\n' % vals['norm'])
        for i, v in vals['aperture']:
            f.write('aperture %d %.17g %.17g\n' % (i, v.real, v.imag))
        for c, j, p, q, v in vals['field']:
            f.write('field %d %d %d %d %.17g %.17g\n' % (c, j, p, q, v.real, v.imag))


def read(path):
    out = dict(aperture=[], field=[])
    with open(path) as f:
        for line in f:
            if line.startswith('#') or not line.strip():
                continue
            t = line.split()
            if t[0] == 'n_ap':
                out['n_ap'] = int(t[1])
            elif t[0] in ('resid', 'rcs_theta', 'rcs_phi', 'norm'):
                out[t[0]] = float(t[1])
            elif t[0] == 'aperture':
                out['aperture'].append((int(t[1]), complex(float(t[2]), float(t[3]))))
            elif t[0] == 'field':
                out['field'].append((int(t[1]), int(t[2]), int(t[3]), int(t[4]),
                                     complex(float(t[5]), float(t[6]))))
    return out


CASES = ('small', 'layered16', 'small_kept10', 'layered16_parseval')

if __name__ == '__main__':
    for name in CASES:
        write(name, compute(name), os.path.join(HERE, '%s_oracle.txt' % name))
        print('wrote', name)
