"""Seeded synthetic workloads for the cavity solver.

This module only draws and lists inputs (geometry, grid, wavenumber,
permittivity profile, incident directions).  It holds none of the solver's
arithmetic and is shared by the tests, the benchmark and the oracle checks so
that both sides see identical inputs.  Random draws use numpy's PCG64.

Workloads (all a = b = 1, c = 0.5 in the same length unit):
  small      32 x 32 x 32, eps = 1, kappa0 = 8 pi (aperture 4 wavelengths),
             one normally incident wave (theta = phi = alpha = 0)
  dirs16     256 x 256 x 128, eps = 1, kappa0 = 2 pi * 25.6 (10 points per
             wavelength horizontally and vertically), 16 directions with
             theta ~ U[0, pi/3], phi ~ U[0, 2 pi), alpha = 0, seed 2
  layered4   512 x 512 x 256, four layers of 64 steps with eps a seeded
             permutation of {4+1i, 2+0.5i, 6+0.1i, 1} (top to bottom),
             kappa0 = 2 pi / (10 h sqrt(6)) (10 points per wavelength in the
             densest layer), 8 directions, seed 3
  rcs_sweep48()  48 cavities of uneven sizes (seed 4): side s in {64, 128,
             256, 512}, Nz = s/2, a = b = 1, c = 0.5; homogeneous with
             probability 1/2, else 2-4 layers of equal depth with
             Re eps ~ U[1, 6], Im eps ~ U[0, 1]; four wavenumbers f kappa_10,
             f in {0.25, 0.5, 0.75, 1}, kappa_10 at 10 points per wavelength in
             the densest layer; 64 directions each
"""

import numpy as np

EPS_SET = (4 + 1j, 2 + 0.5j, 6 + 0.1j, 1 + 0j)


def directions(ndir, seed, theta_max=np.pi / 3):
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.uniform(0.0, theta_max, ndir)
    phi = rng.uniform(0.0, 2 * np.pi, ndir)
    alpha = np.zeros(ndir)
    return theta, phi, alpha


def workload(name):
    """Return a dict with keys a, b, c, nx, ny, nz, kappa0, layers (top to
    bottom list of (nlev, eps)), theta, phi, alpha."""
    if name == 'small':
        return dict(a=1.0, b=1.0, c=0.5, nx=32, ny=32, nz=32, kappa0=8 * np.pi,
                    layers=[(32, 1.0 + 0j)], theta=np.zeros(1), phi=np.zeros(1),
                    alpha=np.zeros(1))
    if name == 'dirs16':
        th, ph, al = directions(16, 2)
        return dict(a=1.0, b=1.0, c=0.5, nx=256, ny=256, nz=128,
                    kappa0=2 * np.pi * 25.6, layers=[(128, 1.0 + 0j)],
                    theta=th, phi=ph, alpha=al)
    if name == 'layered4':
        rng = np.random.Generator(np.random.PCG64(3))
        order = rng.permutation(4)
        eps = [EPS_SET[i] for i in order]
        th, ph, al = directions(8, 3)
        nz = 256
        h = 0.5 / nz
        return dict(a=1.0, b=1.0, c=0.5, nx=512, ny=512, nz=nz,
                    kappa0=2 * np.pi / (10 * h * np.sqrt(6.0)),
                    layers=[(64, e) for e in eps], theta=th, phi=ph, alpha=al)
    raise KeyError(name)


def scaled(name, nx, ny=None, nz=None, ndir=None):
    """The workload `name` at a smaller grid with the same points per
    wavelength (used for parity cases the oracle finishes in seconds)."""
    w = dict(workload(name))
    ny = ny or nx
    f = nx / w['nx']
    nz = nz or max(4, int(round(w['nz'] * f)))
    w['kappa0'] = w['kappa0'] * f if name != 'layered4' else \
        2 * np.pi / (10 * (w['c'] / nz) * np.sqrt(6.0))
    if len(w['layers']) > 1:
        k = len(w['layers'])
        base = nz // k
        lev = [base] * k
        lev[0] += nz - base * k
        w['layers'] = [(l, e) for l, (_, e) in zip(lev, w['layers'])]
    else:
        w['layers'] = [(nz, w['layers'][0][1])]
    w['nx'], w['ny'], w['nz'] = nx, ny, nz
    if ndir is not None:
        for k in ('theta', 'phi', 'alpha'):
            w[k] = np.resize(w[k], ndir)
    return w


def rcs_sweep48(seed=4):
    """The 48-cavity backscatter sweep: a list of dicts with keys a, b, c, nx,
    ny, nz, layers, kappas (four wavenumbers), theta, phi, alpha (64 each)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(48):
        s = int(rng.choice([64, 128, 256, 512]))
        nz = s // 2
        if rng.uniform() < 0.5:
            layers = [(nz, 1.0 + 0j)]
        else:
            k = int(rng.integers(2, 5))
            base = nz // k
            lev = [base] * k
            lev[0] += nz - base * k
            eps = rng.uniform(1.0, 6.0, k) + 1j * rng.uniform(0.0, 1.0, k)
            layers = [(l, complex(e)) for l, e in zip(lev, eps)]
        h = 0.5 / nz
        emax = max(abs(e.real) for _, e in layers)
        k10 = 2 * np.pi / (10 * h * np.sqrt(emax))
        th, ph, al = directions(64, 1000 * seed + i)
        out.append(dict(a=1.0, b=1.0, c=0.5, nx=s, ny=s, nz=nz, layers=layers,
                        kappas=[f * k10 for f in (0.25, 0.5, 0.75, 1.0)],
                        theta=th, phi=ph, alpha=al))
    return out
