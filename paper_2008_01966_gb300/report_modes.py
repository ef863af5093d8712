"""Truncated aperture expansion against the full one on the GPU.

The paper's runs keep few aperture modes (Sec. 7, Table 2: M ~ 2a/lambda);
this library keeps all M = nx - 1, N = ny - 1 by default.  For the 16-direction
256 x 256 x 128 workload (10 points per wavelength, 2a/lambda = 51.2) this
solves with modes_m = modes_n = K for several K and reports, against the
full-expansion solve (mixed precision, tolerance 1e-7): the relative L2
difference of the aperture coefficients, of the field and of the backscatter
RCS, the block steps and the solve time.

    python -m paper_2008_01966_gb300.report_modes
"""

import time

import numpy as np
import torch

import workloads
import paper_2008_01966_gb300 as gb


def run(w, modes, reps=3):
    g = gb.Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], precision="mixed",
                  gmres_tol=1e-7, modes_m=modes, modes_n=modes)
    g.prepare(w['kappa0'], w['layers'])
    out = None
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = g.solve(w['kappa0'], w['layers'], w['theta'], w['phi'], w['alpha'])
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    ap, fl, it, res = out
    sig = g.rcs(ap, w['theta'], w['phi'], "theta")
    return ap, fl, it, res, sig, min(ts)


def rel(a, b):
    return float(torch.linalg.vector_norm((a - b).flatten()) / torch.linalg.vector_norm(b.flatten()))


def main():
    w = workloads.workload('dirs16')
    lam = 2 * np.pi / w['kappa0']
    print("2a/lambda = %.1f, full expansion M = N = %d" % (2 * w['a'] / lam, w['nx'] - 1))
    ap0, fl0, it0, res0, sig0, t0 = run(w, 0)
    print("%-10s %10s %10s %10s %8s %9s" % ("modes", "aperture", "field", "RCS", "steps", "solve ms"))
    print("%-10s %10s %10s %10s %8d %9.1f" % ("all (255)", "-", "-", "-", int(it0.max()), 1e3 * t0))
    for K in (51, 55, 59, 67, 83, 127):
        ap, fl, it, res, sig, t = run(w, K)
        srel = float(np.max(np.abs(sig - sig0)) / np.max(sig0))
        print("%-10d %10.2e %10.2e %10.2e %8d %9.1f" % (K, rel(ap, ap0), rel(fl, fl0), srel,
                                                         int(it.max()), 1e3 * t))


if __name__ == "__main__":
    main()
