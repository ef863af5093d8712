"""Check the requests a serving run kept against the oracle (run by hand after
the run; the oracle is slow, so only a sample is kept):

    python -m paper_2008_01966_gb300.serving --requests 400 --catalogue 12 \
        --keep-every 50 --dump serving_sample.npz
    python tests/check_serving_sample.py serving_sample.npz

For every kept request, the first direction is solved by the oracle: it
assembles the discretised system of Sec. 3 / Sec. 4 with rule D for the TBC
integrals of Sec. 5 and solves it by GMRES to a relative residual of 1e-12,
recomputing the true residual.  The served aperture vector is compared with
it, relative L2 <= 1e-10 (FP64 path solved to a residual of 1e-12 or less)
or 1e-5 (mixed path, or either path at a looser solver tolerance, which the
serving loop's 1e-7 is), and so is the served backscatter RCS (relative, ten
times that).  Requests on grids above 512 points per side are listed but not
checked (the oracle would take hours).  Prints one line per request and
exits 1 if any of them is out of tolerance.
"""

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle.aperture import ApertureSystem  # noqa: E402
from oracle.excitation import rhs  # noqa: E402
from oracle.geometry import Cavity, Layer  # noqa: E402
from oracle.rcs import backscatter  # noqa: E402


# the oracle's kernel table and GMRES take hours beyond this side
MAX_SIDE = 512


def main(path):
    d = np.load(path)
    precision = str(d["precision"])
    solver_tol = float(d["tol"]) if "tol" in d else 1e-7
    tol = 1e-10 if (precision == "fp64" and solver_tol <= 1e-12) else 1e-5
    ok = True
    print("rid  grid            aperture_rel  rcs_rel   served_resid  oracle_s")
    for i in range(len(d["rid"])):
        a, b, c, nx, ny, nz = d["geom"][i]
        nx, ny, nz = int(nx), int(ny), int(nz)
        if max(nx, ny) > MAX_SIDE:
            print("%4d %4dx%-4dx%-4d skipped (the oracle would take hours)" % (d["rid"][i], nx, ny, nz))
            continue
        layers = [Layer(int(round(n.real)), complex(e)) for n, e in d["layers"][i]]
        t0 = time.perf_counter()
        cav = Cavity(a, b, c, nx, ny, nz, float(d["kappa0"][i]), layers=layers)
        sysm = ApertureSystem(cav)
        th, ph, al = float(d["theta"][i]), float(d["phi"][i]), float(d["alpha"][i])
        bvec = rhs(cav, th, ph, al)
        X, res = sysm.solve_gmres(bvec, rtol=1e-12, restart=300, maxiter=300)
        ref = X[0]
        sig = backscatter(cav, ref, th, ph, "theta")
        dt = time.perf_counter() - t0
        got = d["aperture_%d" % i]
        e_ap = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        e_rcs = abs(d["rcs"][i] - sig) / abs(sig)
        good = res[0] < 1e-11 and e_ap <= tol and e_rcs <= 10 * tol
        ok = ok and good
        print("%4d %4dx%-4dx%-4d %12.3e %9.2e %12.2e %9.1f %s" % (
            d["rid"][i], nx, ny, nz, e_ap, e_rcs, d["resid"][i], dt, "" if good else "FAIL"))
        sys.stdout.flush()
    return 0 if ok else 1


if __name__ == "__main__":
    if len(sys.argv) == 2:
        sys.exit(main(sys.argv[1]))
    print(__doc__)
    sys.exit(2)
