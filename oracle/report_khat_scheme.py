"""Error report of the paper's kernel-table scheme (Sec. 5.2 large-frequency
asymptotics, `khat_paper`) against the quadrature table (`khat`), and its
effect on the solved aperture coefficients, the interior field and the
backscatter RCS.  Oracle only (test infrastructure): run from the repository
root as  python -m oracle.report_khat_scheme
"""

import numpy as np

import workloads
from .aperture import ApertureSystem
from .excitation import rhs
from .field import field
from .geometry import Cavity, Layer
from .rcs import backscatter
from .tbc import TBCOperator


def report(name, w, ndir=3, dense=False):
    cav = Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], w['kappa0'],
                 layers=[Layer(n, e) for n, e in w['layers']])
    ref_t = TBCOperator(cav)
    pap_t = TBCOperator(cav, scheme='paper')
    K, Kp = ref_t.Kh, pap_t.Kh
    err = np.abs(Kp - K)
    rel = err / np.abs(K)
    # the ridge band: |2 pi rho - kappa0| R < 10
    jx, jy = ref_t.jx, ref_t.jy
    rho = np.hypot(jx[:, None] / ref_t.Lx, jy[None, :] / ref_t.Ly)
    band = np.abs(2 * np.pi * rho - cav.kappa0) * np.sqrt(2) * max(cav.a, cav.b) < 10
    th, ph, al = w['theta'][:ndir], w['phi'][:ndir], w['alpha'][:ndir]
    B = np.array([rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    s_ref = ApertureSystem(cav, tbc=ref_t)
    s_pap = ApertureSystem(cav, tbc=pap_t, prof=s_ref.prof)
    if dense:
        X, Xp = s_ref.solve_dense(B), s_pap.solve_dense(B)
    else:
        X, _ = s_ref.solve_gmres(B)
        Xp, _ = s_pap.solve_gmres(B)
    ea = max(np.linalg.norm(Xp[d] - X[d]) / np.linalg.norm(X[d]) for d in range(ndir))
    ef = max(np.linalg.norm(field(cav, s_ref.prof, Xp[d]) - field(cav, s_ref.prof, X[d])) /
             np.linalg.norm(field(cav, s_ref.prof, X[d])) for d in range(ndir))
    er = max(abs(backscatter(cav, Xp[d], th[d], ph[d]) / backscatter(cav, X[d], th[d], ph[d]) - 1)
             for d in range(ndir))
    print("%-10s table: max rel %.1e (off the ridge band %.1e, max abs / max|K| %.1e, "
          "max|K_paper| / max|K| %.1e); aperture %.1e, field %.1e, RCS %.1e (max over %d "
          "directions)" % (name, rel.max(), rel[~band].max() if np.any(~band) else 0.0,
                           err.max() / np.abs(K).max(), np.abs(Kp).max() / np.abs(K).max(),
                           ea, ef, er, ndir))


if __name__ == "__main__":
    report("small", workloads.workload("small"), ndir=1)
    report("dirs16@64", workloads.scaled("dirs16", 64, nz=32, ndir=3))
    report("layer4@64", workloads.scaled("layered4", 64, nz=32, ndir=3))
    th, ph, al = workloads.directions(2, 12)
    ridge = dict(a=1.0, b=1.0, c=0.5, nx=32, ny=32, nz=12, kappa0=2 * np.pi * 15.3,
                 layers=[(12, 1.0 + 0j)], theta=th, phi=ph, alpha=al)
    report("ridge@32", ridge, ndir=2, dense=True)
    import sys
    if "--full" in sys.argv:
        report("dirs16", workloads.scaled("dirs16", 256, nz=128, ndir=1), ndir=1)
