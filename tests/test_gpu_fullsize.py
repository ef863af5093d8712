"""Whole solves at full size against the oracle, per result.

The homogeneous 256 x 256 x 128 workload (16 directions at 10 points per
wavelength) and the four-layer 512 x 512 x 256 workload (8 directions), the
two benchmark configurations: the oracle assembles the discretised system of
Sec. 3 / Sec. 4 with rule D for the TBC integrals of Sec. 5 and solves two
directions of each by GMRES to a relative residual of 1e-13 (its true
residual recomputed), then synthesises the field on every level by (E123F).
The GPU solves the whole batch, once on the FP64 path and once in mixed
precision, and each of the two directions is compared on its own:

  aperture vector E_{l,Nz}                       rel-L2  <= 1e-10 (FP64), 1e-5 (mixed)
  field of the direction (all levels together)   rel-L2  <= 1e-10 (FP64), 1e-5 (mixed)
  every single level                             rel-L2  <= 1e-9  (FP64), 1e-4 (mixed)
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle.aperture import ApertureSystem
from oracle.excitation import rhs as oracle_rhs
from oracle.field import field_level, synth_mats
from oracle.geometry import Cavity as OCavity, Layer

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
LEVEL_TOL = {"fp64": 1e-9, "mixed": 1e-4}
DIRS = (0, 1)


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01966_gb300 as gb
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return gb


def oracle_solutions(w):
    cav = OCavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], w['kappa0'],
                  layers=[Layer(n, e) for n, e in w['layers']])
    sysm = ApertureSystem(cav)
    B = np.array([oracle_rhs(cav, w['theta'][d], w['phi'][d], w['alpha'][d]) for d in DIRS])
    X, res = sysm.solve_gmres(B, rtol=1e-13, restart=300, maxiter=300)
    assert np.all(res < 1e-12), res
    return cav, sysm, X


def gpu_solve(gb, w, precision):
    g = gb.Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], precision=precision,
                  gmres_tol=1e-13 if precision == "fp64" else 1e-10)
    ap, fl, it, res = g.solve(w['kappa0'], w['layers'], w['theta'], w['phi'], w['alpha'])
    assert np.all(res <= (1e-12 if precision == "fp64" else 1e-10)), (precision, res)
    # keep the two compared directions only (on the host, as complex128)
    return {d: (ap[d].cpu().numpy(), fl[d].cpu()) for d in DIRS}


def compare(gb, w, cav, sysm, X):
    """Both precisions against the oracle, the oracle's field synthesised once
    per level."""
    got = {p: gpu_solve(gb, w, p) for p in ("fp64", "mixed")}
    torch.cuda.empty_cache()
    mats = synth_mats(cav)
    S = (cav.nx + 1) * (cav.ny - 1) + (cav.nx - 1) * (cav.ny + 1) + (cav.nx - 1) * (cav.ny - 1)
    report = []
    for k, d in enumerate(DIRS):
        x = X[k]
        num = {p: 0.0 for p in got}
        worst = {p: 0.0 for p in got}
        den = 0.0
        for j in range(1, cav.nz + 1):
            F = field_level(cav, sysm.prof, x, j, mats)
            n = np.vdot(F, F).real
            den += n
            for p in got:
                G = got[p][d][1][(j - 1) * S:j * S].numpy().astype(np.complex128)
                e = np.vdot(G - F, G - F).real
                num[p] += e
                worst[p] = max(worst[p], (e / n) ** 0.5)
        for p in got:
            e_ap = np.linalg.norm(got[p][d][0] - x) / np.linalg.norm(x)
            e_fl = (num[p] / den) ** 0.5
            report.append((p, d, e_ap, e_fl, worst[p]))
    for p, d, e_ap, e_fl, wl in report:
        print("%s dir %d: aperture %.2e field %.2e worst level %.2e" % (p, d, e_ap, e_fl, wl))
    for p, d, e_ap, e_fl, wl in report:
        assert e_ap <= TOL[p], (p, d, e_ap)
        assert e_fl <= TOL[p], (p, d, e_fl)
        assert wl <= LEVEL_TOL[p], (p, d, wl)


def test_dirs16_whole_solve_against_oracle(gb):
    w = workloads.workload('dirs16')
    compare(gb, w, *oracle_solutions(w))


def test_layered4_whole_solve_against_oracle(gb):
    w = workloads.workload('layered4')
    compare(gb, w, *oracle_solutions(w))
