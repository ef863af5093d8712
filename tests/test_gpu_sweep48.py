"""The 48-cavity backscatter sweep (uneven sizes 64..512, homogeneous and
layered fills, four wavenumbers, 64 directions each) on a seeded subset, as in
the measurement plan: the first cavity of every size class, all four
wavenumbers and all 64 directions on the GPU (mixed precision, aperture and
RCS); against the oracle's GMRES solve at one wavenumber: 8 directions for
the 64 and 128 classes, 2 for the 256 and 512 classes (whose oracle setup
and solves take minutes), plus, for those two classes, the FP64 residual of
every direction and agreement with the FP64 path.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle.aperture import ApertureSystem
from oracle.excitation import rhs as oracle_rhs
from oracle.geometry import Cavity as OCavity, Layer
from oracle.rcs import backscatter

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01966_gb300 as gb
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return gb


def first_of_each_size():
    seen, out = set(), []
    for i, cv in enumerate(workloads.rcs_sweep48()):
        if cv['nx'] not in seen:
            seen.add(cv['nx'])
            out.append((i, cv))
    return sorted(out, key=lambda t: t[1]['nx'])


@pytest.mark.parametrize("index,cv", first_of_each_size(), ids=lambda v: str(v) if isinstance(v, int) else "")
def test_sweep48_subset(gb, index, cv):
    th, ph, al = cv['theta'], cv['phi'], cv['alpha']
    g = gb.Cavity(cv['a'], cv['b'], cv['c'], cv['nx'], cv['ny'], cv['nz'], precision="mixed",
                  gmres_tol=1e-8)
    sig = []
    for kappa0 in cv['kappas']:
        ap, _, it, res = g.solve(kappa0, cv['layers'], th, ph, al, field=False)
        assert np.all(res <= 1e-8) and np.all(it > 0)
        s = g.rcs(ap, th, ph, "theta")
        assert np.all(np.isfinite(s)) and np.all(s >= 0)
        sig.append((kappa0, ap, s))
    kappa0, ap, s = sig[1]
    cav = OCavity(cv['a'], cv['b'], cv['c'], cv['nx'], cv['ny'], cv['nz'], kappa0,
                  layers=[Layer(n, e) for n, e in cv['layers']])
    sysm = ApertureSystem(cav)
    sel = np.arange(0, 64, 8) if cv['nx'] <= 128 else np.array([0, 32])
    B = np.array([oracle_rhs(cav, th[d], ph[d], al[d]) for d in sel])
    X, ores = sysm.solve_gmres(B, rtol=1e-12, restart=300, maxiter=300)
    assert np.all(ores < 1e-11)
    ref = np.array([backscatter(cav, X[k], th[d], ph[d]) for k, d in enumerate(sel)])
    apn = ap.cpu().numpy()
    for k, d in enumerate(sel):
        assert np.linalg.norm(apn[d] - X[k]) <= 1e-6 * np.linalg.norm(X[k]), d
    assert np.all(np.abs(s[sel] - ref) <= 1e-5 * ref.max())
    if cv['nx'] > 128:
        g.prepare(kappa0, cv['layers'])
        b = g.rhs(th, ph, al)
        r = b - g.apply(ap, "fp64")
        rr = (torch.linalg.vector_norm(r, dim=1) / torch.linalg.vector_norm(b, dim=1)).cpu().numpy()
        assert np.all(rr <= 2e-8), rr.max()
        g64 = gb.Cavity(cv['a'], cv['b'], cv['c'], cv['nx'], cv['ny'], cv['nz'],
                        precision="fp64", gmres_tol=1e-10)
        ap64, _, _, _ = g64.solve(kappa0, cv['layers'], th[:4], ph[:4], al[:4], field=False)
        s64 = g64.rcs(ap64, th[:4], ph[:4], "theta")
        assert np.all(np.abs(s[:4] - s64) <= 1e-5 * s64.max())
