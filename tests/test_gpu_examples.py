"""The paper's example geometries (Sec. 7, Examples 1-3) as backscatter RCS
sweeps against the oracle.

The paper's RCS curves are figures that are not available, so these are
self-consistency cases: the GPU path (FP64, all 180 incidence angles of a
0.5-degree sweep solved as one batch of right-hand sides) against the oracle's
direct solve of the same discretisation, for both polarisations.  Grids are
coarse (16 points per wavelength horizontally) so the oracle finishes in
seconds; lengths in wavelengths (kappa0 = 2 pi).

  Example 1 (small): a = b = 1, c = 3, empty cavity
  Example 2:         a = 1, b = c = 0.25, eps_r = 7 + 1.5i, M = N = 15 as in
                     the paper's Table 3.  The periodised convolution of the
                     TBC integrals needs a period longer than side + sqrt(2) a
                     on each axis: 4 a along x1 but 8 b along the short side.
                     The FFT operator has period 4 on both axes, so this
                     geometry runs on the dense solver (the paper's own
                     direct solve), FP64 and mixed; the Krylov solver refuses
                     it at setup.  The fill is also run in a square aperture
                     a = b = 0.5 on the Krylov path
  Example 3:         a = b = 1, top layer eps_r = 7 + 1.5i of depth 1 over
                     eps_r = 3 + 0.05i of depth 2
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.aperture import ApertureSystem
from oracle.excitation import rhs as oracle_rhs
from oracle.geometry import Cavity as OCavity, Layer
from oracle.rcs import backscatter

pytestmark = pytest.mark.gpu

EXAMPLES = {
    "example1_small": dict(a=1.0, b=1.0, c=3.0, nx=16, ny=16, nz=48, layers=[(48, 1.0 + 0j)]),
    "example2": dict(a=1.0, b=0.25, c=0.25, nx=16, ny=16, nz=8, layers=[(8, 7 + 1.5j)], pad_y=8,
                     solver="dense"),
    "example2_fill": dict(a=0.5, b=0.5, c=0.25, nx=8, ny=8, nz=4, layers=[(4, 7 + 1.5j)]),
    "example3": dict(a=1.0, b=1.0, c=3.0, nx=16, ny=16, nz=48,
                     layers=[(16, 7 + 1.5j), (32, 3 + 0.05j)]),
}


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01966_gb300 as gb
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return gb


@pytest.mark.parametrize("name", list(EXAMPLES))
def test_example_rcs_sweep(gb, name):
    w = EXAMPLES[name]
    kappa0 = 2 * np.pi
    cav = OCavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], kappa0,
                  layers=[Layer(n, e) for n, e in w['layers']], pad_y=w.get('pad_y', 0))
    sysm = ApertureSystem(cav)
    theta = np.deg2rad(np.arange(0.0, 90.0, 0.5))
    phi = np.zeros_like(theta)
    g = gb.Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], precision="fp64",
                  gmres_tol=1e-12, aperture_solver=w.get('solver', "krylov"))
    assert (g.pad_x, g.pad_y) == (cav.pad, cav.pad_y)
    for pol, alpha in (("theta", 0.0), ("phi", np.pi / 2)):
        al = np.full_like(theta, alpha)
        B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(theta, phi, al)])
        X = sysm.solve_dense(B)
        ref = np.array([backscatter(cav, X[d], theta[d], phi[d], pol) for d in range(len(theta))])
        ap, _, it, res = g.solve(kappa0, w['layers'], theta, phi, al, field=False)
        assert np.all(res <= 1e-12)
        sig = g.rcs(ap, theta, phi, pol)
        # relative to the sweep's peak (the curves have deep nulls)
        assert np.abs(sig - ref).max() <= 1e-9 * ref.max(), (pol, np.abs(sig - ref).max() / ref.max())
        assert np.all(np.isfinite(sig)) and np.all(sig >= 0)


def test_example2_aperture_needs_the_dense_solver(gb):
    """The 4:1 aperture of Example 2 needs the period 8 b along its short
    side; the FFT operator (Krylov solver) has 4 a x 4 b and refuses it at
    setup with CAVITY_EINVAL, the dense solver takes it."""
    with pytest.raises(gb.CavityError) as e:
        gb.Cavity(1.0, 0.25, 0.25, 16, 16, 4)
    assert e.value.status == 1
    g = gb.Cavity(1.0, 0.25, 0.25, 16, 16, 4, aperture_solver="dense")
    assert (g.pad_x, g.pad_y) == (4, 8)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_example2_solve_and_field_against_oracle(gb, precision):
    """Example 2 (a = lambda, b = c = lambda/4, eps_r = 7 + 1.5i, M = N = 15)
    on the dense solver against the oracle's direct solve with the period 8 b:
    aperture and field per direction, 1e-10 (FP64) / 1e-8 and 1e-5 (mixed)."""
    from oracle.field import field as oracle_field
    import workloads
    w = EXAMPLES["example2"]
    kappa0 = 2 * np.pi
    cav = OCavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], kappa0,
                  layers=[Layer(n, e) for n, e in w['layers']], pad_y=8)
    sysm = ApertureSystem(cav)
    th, ph, al = workloads.directions(4, 41)
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X = sysm.solve_dense(B)
    fp64 = precision == "fp64"
    g = gb.Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], precision=precision,
                  gmres_tol=1e-12 if fp64 else 1e-10, aperture_solver="dense")
    ap, fl, it, res = g.solve(kappa0, w['layers'], th, ph, al)
    ap, fl = ap.cpu().numpy(), fl.cpu().numpy()
    for d in range(len(th)):
        assert np.linalg.norm(ap[d] - X[d]) <= (1e-10 if fp64 else 1e-8) * np.linalg.norm(X[d])
        F = oracle_field(cav, sysm.prof, X[d]).ravel()
        assert np.linalg.norm(fl[d] - F) <= (1e-10 if fp64 else 1e-5) * np.linalg.norm(F)
