"""GPU parity: every row of the hot path, called through the C ABI, against
the CPU oracle on identical seeded inputs.

Tolerances (relative L2 over the compared array):
  FP64 path   1e-10   (the FP64 tolerance the solver is specified to)
  MIXED path  1e-5    (complex64 transforms and FP32 inner Krylov iterations)
Sizes span several FFT lines and thread blocks with ragged tails (Nz not a
power of two, M = Nx-1 odd, rectangular apertures, layered fills).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle.aperture import ApertureSystem
from oracle.excitation import rhs as oracle_rhs
from oracle.field import field as oracle_field
from oracle.geometry import Cavity as OCavity, Layer
from oracle.khat import khat as oracle_khat, khat_paper as oracle_khat_paper
from oracle.rcs import backscatter
from oracle.tbc import TBCOperator
from oracle.zsystem import Profiles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01966_gb300 as gb
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return gb


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def ocav(w, layers=None):
    lay = [Layer(n, e) for n, e in (layers or w['layers'])]
    return OCavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], w['kappa0'], layers=lay)


def gcav(gb, w, precision="fp64", **kw):
    return gb.Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], precision=precision, **kw)


CASES = {
    "homog": dict(a=1.0, b=1.0, c=0.5, nx=16, ny=16, nz=21, kappa0=2 * np.pi * 16 / 8,
                  layers=[(21, 1.0 + 0j)]),
    "rect": dict(a=1.0, b=0.75, c=0.4, nx=16, ny=8, nz=13, kappa0=9.0,
                 layers=[(13, 2.0 + 0.3j)]),
    "layer3": dict(a=1.0, b=1.0, c=0.5, nx=16, ny=16, nz=23, kappa0=7.5,
                   layers=[(7, 4 + 1j), (9, 2 + 0.5j), (7, 1.0 + 0j)]),
}


def oracle_profiles_flat(cav, prof):
    nz = cav.nz
    P = np.stack([np.concatenate([prof.P1[:, :, j].ravel(), prof.P2[:, :, j].ravel(),
                                  prof.P3[:, :, j].ravel()]) for j in range(1, nz)])
    Q = np.stack([np.concatenate([prof.Q1[:, :, j].ravel(), prof.Q2[:, :, j].ravel()])
                  for j in range(1, nz)])
    top = np.concatenate([prof.tau1.ravel(), prof.tau2.ravel(), prof.tau3.ravel(),
                          prof.vs1.ravel(), prof.vs2.ravel()])
    return P, Q, top


@pytest.mark.parametrize("case", list(CASES))
def test_zsweep_matches_banded_lu(gb, case):
    """a1: the GPU ratio sweep reproduces the oracle's pivoted banded LU: top
    relations tau, varsigma and all per-level profiles P, Q."""
    w = CASES[case]
    cav = ocav(w)
    prof = Profiles(cav)
    P, Q, top = oracle_profiles_flat(cav, prof)
    g = gcav(gb, w)
    g.prepare(w['kappa0'], w['layers'])
    gtop, gprof, gq = (t.cpu().numpy() for t in g.export_elimination())
    assert rel(gtop, top) < 1e-12
    assert rel(gprof, P) < 1e-12
    assert rel(gq, Q) < 1e-12 or np.abs(Q).max() == 0 and np.abs(gq).max() == 0


@pytest.mark.parametrize("case", ["homog", "rect"])
def test_kernel_table_matches_quadrature(gb, case):
    """a3: F(G) on the quarter frequency box vs the oracle's Gauss-Legendre
    quadrature with scipy's j0."""
    w = CASES[case]
    g = gcav(gb, w)
    g.prepare(w['kappa0'], w['layers'])
    kh = g.export_khat().cpu().numpy()
    Lx, Ly = 4 * w['a'], 4 * w['b']
    j1 = np.arange(2 * w['nx'])[:, None]
    j2 = np.arange(2 * w['ny'])[None, :]
    rho = np.sqrt((j1 / Lx) ** 2 + (j2 / Ly) ** 2)
    ref = oracle_khat(rho, w['kappa0'], np.sqrt(2) * max(w['a'], w['b']))
    assert np.abs(kh - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("nx,kappa0", [(64, 2 * np.pi * 6.4), (32, 2 * np.pi * 15.3)])
def test_kernel_table_paper_scheme(gb, nx, kappa0):
    """f1: the table by the paper's Sec. 5.2 scheme (khat_scheme="paper")
    against the oracle's restatement of the same scheme.  At 64 x 64 the box
    reaches c R = 400 with the ridge 2 pi rho = kappa0 in the quadrature range;
    at 32 x 32 with kappa0 = 30.6 pi the ridge lies in the asymptotic range."""
    w = dict(a=1.0, b=1.0, c=0.5, nx=nx, ny=nx, nz=8, layers=[(8, 1.0 + 0j)])
    g = gcav(gb, w, khat_scheme="paper")
    g.prepare(kappa0, w['layers'])
    kh = g.export_khat().cpu().numpy()
    j1 = np.arange(2 * nx)[:, None]
    j2 = np.arange(2 * nx)[None, :]
    rho = np.sqrt((j1 / 4.0) ** 2 + (j2 / 4.0) ** 2)
    ref = oracle_khat_paper(rho, kappa0, np.sqrt(2.0))
    # the scheme's integral to infinity, 1/sqrt(c^2 - kappa0^2), amplifies the
    # rounding of c by c^2/|c^2 - kappa0^2| next to the ridge
    c = 2 * np.pi * rho
    cond = 1.0 + c * c / np.abs(c * c - kappa0 ** 2)
    assert np.all(np.abs(kh - ref) <= 1e-12 * cond * np.abs(ref)), \
        (np.abs(kh - ref) / (cond * np.abs(ref))).max()


def test_solve_with_paper_scheme(gb):
    """f1: whole FP64 solve with the paper's table against the oracle's direct
    solve with the same table (64 x 64, ten points per wavelength: the
    asymptotic range starts beyond the ridge)."""
    w = dict(a=1.0, b=1.0, c=0.5, nx=64, ny=64, nz=12, kappa0=2 * np.pi * 6.4,
             layers=[(12, 1.0 + 0j)])
    cav = ocav(w)
    sysm = ApertureSystem(cav, tbc=TBCOperator(cav, scheme='paper'))
    th, ph, al = workloads.directions(2, 12)
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X, ores = sysm.solve_gmres(B)
    assert np.all(ores < 1e-12)
    g = gcav(gb, w, gmres_tol=1e-13, khat_scheme="paper")
    ap, fl, it, res = g.solve(w['kappa0'], w['layers'], th, ph, al, field=False)
    for d in range(2):
        assert rel(ap[d].cpu().numpy(), X[d]) < 1e-10


def test_rhs_matches_trapezoid_tests(gb):
    """a2: g1, g2 for several seeded directions."""
    w = CASES["rect"]
    cav = ocav(w)
    th, ph, al = workloads.directions(5, 11)
    al = np.array([0.0, 0.3, 1.2, np.pi / 2, 2.0])
    g = gcav(gb, w)
    g.prepare(w['kappa0'], w['layers'])
    got = g.rhs(th, ph, al).cpu().numpy()
    ref = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    assert rel(got, ref) < 1e-13


@pytest.mark.parametrize("case", list(CASES))
def test_operator_matches_fft_rule(gb, case):
    """a4 operator: y = A x of (EJ1)/(uT1) (cavity part plus the TBC integrals
    by the FFT rule of Sec. 5) in FP64 and in FP32."""
    w = CASES[case]
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, cav.n_ap)) + 1j * rng.standard_normal((3, cav.n_ap))
    ref = np.array([sysm.apply(v) for v in x])
    g = gcav(gb, w)
    g.prepare(w['kappa0'], w['layers'])
    y64 = g.apply(torch.tensor(x, dtype=torch.complex128, device="cuda"), "fp64").cpu().numpy()
    assert rel(y64, ref) < 1e-12
    y32 = g.apply(torch.tensor(x, dtype=torch.complex64, device="cuda"), "mixed").cpu().numpy()
    assert rel(y32, ref) < 1e-5


# grid sizes covering log2 nx and log2 ny = 2..10: every per-size instantiation
# of the transform passes (line lengths 8 .. 4096, warp and block transforms;
# at 4096 points 16 per thread, and pass B of the 16-byte types without its
# tables in shared memory)
SIZES = [(4, 256), (256, 4), (8, 512), (512, 8), (32, 64), (64, 32), (128, 128), (4, 1024),
         (1024, 4)]


@pytest.mark.parametrize("nx,ny", SIZES)
def test_operator_and_field_every_size(gb, nx, ny):
    """a4 operator and a5+a6 field synthesis at every supported line length,
    FP64 (1e-12) and FP32 (1e-5), against the oracle on random inputs."""
    w = dict(a=1.0, b=0.8, c=0.3, nx=nx, ny=ny, nz=5, kappa0=9.0,
             layers=[(2, 3.0 + 0.5j), (3, 1.0 + 0j)])
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    rng = np.random.default_rng(nx * 1000 + ny)
    x = rng.standard_normal((2, cav.n_ap)) + 1j * rng.standard_normal((2, cav.n_ap))
    ref = np.array([sysm.apply(v) for v in x])
    F = np.array([oracle_field(cav, sysm.prof, v).ravel() for v in x])
    for prec, tol in (("fp64", 1e-12), ("mixed", 1e-5)):
        g = gcav(gb, w, precision=prec)
        g.prepare(w['kappa0'], w['layers'])
        dt = torch.complex128 if prec == "fp64" else torch.complex64
        y = g.apply(torch.tensor(x, dtype=dt, device="cuda"), prec).cpu().numpy()
        assert rel(y, ref) < tol, (prec, rel(y, ref))
        fl = g.field(torch.tensor(x, dtype=torch.complex128, device="cuda")).cpu().numpy()
        assert rel(fl, F) < tol, (prec, rel(fl, F))
        if prec == "mixed":
            # the residual operator of the mixed solve: pair-of-FP32 arithmetic
            yp = g.apply(torch.tensor(x, device="cuda"), "pair32").cpu().numpy()
            assert rel(yp, ref) < 1e-11, rel(yp, ref)


@pytest.mark.parametrize("case", list(CASES))
def test_solve_fp64_matches_dense_oracle(gb, case):
    """Whole path in FP64: aperture coefficients and interior field within 1e-10
    of the oracle's direct solve."""
    w = CASES[case]
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    th, ph, al = workloads.directions(3, 7)
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X = sysm.solve_dense(B)
    g = gcav(gb, w, gmres_tol=1e-13)
    ap, fl, it, res = g.solve(w['kappa0'], w['layers'], th, ph, al, field=True)
    ap = ap.cpu().numpy()
    fl = fl.cpu().numpy()
    assert np.all(res < 1e-12) and np.all(it > 0)
    for d in range(3):
        assert rel(ap[d], X[d]) < 1e-10
        F = oracle_field(cav, sysm.prof, X[d]).ravel()
        assert rel(fl[d], F) < 1e-10


@pytest.mark.parametrize("case", ["homog", "layer3"])
def test_solve_mixed_matches_dense_oracle(gb, case):
    """Mixed path (FP32 transforms and inner iterations, FP64 refinement):
    within 1e-5 of the FP64 oracle per result."""
    w = CASES[case]
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    th, ph, al = workloads.directions(2, 9)
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X = sysm.solve_dense(B)
    g = gcav(gb, w, precision="mixed", gmres_tol=1e-10)
    ap, fl, it, res = g.solve(w['kappa0'], w['layers'], th, ph, al, field=True)
    assert fl.dtype == torch.complex64
    ap = ap.cpu().numpy()
    fl = fl.cpu().numpy()
    for d in range(2):
        assert rel(ap[d], X[d]) < 1e-8
        F = oracle_field(cav, sysm.prof, X[d]).ravel()
        assert rel(fl[d], F) < 1e-5


def test_small_workload_end_to_end(gb):
    """The 32x32x32 normal-incidence workload (kappa0 = 8 pi), FP64, with the
    exact selection rules of the symmetric problem checked on the GPU result."""
    w = workloads.workload('small')
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    X = sysm.solve_dense(oracle_rhs(cav, 0.0, 0.0, 0.0))
    g = gcav(gb, w, gmres_tol=1e-13)
    ap, fl, it, res = g.solve(w['kappa0'], w['layers'], w['theta'], w['phi'], w['alpha'])
    ap = ap.cpu().numpy()[0]
    assert rel(ap, X) < 1e-10
    F = oracle_field(cav, sysm.prof, X).ravel()
    assert rel(fl.cpu().numpy()[0], F) < 1e-10
    e1 = ap[:cav.n1].reshape(cav.M + 1, cav.N)
    m = np.arange(cav.M + 1)[:, None]
    n = np.arange(1, cav.N + 1)[None, :]
    assert np.abs(e1[(m % 2 == 1) | (n % 2 == 0)]).max() < 1e-12 * np.abs(ap).max()


def test_rcs_matches_far_field_formula(gb):
    w = CASES["rect"]
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    th, ph, al = workloads.directions(3, 4)
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X = sysm.solve_dense(B)
    g = gcav(gb, w)
    g.prepare(w['kappa0'], w['layers'])
    for pol in ("theta", "phi"):
        s = g.rcs(torch.tensor(X, device="cuda"), th, ph, pol)
        ref = np.array([backscatter(cav, X[d], th[d], ph[d], pol) for d in range(3)])
        assert rel(s, ref) < 1e-11
        s_host = g.rcs(torch.tensor(X), th, ph, pol)
        assert rel(s_host, ref) < 1e-11


def test_batch_isolation(gb):
    """A direction's result does not depend on the other directions of the
    batch (fixed-order reductions, per-direction Krylov bases)."""
    w = CASES["homog"]
    th, ph, al = workloads.directions(4, 21)
    g = gcav(gb, w, gmres_tol=1e-12)
    ap4, _, _, _ = g.solve(w['kappa0'], w['layers'], th, ph, al, field=False)
    ap4 = ap4.cpu().numpy()
    for d in (0, 3):
        ap1, _, _, _ = g.solve(w['kappa0'], w['layers'], th[d:d + 1], ph[d:d + 1], al[d:d + 1],
                               field=False)
        assert rel(ap1.cpu().numpy()[0], ap4[d]) < 1e-11


def test_host_buffers_match_device_buffers(gb):
    w = CASES["layer3"]
    th, ph, al = workloads.directions(2, 3)
    g = gcav(gb, w, precision="mixed", gmres_tol=1e-10)
    apd, fld, _, _ = g.solve(w['kappa0'], w['layers'], th, ph, al)
    aph, flh, _, _ = g.solve(w['kappa0'], w['layers'], th, ph, al, host=True)
    assert not aph.is_cuda and not flh.is_cuda
    assert rel(aph.numpy(), apd.cpu().numpy()) < 1e-14
    assert rel(flh.numpy(), fld.cpu().numpy()) < 1e-7


def test_minimal_grid_and_errors(gb):
    """Degenerate sizes: 4x4 aperture, two vertical steps; argument errors and
    the resonance status come back as codes, not crashes."""
    w = dict(a=1.0, b=1.0, c=0.3, nx=4, ny=4, nz=2, kappa0=3.0, layers=[(2, 1.0 + 0j)])
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    X = sysm.solve_dense(oracle_rhs(cav, 0.2, 0.4, 0.1))
    g = gcav(gb, w, gmres_tol=1e-13)
    ap, fl, it, res = g.solve(w['kappa0'], w['layers'], [0.2], [0.4], [0.1])
    assert rel(ap.cpu().numpy()[0], X) < 1e-10
    with pytest.raises(gb.CavityError) as e:
        gb.Cavity(1.0, 1.0, 0.5, 12, 16, 8)
    assert e.value.status == 1
    with pytest.raises(gb.CavityError) as e:
        g.prepare(3.0, [(1, 1.0), (1, 2.0)])
    assert e.value.status == 1
    g2 = gcav(gb, w, pivot_tol=1e9)
    with pytest.raises(gb.CavityError) as e:
        g2.prepare(3.0, w['layers'])
    assert e.value.status == 3


def test_mixed_block_solver_groups_duplicates_restarts(gb):
    """The mixed path's inner solves run block GMRES over groups of at most 16
    directions.  21 directions (groups of 11 and 10) with two repeated pairs,
    solved with the default block length and with restarts after every 2
    block steps: every aperture within 1e-8 of the oracle's dense solve, and
    the repeated directions give the same result."""
    w = CASES["layer3"]
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    th, ph, al = workloads.directions(19, 41)
    th = np.concatenate([th, th[[3, 11]]])
    ph = np.concatenate([ph, ph[[3, 11]]])
    al = np.concatenate([al, al[[3, 11]]])
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X = sysm.solve_dense(B)
    for restart in (40, 2):
        g = gcav(gb, w, precision="mixed", gmres_tol=1e-10, gmres_restart=restart,
                 gmres_max_iter=400)
        ap, _, it, res = g.solve(w['kappa0'], w['layers'], th, ph, al, field=False)
        assert np.all(res <= 1e-10), (restart, res.max())
        ap = ap.cpu().numpy()
        for d in range(len(th)):
            assert rel(ap[d], X[d]) < 1e-8, (restart, d)
        assert rel(ap[19], ap[3]) < 1e-9 and rel(ap[20], ap[11]) < 1e-9


def test_mixed_result_alone_and_in_the_mix(gb):
    """A direction solved alone and inside a batch (where it shares a Krylov
    block with the others) agrees within the solver tolerance."""
    w = CASES["homog"]
    th, ph, al = workloads.directions(6, 23)
    g = gcav(gb, w, precision="mixed", gmres_tol=1e-10)
    ap6, _, _, _ = g.solve(w['kappa0'], w['layers'], th, ph, al, field=False)
    ap6 = ap6.cpu().numpy()
    for d in (0, 5):
        ap1, _, _, _ = g.solve(w['kappa0'], w['layers'], th[d:d + 1], ph[d:d + 1], al[d:d + 1],
                               field=False)
        assert rel(ap1.cpu().numpy()[0], ap6[d]) < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_truncated_expansion_matches_oracle(gb, precision):
    """Aperture expansion truncated to m <= 6, n <= 9 (the paper's runs keep
    few modes, Sec. 7): aperture and field against the oracle's restricted
    dense solve, per result; the dropped unknowns are exactly zero."""
    w = CASES["layer3"]
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    th, ph, al = workloads.directions(3, 17)
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X = sysm.solve_truncated(B, 6, 9)
    keep = sysm.kept_modes(6, 9)
    fp64 = precision == "fp64"
    g = gcav(gb, w, precision=precision, gmres_tol=1e-12 if fp64 else 1e-10, modes_m=6, modes_n=9)
    ap, fl, it, res = g.solve(w['kappa0'], w['layers'], th, ph, al)
    ap = ap.cpu().numpy()
    fl = fl.cpu().numpy()
    for d in range(3):
        assert np.all(ap[d][~keep] == 0)
        assert rel(ap[d], X[d]) < (1e-10 if fp64 else 1e-8)
        F = oracle_field(cav, sysm.prof, X[d]).ravel()
        assert rel(fl[d], F) < (1e-10 if fp64 else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny", [(1024, 32), (32, 1024)])
def test_solve_on_1024_point_sides(gb, precision, nx, ny):
    """Whole solves with a 1024-point side (4096-point lines in the operator,
    2048-point lines in the field synthesis) against the oracle's GMRES solve
    (1e-12, true residual): aperture and field per direction, 1e-10 (FP64) and
    1e-5 (mixed)."""
    w = dict(a=1.0, b=1.0, c=0.25, nx=nx, ny=ny, nz=6, kappa0=2 * np.pi * 3.0,
             layers=[(3, 2.0 + 0.5j), (3, 1.0 + 0j)])
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    th, ph, al = workloads.directions(2, 53)
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X, res = sysm.solve_gmres(B, rtol=1e-13, restart=300, maxiter=300)
    assert np.all(res < 1e-12), res
    fp64 = precision == "fp64"
    g = gcav(gb, w, precision=precision, gmres_tol=1e-13 if fp64 else 1e-10)
    ap, fl, it, r = g.solve(w['kappa0'], w['layers'], th, ph, al)
    ap, fl = ap.cpu().numpy(), fl.cpu().numpy()
    for d in range(2):
        assert rel(ap[d], X[d]) < (1e-10 if fp64 else 1e-5)
        F = oracle_field(cav, sysm.prof, X[d]).ravel()
        assert rel(fl[d], F) < (1e-10 if fp64 else 1e-5)


def test_1024_square_layered_full_size(gb):
    """The largest serving grid, 1024 x 1024 x 512 with the four-layer fill at
    10 points per wavelength in the densest layer, 4 directions: the mixed and
    the FP64 paths reach their residuals and agree (1e-6 on the aperture,
    RCS to 1e-5), which the oracle cannot check at this size in a test's time;
    the 1024-point lines themselves are checked against the oracle above."""
    import workloads as wl
    w = wl.scaled("layered4", 1024, nz=512, ndir=4)
    sols = {}
    for prec in ("mixed", "fp64"):
        g = gcav(gb, w, precision=prec, gmres_tol=1e-10)
        ap, _, it, r = g.solve(w['kappa0'], w['layers'], w['theta'], w['phi'], w['alpha'],
                               field=False)
        assert np.all(np.asarray(r) <= 1e-10), (prec, r)
        sig = g.rcs(ap, w['theta'], w['phi'], "theta")
        sols[prec] = (ap.cpu().numpy(), np.asarray(sig))
        g.close()
        del ap
        torch.cuda.empty_cache()
    for d in range(4):
        assert rel(sols["mixed"][0][d], sols["fp64"][0][d]) < 1e-6
    assert np.all(np.abs(sols["mixed"][1] - sols["fp64"][1]) <= 1e-5 * np.abs(sols["fp64"][1]))
