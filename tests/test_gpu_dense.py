"""Dense direct solve of the aperture system on the kept modes (Algorithm I/II
Step 3; the truncated expansion of Sec. 7, Table 2), through the C ABI:

  * the FP32 LU with partial pivoting on seeded complex matrices -- sizes 1,
    one panel, a panel plus one, several panels with a ragged tail -- checked
    by what partial pivoting fixes: P A = L U to FP32 rounding, |L| <= 1, and
    the backward error of the solves; a zero pivot column is reported;
  * the kept block against the oracle's dense_kept, element by element
    (FP32: 2e-6 of the largest entry);
  * whole solves (FP64 refinement around the FP32 factors) against the
    oracle's dense solves of the same kept system, per direction:
    rel-L2 <= 1e-10 (FP64 path) and 1e-8 on the aperture vector for the
    mixed path (its residual target 1e-10), the field 1e-10 / 1e-5;
  * the dense and the Krylov solver on the same truncated system agree.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle.aperture import ApertureSystem
from oracle.excitation import rhs as oracle_rhs
from oracle.field import field as oracle_field
from oracle.geometry import Cavity as OCavity, Layer
from oracle.tbc import TBCOperator

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


CASES = {
    "homog": dict(a=1.0, b=1.0, c=0.5, nx=16, ny=16, nz=21, kappa0=2 * np.pi * 16 / 8,
                  layers=[(21, 1.0 + 0j)]),
    "rect": dict(a=1.0, b=0.75, c=0.4, nx=16, ny=8, nz=13, kappa0=9.0,
                 layers=[(13, 2.0 + 0.3j)]),
    "layer3": dict(a=1.0, b=1.0, c=0.5, nx=16, ny=16, nz=23, kappa0=7.5,
                   layers=[(7, 4 + 1j), (9, 2 + 0.5j), (7, 1.0 + 0j)]),
}


def ocav(w):
    return OCavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], w['kappa0'],
                   layers=[Layer(n, e) for n, e in w['layers']])


def gcav(gb, w, **kw):
    return gb.Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], **kw)


def unpack_lu(lu, ipiv):
    n = lu.shape[0]
    L = np.tril(lu, -1) + np.eye(n)
    U = np.triu(lu)
    perm = np.arange(n)
    for i, p in enumerate(ipiv):
        perm[[i, p]] = perm[[p, i]]
    return L, U, perm


@pytest.mark.parametrize("n", [1, 7, 64, 65, 200, 1031])
def test_lu_partial_pivoting(gb, n):
    """LU of a seeded complex matrix whose diagonal is zeroed (so that every
    step must exchange rows): P A = L U within FP32 rounding, every multiplier
    |l| <= 1 (the pivot is the column's largest entry), and solves of four
    right-hand sides with normwise backward error within a few sqrt(n) FP32
    units (the typical growth of partial pivoting)."""
    rng = np.random.default_rng(1000 + n)
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    if n > 1:
        np.fill_diagonal(A, 0)
    g = gcav(gb, CASES["homog"])
    a = torch.from_numpy(A.copy()).to(g.device)
    ipiv, info = g.lu_factor(a)
    assert info == -1
    lu = a.cpu().numpy().astype(np.complex128)
    piv = ipiv.cpu().numpy()
    assert np.all((piv >= np.arange(n)) & (piv < n))
    L, U, perm = unpack_lu(lu, piv)
    A64 = A.astype(np.complex128)
    err = np.abs(L @ U - A64[perm]).max() / np.abs(A64).max()
    assert err < 2e-6 * max(1.0, np.sqrt(n)), err
    assert np.abs(np.tril(lu, -1)).max(initial=0) <= 1 + 1e-6
    B = (rng.standard_normal((4, n)) + 1j * rng.standard_normal((4, n))).astype(np.complex64)
    b = torch.from_numpy(B.copy()).to(g.device)
    g.lu_solve(a, ipiv, b)
    X = b.cpu().numpy().astype(np.complex128)
    for r in range(4):
        res = np.linalg.norm(A64 @ X[r] - B[r]) / (np.linalg.norm(A64, 2) * np.linalg.norm(X[r]))
        assert res < 3e-7 * max(3.0, np.sqrt(n)), (r, res)


def test_lu_reports_a_zero_pivot_column(gb):
    """A matrix whose column 70 is zero: the factorisation completes, reports
    step 70 and returns ESINGULAR's info without raising."""
    rng = np.random.default_rng(7)
    n = 150
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    A[:, 70] = 0
    g = gcav(gb, CASES["homog"])
    a = torch.from_numpy(A).to(g.device)
    _, info = g.lu_factor(a)
    assert info == 70


def test_lu_solve_rejects_pivots_out_of_range(gb):
    """A pivot sequence with an entry outside 0..n-1 (here n and -1) is
    caught on the device before b is touched: CAVITY_EINVAL, b unchanged;
    the same call with the factor's own pivots then solves."""
    rng = np.random.default_rng(11)
    n = 96
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    g = gcav(gb, CASES["homog"])
    a = torch.from_numpy(A).to(g.device)
    ipiv, info = g.lu_factor(a)
    assert info == -1
    B = (rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))).astype(np.complex64)
    for bad in (n, -1):
        wrong = ipiv.clone()
        wrong[n // 2] = bad
        b = torch.from_numpy(B.copy()).to(g.device)
        with pytest.raises(gb.CavityError) as e:
            g.lu_solve(a, wrong, b)
        assert e.value.status == gb._lib.CAVITY_EINVAL
        assert torch.equal(b.cpu(), torch.from_numpy(B))
    b = torch.from_numpy(B.copy()).to(g.device)
    g.lu_solve(a, ipiv, b)
    X = b.cpu().numpy().astype(np.complex128)
    res = np.linalg.norm(A.astype(np.complex128) @ X.T - B.T) / np.linalg.norm(B)
    assert res < 1e-4, res


@pytest.mark.parametrize("case,mm,nn", [("homog", 5, 7), ("rect", 15, 7), ("layer3", 15, 15),
                                        ("layer3", 1, 1)])
def test_kept_block_matches_oracle(gb, case, mm, nn):
    """The assembled kept block (per-axis factor GEMMs, cavity part, row
    combination) against the oracle's dense_kept, entry by entry."""
    w = CASES[case]
    cav = ocav(w)
    ref = ApertureSystem(cav).dense_kept(mm, nn)
    g = gcav(gb, w, modes_m=mm if mm < w['nx'] - 1 else 0, modes_n=nn if nn < w['ny'] - 1 else 0)
    g.prepare(w['kappa0'], w['layers'])
    A = g.dense_assemble().cpu().numpy()
    assert A.shape == ref.shape
    err = np.abs(A - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case,mm,nn", [("layer3", 6, 9), ("rect", 0, 0), ("homog", 15, 4)])
def test_dense_solve_matches_oracle(gb, precision, case, mm, nn):
    """Whole dense solves (FP64 refinement around the FP32 factors) against
    the oracle's direct solve of the same kept system; the unknowns outside
    the kept set are exactly zero; a few refinement steps suffice."""
    w = CASES[case]
    cav = ocav(w)
    sysm = ApertureSystem(cav)
    mmo = mm or cav.M
    nno = nn or cav.N
    th, ph, al = workloads.directions(3, 31)
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X = sysm.solve_kept(B, mmo, nno)
    keep = sysm.kept_modes(mmo, nno)
    fp64 = precision == "fp64"
    g = gcav(gb, w, precision=precision, gmres_tol=1e-12 if fp64 else 1e-10,
             modes_m=mm if mm < cav.M else 0, modes_n=nn if nn < cav.N else 0,
             aperture_solver="dense")
    ap, fl, it, res = g.solve(w['kappa0'], w['layers'], th, ph, al)
    ap = ap.cpu().numpy()
    fl = fl.cpu().numpy()
    assert np.all(np.asarray(it) <= 6), it
    for d in range(3):
        assert np.all(ap[d][~keep] == 0)
        assert rel(ap[d], X[d]) < (1e-10 if fp64 else 1e-8)
        F = oracle_field(cav, sysm.prof, X[d]).ravel()
        assert rel(fl[d], F) < (1e-10 if fp64 else 1e-5)


def test_dense_and_krylov_agree_on_a_truncated_256_grid(gb):
    """The homogeneous 256 x 256 x 128 workload truncated to m, n <= 52 (about
    2a / lambda + 1 modes per axis, 8.2k kept unknowns): the dense and the
    Krylov solvers reach the same solution of the same system (FP64 path)."""
    w = workloads.workload("dirs16")
    nd = 4
    kw = dict(precision="fp64", gmres_tol=1e-12, modes_m=52, modes_n=52)
    sols = {}
    for solver in ("dense", "krylov"):
        g = gb.Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], aperture_solver=solver, **kw)
        ap, _, it, res = g.solve(w['kappa0'], w['layers'], w['theta'][:nd], w['phi'][:nd],
                                 w['alpha'][:nd], field=False)
        assert np.all(np.asarray(res) <= 1e-12), (solver, res)
        sols[solver] = ap.cpu().numpy()
        g.close()
    for d in range(nd):
        assert rel(sols["dense"][d], sols["krylov"][d]) < 1e-10


def test_two_level_preconditioner_same_solution_fewer_steps(gb):
    """The mixed solve's two-level preconditioner (coarse level: the exact
    solve of the modes m, n <= 24 by their LU factors) on a layered 128 x 128
    cavity: the same solution as the one-level preconditioner within the
    solver tolerance, in fewer block steps."""
    w = workloads.scaled("layered4", 128, nz=64, ndir=8)
    out = {}
    for mc in (0, 24):
        g = gb.Cavity(w['a'], w['b'], w['c'], w['nx'], w['ny'], w['nz'], precision="mixed",
                      gmres_tol=1e-10)
        g.set_option("coarse_modes", mc)
        assert g.get_option("coarse_modes") == mc
        ap, _, it, res = g.solve(w['kappa0'], w['layers'], w['theta'], w['phi'], w['alpha'],
                                 field=False)
        assert np.all(np.asarray(res) <= 1e-10), (mc, res)
        out[mc] = (ap.cpu().numpy(), np.asarray(it))
        g.close()
    for d in range(len(w['theta'])):
        assert rel(out[24][0][d], out[0][0][d]) < 1e-8
    assert out[24][1].max() < out[0][1].max(), (out[0][1], out[24][1])


@pytest.mark.parametrize("case,mm,nn", [("homog", 5, 7), ("rect", 15, 7), ("layer3", 15, 15)])
def test_parseval_kept_block_matches_oracle(gb, case, mm, nn):
    """The Parseval form of the TBC blocks (Sec. 5.2 with the outer integral
    taken exactly: Phi^H diag(F(G)) Phi) assembled on the GPU against the
    oracle's dense_kept under outer='parseval', entry by entry."""
    w = CASES[case]
    cav = ocav(w)
    ref = ApertureSystem(cav, tbc=TBCOperator(cav, outer='parseval')).dense_kept(mm, nn)
    g = gcav(gb, w, modes_m=mm if mm < w['nx'] - 1 else 0, modes_n=nn if nn < w['ny'] - 1 else 0,
             aperture_solver="dense", outer_rule="parseval")
    g.prepare(w['kappa0'], w['layers'])
    A = g.dense_assemble().cpu().numpy()
    err = np.abs(A - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case,mm,nn", [("layer3", 6, 9), ("rect", 0, 0)])
def test_parseval_dense_solve_matches_oracle(gb, precision, case, mm, nn):
    """Whole solves under the Parseval rule (dense solver: FP32 factors, FP64
    residuals from the FP64 kept block) against the oracle's direct solve of
    the same system, aperture and field per direction."""
    w = CASES[case]
    cav = ocav(w)
    sysm = ApertureSystem(cav, tbc=TBCOperator(cav, outer='parseval'))
    mmo, nno = mm or cav.M, nn or cav.N
    th, ph, al = workloads.directions(3, 37)
    B = np.array([oracle_rhs(cav, t, p, a) for t, p, a in zip(th, ph, al)])
    X = sysm.solve_kept(B, mmo, nno)
    fp64 = precision == "fp64"
    g = gcav(gb, w, precision=precision, gmres_tol=1e-12 if fp64 else 1e-10,
             modes_m=mm if mm < cav.M else 0, modes_n=nn if nn < cav.N else 0,
             aperture_solver="dense", outer_rule="parseval")
    ap, fl, it, res = g.solve(w['kappa0'], w['layers'], th, ph, al)
    ap = ap.cpu().numpy()
    fl = fl.cpu().numpy()
    assert np.all(np.asarray(it) <= 6), it
    for d in range(3):
        assert rel(ap[d], X[d]) < (1e-10 if fp64 else 1e-8)
        F = oracle_field(cav, sysm.prof, X[d]).ravel()
        assert rel(fl[d], F) < (1e-10 if fp64 else 1e-5)


def test_parseval_needs_the_dense_solver(gb):
    w = CASES["homog"]
    with pytest.raises(gb.CavityError):
        gcav(gb, w, outer_rule="parseval")
