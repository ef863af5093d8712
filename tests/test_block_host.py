"""Host logic of the mixed solve's FP32 block GMRES, on the CPU: the FP64
routines of csrc/bgmres_host.h (Jacobi eigendecomposition, Cholesky QR and
SVQB orthonormalisation steps, Householder least squares of the block upper
Hessenberg system), built on their own with g++ through tests/block_host_shim.cpp
and checked against numpy's LAPACK routines and the identities each step
promises to the solver (T S = I, so W = (W T) S exactly; T^H G T = I for an
accepted Cholesky step; the least-squares residual equals the norm of the
residual it reports).
"""

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2008_01966_gb300", "csrc")
BG_MAX = 16

D = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("shim") / "libblockhost.so")
    # same host arithmetic flags as the library build (complex products
    # without the C99 infinity recovery)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-fcx-limited-range",
                    "-I", CSRC, os.path.join(ROOT, "tests", "block_host_shim.cpp"), "-o", out],
                   check=True)
    lib = ctypes.CDLL(out)
    lib.shim_herm_eig.argtypes = [D, ctypes.c_int, D, D]
    lib.shim_cholqr.argtypes = [D, ctypes.c_int, D, D, D]
    lib.shim_cholqr.restype = ctypes.c_int
    lib.shim_svqb.argtypes = [D, ctypes.c_int, D, D, D]
    lib.shim_svqb.restype = ctypes.c_double
    lib.shim_matmul_left.argtypes = [D, D, ctypes.c_int]
    lib.shim_blockls.argtypes = [ctypes.c_int, D, ctypes.c_int, D, D, D]
    return lib


def _p(a):
    return a.ctypes.data_as(D)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def herm_eig(lib, A):
    n = A.shape[0]
    A = _c(A)
    lam = np.zeros(n)
    U = np.zeros((n, n), np.complex128)
    lib.shim_herm_eig(_p(A), n, _p(lam), _p(U))
    return lam, U


def cholqr(lib, G):
    n = G.shape[0]
    G = _c(G)
    T = np.zeros((n, BG_MAX), np.complex128)
    S = np.zeros((n, n), np.complex128)
    cond = np.zeros(1)
    ok = lib.shim_cholqr(_p(G), n, _p(T), _p(S), _p(cond))
    return bool(ok), T[:, :n], S, cond[0]


def svqb(lib, G):
    n = G.shape[0]
    G = _c(G)
    T = np.zeros((n, BG_MAX), np.complex128)
    S = np.zeros((n, n), np.complex128)
    ratio = np.zeros(1)
    dev = lib.shim_svqb(_p(G), n, _p(T), _p(S), _p(ratio))
    return dev, T, S, ratio[0]


@pytest.mark.parametrize("n", [1, 2, 5, 16])
def test_herm_eig_matches_lapack(shim, n):
    rng = np.random.default_rng(100 + n)
    X = rand_c(rng, n, n)
    A = X + X.conj().T
    lam, U = herm_eig(shim, A)
    assert np.allclose(np.sort(lam), np.linalg.eigvalsh(A), rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.allclose(U.conj().T @ U, np.eye(n), atol=1e-13)
    assert np.allclose(U @ np.diag(lam) @ U.conj().T, A, atol=1e-12 * np.abs(A).max())


def test_herm_eig_repeated_and_zero(shim):
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rand_c(rng, 6, 6))
    want = np.array([3.0, 3.0, 3.0, -1.0, 0.0, 0.0])
    A = Q @ np.diag(want) @ Q.conj().T
    lam, U = herm_eig(shim, A)
    assert np.allclose(np.sort(lam), np.sort(want), atol=1e-12)
    assert np.allclose(U @ np.diag(lam) @ U.conj().T, A, atol=1e-12)
    lam0, U0 = herm_eig(shim, np.zeros((4, 4)))
    assert np.all(lam0 == 0) and np.allclose(U0, np.eye(4))


@pytest.mark.parametrize("n", [1, 3, 16])
def test_cholqr_orthonormalises_a_block(shim, n):
    rng = np.random.default_rng(200 + n)
    W = rand_c(rng, 300, n)
    G = W.conj().T @ W
    ok, T, S, cond = cholqr(shim, G)
    assert ok
    # S = L^H with G = L L^H: upper triangular, positive real diagonal
    assert np.allclose(np.tril(S, -1), 0) and np.all(np.diag(S).real > 0)
    assert np.allclose(np.diag(S).imag, 0)
    assert np.allclose(S.conj().T @ S, G, rtol=0, atol=1e-12 * np.abs(G).max())
    assert np.allclose(S, np.linalg.cholesky(G).conj().T, atol=1e-10 * np.sqrt(np.abs(G).max()))
    assert np.allclose(T @ S, np.eye(n), atol=1e-12)           # W = (W T) S
    assert np.allclose(T.conj().T @ G @ T, np.eye(n), atol=1e-12)  # W T orthonormal
    assert cond >= np.linalg.cond(G) * (1 - 1e-12)           # an upper bound


def _rotated(rng, lam):
    """U diag(lam) U^H with a random unitary U."""
    n = len(lam)
    Q, _ = np.linalg.qr(rand_c(rng, n, n))
    return Q @ np.diag(lam) @ Q.conj().T


def test_cholqr_condition_bound_on_ill_conditioned_blocks(shim):
    """The acceptance test of the solver (Cholesky QR kept without a second
    pass when the bound is at most 1e3) needs a true upper bound where it
    matters: on blocks of condition 2e3 and 5e5 the bound must exceed
    cond_2(G), so such blocks are not accepted."""
    rng = np.random.default_rng(31)
    for lam in ([1.0, 0.3, 5e-4], [2.0, 1.0, 0.5, 0.1, 4e-6]):
        G = _rotated(rng, np.array(lam))
        G = 0.5 * (G + G.conj().T)
        ok, T, S, cond = cholqr(shim, G)
        assert ok
        c2 = np.linalg.cond(G)
        assert cond >= c2 * (1 - 1e-9) and cond > 1e3
        assert np.allclose(T @ S, np.eye(len(lam)), atol=1e-9)


def test_cholqr_refuses_dependent_blocks(shim):
    rng = np.random.default_rng(9)
    W = rand_c(rng, 100, 4)
    W[:, 3] = W[:, 1]                                         # a repeated direction
    ok, _, _, _ = cholqr(shim, W.conj().T @ W)
    assert not ok
    W = rand_c(rng, 100, 3)
    W[:, 2] = W[:, 0] + 1e-7 * rand_c(rng, 100)               # pivot ~1e-14 of the largest
    ok, _, _, _ = cholqr(shim, W.conj().T @ W)
    assert not ok
    ok, _, _, _ = cholqr(shim, np.zeros((2, 2)))
    assert not ok


def test_svqb_dependent_block(shim):
    rng = np.random.default_rng(11)
    W = rand_c(rng, 200, 5)
    W[:, 4] = 2.0 * W[:, 0]
    G = W.conj().T @ W
    dev, T, S, ratio = svqb(shim, G)
    n = 5
    assert dev == pytest.approx(np.abs(G - np.eye(n)).max(), rel=1e-15)
    lam = np.linalg.eigvalsh(G)
    assert ratio == pytest.approx(lam.min() / lam.max(), abs=1e-14)
    assert np.all(T[:, n:] == 0)
    T = T[:, :n]
    assert np.allclose(T @ S, np.eye(n), atol=1e-8)           # W = (W T) S holds exactly
    assert np.allclose((W @ T) @ S, W, atol=1e-8 * np.abs(W).max())
    # the new block: orthonormal on the range; the null direction is scaled by
    # the floor (1e-12 of the largest eigenvalue), so what is left of it is
    # the rounding of U^H G U there (~1e-16 of the largest) over the floor
    ev = np.linalg.eigvalsh(T.conj().T @ G @ T)
    assert np.allclose(ev[1:], 1.0, atol=1e-10) and abs(ev[0]) < 1e-3


def test_svqb_well_conditioned_and_vanished(shim):
    rng = np.random.default_rng(12)
    W = rand_c(rng, 200, 4)
    G = W.conj().T @ W
    dev, T, S, ratio = svqb(shim, G)
    T = T[:, :4]
    assert np.allclose(T.conj().T @ G @ T, np.eye(4), atol=1e-12)
    assert np.allclose(T @ S, np.eye(4), atol=1e-12)
    # exact breakdown: a zero block stays zero, nothing divides by zero
    dev, T, S, ratio = svqb(shim, np.zeros((3, 3)))
    assert dev == 1.0 and ratio == 0.0 and np.all(T == 0) and np.all(S == 0)


def test_svqb_orthonormalises_a_widely_spread_block(shim):
    """Eigenvalues spread over nine decades (above Cholesky QR's pivot
    threshold) are all above SVQB's floor of 1e-12 of the largest: the new
    block must come out orthonormal in every direction, not just the large
    ones."""
    rng = np.random.default_rng(32)
    lam = np.array([1.0, 1e-3, 1e-6, 1e-9])
    G = _rotated(rng, lam)
    G = 0.5 * (G + G.conj().T)
    dev, T, S, ratio = svqb(shim, G)
    T = T[:, :4]
    assert ratio == pytest.approx(1e-9, rel=1e-5)
    ev = np.linalg.eigvalsh(T.conj().T @ G @ T)
    assert np.allclose(ev, 1.0, atol=1e-5), ev
    assert np.allclose(T @ S, np.eye(4), atol=1e-6)


def test_matmul_left(shim):
    rng = np.random.default_rng(13)
    S2, S = _c(rand_c(rng, 6, 6)), _c(rand_c(rng, 6, 6))
    want = S2 @ S
    shim.shim_matmul_left(_p(S2), _p(S), 6)
    assert np.allclose(S, want, atol=1e-13)


@pytest.mark.parametrize("r,nblk", [(1, 1), (1, 12), (3, 5), (16, 4)])
def test_block_least_squares_matches_lstsq(shim, r, nblk):
    rng = np.random.default_rng(300 + 10 * r + nblk)
    m, k = (nblk + 1) * r, nblk * r
    H = rand_c(rng, m, k)
    for c in range(nblk):                                     # block upper Hessenberg
        H[(c + 2) * r:, c * r:(c + 1) * r] = 0
    S0 = np.triu(rand_c(rng, r, r))
    E = np.zeros((m, r), np.complex128)
    E[:r] = S0
    Y = np.zeros((k, r), np.complex128)
    res = np.zeros(nblk * r)
    H, S0 = _c(H), _c(S0)
    shim.shim_blockls(r, _p(S0), nblk, _p(H), _p(Y), _p(res))
    Yref = np.linalg.lstsq(H, E, rcond=None)[0]
    assert np.allclose(Y, Yref, atol=1e-9 * np.abs(Yref).max())
    # reported residuals after every block column against the truncated problems
    for c in range(nblk):
        mm, kk = (c + 2) * r, (c + 1) * r
        Hc = H[:mm, :kk]
        Yc = np.linalg.lstsq(Hc, E[:mm], rcond=None)[0]
        want = np.linalg.norm(E[:mm] - Hc @ Yc, axis=0)
        assert np.allclose(res[c * r:(c + 1) * r], want, rtol=1e-9, atol=1e-12)
    assert np.allclose(res[-r:], np.linalg.norm(E - H @ Y, axis=0), rtol=1e-9, atol=1e-12)


def test_block_least_squares_exact_breakdown(shim):
    """The new block vanished (SVQB returned a zero block): the subdiagonal
    block of the last block column is zero, the right-hand sides lie in the
    Krylov space, and the least-squares residual drops to zero (up to
    rounding) with Y solving the square system."""
    rng = np.random.default_rng(21)
    r, nblk = 2, 3
    m, k = (nblk + 1) * r, nblk * r
    H = rand_c(rng, m, k)
    for c in range(nblk):
        H[(c + 2) * r:, c * r:(c + 1) * r] = 0
    H[nblk * r:, :] = 0                                       # S of the last block = 0
    S0 = np.triu(rand_c(rng, r, r))
    E = np.zeros((m, r), np.complex128)
    E[:r] = S0
    Y = np.zeros((k, r), np.complex128)
    res = np.zeros(nblk * r)
    H, S0 = _c(H), _c(S0)
    shim.shim_blockls(r, _p(S0), nblk, _p(H), _p(Y), _p(res))
    assert np.all(res[:-r] > 1e-3)                            # not solved before the last block
    assert np.all(res[-r:] <= 1e-12 * np.abs(S0).max())
    Ysq = np.linalg.solve(H[:k], E[:k])
    assert np.allclose(Y, Ysq, atol=1e-10 * np.abs(Ysq).max())


def test_block_least_squares_zero_column_stays_finite(shim):
    """A column that is zero in full (not reachable with a nonsingular
    operator) gives a zero diagonal entry of R: the solve sets that
    coefficient to zero instead of dividing by it."""
    rng = np.random.default_rng(22)
    r, nblk = 2, 3
    m, k = (nblk + 1) * r, nblk * r
    H = rand_c(rng, m, k)
    for c in range(nblk):
        H[(c + 2) * r:, c * r:(c + 1) * r] = 0
    H[:, 2 * r + 1] = 0
    S0 = np.triu(rand_c(rng, r, r))
    E = np.zeros((m, r), np.complex128)
    E[:r] = S0
    Y = np.zeros((k, r), np.complex128)
    res = np.zeros(nblk * r)
    H, S0 = _c(H), _c(S0)
    shim.shim_blockls(r, _p(S0), nblk, _p(H), _p(Y), _p(res))
    assert np.all(np.isfinite(Y)) and np.all(np.isfinite(res)) and np.all(Y[2 * r + 1] == 0)
    Yref = np.linalg.lstsq(np.delete(H, 2 * r + 1, axis=1), E, rcond=None)[0]
    assert np.allclose(np.delete(Y, 2 * r + 1, axis=0), Yref, atol=1e-9 * np.abs(Yref).max())
