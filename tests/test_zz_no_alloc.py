"""The allocation-free operator entry point, for callers that may not allocate
device memory in their solve loop (an application that owns a fixed device
budget and forbids library allocations, which would also synchronise the
device).  Checked here through the C ABI:

  * it gives the same y = A x as the ordinary entry point -- the same kernels
    on the same inputs, so to rounding -- on calls in a row with different
    inputs and with fewer directions after more (the fixed scratch keeps the
    previous call's contents, which must not leak into the next);
  * with a truncated mode set (the extra masking pass);
  * against the oracle's operator directly;
  * sizes beyond its fixed scratch are rejected.

Collected last on purpose; it also passes alone in a fresh process."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.aperture import ApertureSystem
from oracle.geometry import Cavity as OCavity, Layer

pytestmark = pytest.mark.gpu

GEO = dict(a=1.0, b=0.75, c=0.4, nx=16, ny=8, nz=13)
KAPPA0 = 9.0
LAYERS = [(7, 2.0 + 0.3j), (6, 1.0 + 0j)]
# FP64: the same FP64 kernels on both entry points.  Mixed: the FP32 operator
# (relative error 1e-7 .. 4e-7 against the FP64 operator) on both entry points.
SAME = {"fp64": 1e-14, "mixed": 1e-7}
ORACLE = {"fp64": 1e-12, "mixed": 1e-5}


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01966_gb300 as gb
    assert torch.cuda.is_available()
    return gb


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def draw(rng, ndir, n, scale, dt):
    x = rng.standard_normal((ndir, n)) + 1j * rng.standard_normal((ndir, n))
    return torch.tensor(x * scale, dtype=dt, device="cuda")


def context(gb, **kw):
    g = gb.Cavity(GEO['a'], GEO['b'], GEO['c'], GEO['nx'], GEO['ny'], GEO['nz'],
                  precision="fp64", **kw)
    g.prepare(KAPPA0, LAYERS)
    return g


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_apply_matches_apply_in_a_row(gb, precision):
    g = context(gb)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    rng = np.random.default_rng(17)
    # two calls of two directions, then one of a single direction
    for call, ndir in enumerate((2, 2, 1)):
        x = draw(rng, ndir, g.n_ap, 1 + 10 * call, dt)
        ref = g.apply(x, precision)
        got = g.apply_noalloc(x, precision)
        assert rel(got, ref) <= SAME[precision], (call, ndir)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_apply_truncated_modes(gb, precision):
    g = context(gb, modes_m=5, modes_n=3)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    rng = np.random.default_rng(23)
    for call, ndir in enumerate((2, 1)):
        x = draw(rng, ndir, g.n_ap, 1 + call, dt)
        ref = g.apply(x, precision)
        got = g.apply_noalloc(x, precision)
        assert rel(got, ref) <= SAME[precision], (call, ndir)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_apply_matches_the_oracle(gb, precision):
    g = context(gb)
    cav = OCavity(GEO['a'], GEO['b'], GEO['c'], GEO['nx'], GEO['ny'], GEO['nz'], KAPPA0,
                  layers=[Layer(n, e) for n, e in LAYERS])
    sysm = ApertureSystem(cav)
    rng = np.random.default_rng(29)
    x = rng.standard_normal((2, cav.n_ap)) + 1j * rng.standard_normal((2, cav.n_ap))
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    got = g.apply_noalloc(torch.tensor(x, dtype=dt, device="cuda"), precision)
    got = got.to(torch.complex128).cpu().numpy()
    for d in range(2):
        ref = sysm.apply(x[d])
        assert np.linalg.norm(got[d] - ref) / np.linalg.norm(ref) <= ORACLE[precision], d


def test_noalloc_rejects_sizes_beyond_its_scratch(gb):
    g = gb.Cavity(1.0, 1.0, 0.5, 64, 64, 8, precision="fp64")
    g.prepare(20.0, [(8, 1.0 + 0j)])
    x = torch.zeros((8, g.n_ap), dtype=torch.complex128, device="cuda")
    with pytest.raises(gb.CavityError) as e:
        g.apply_noalloc(x, "fp64")
    assert e.value.status == 1 and "scratch" in str(e.value)
