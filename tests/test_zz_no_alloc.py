"""The allocation-free operator entry point (for callers that may not allocate
device memory in their solve loop) gives the same y = A x as the ordinary
entry point, on two calls in a row with different inputs (the fixed scratch
keeps the previous call's contents, which must not leak into the next), and
rejects sizes beyond its fixed scratch.  Collected last on purpose."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01966_gb300 as gb
    assert torch.cuda.is_available()
    return gb


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_noalloc_apply_matches_apply_twice(gb, precision, tol):
    g = gb.Cavity(1.0, 0.75, 0.4, 16, 8, 13, precision="fp64")
    g.prepare(9.0, [(7, 2.0 + 0.3j), (6, 1.0 + 0j)])
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    rng = np.random.default_rng(17)
    for call in range(2):
        x = rng.standard_normal((2, g.n_ap)) + 1j * rng.standard_normal((2, g.n_ap))
        x = torch.tensor(x * (1 + 10 * call), dtype=dt, device="cuda")
        ref = g.apply(x, precision)
        got = g.apply_noalloc(x, precision)
        assert rel(got, ref) < tol


def test_noalloc_rejects_sizes_beyond_its_scratch(gb):
    g = gb.Cavity(1.0, 1.0, 0.5, 64, 64, 8, precision="fp64")
    g.prepare(20.0, [(8, 1.0 + 0j)])
    x = torch.zeros((8, g.n_ap), dtype=torch.complex128, device="cuda")
    with pytest.raises(gb.CavityError) as e:
        g.apply_noalloc(x, "fp64")
    assert e.value.status == 1 and "scratch" in str(e.value)
