"""Implementation options on the GPU (include/cavity.h, CAVITY_OPT_*): the
variants compute the same operator and the same solution, and the
autotuner picks and caches one.  A 512 x 512 grid with 16 levels (the
passes at 2048 points do not depend on the depth), four layers, mixed
precision."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

LAYERS = [(4, 4 + 1j), (4, 2 + 0.5j), (4, 6 + 0.1j), (4, 1 + 0j)]
KAPPA0 = 2 * np.pi / (10 * (0.5 / 256) * np.sqrt(6.0))


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01966_gb300 as gb
    assert torch.cuda.is_available()
    return gb


@pytest.fixture(scope="module")
def cav(gb):
    g = gb.Cavity(1.0, 1.0, 0.5, 512, 512, 16, precision="mixed", gmres_tol=1e-10)
    g.prepare(KAPPA0, LAYERS)
    return g


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_pass_variants_compute_the_same_operator(cav):
    rng = np.random.default_rng(5)
    x64 = torch.tensor(rng.standard_normal((4, cav.n_ap)) + 1j * rng.standard_normal((4, cav.n_ap)),
                       dtype=torch.complex128, device="cuda")
    ref = cav.apply(x64, "fp64")
    x = x64.to(torch.complex64)
    out = {}
    for b in (0, 1):
        for c in (0, 1):
            cav.set_option("pass_b_2048", b)
            cav.set_option("pass_c_2048", c)
            assert cav.get_option("pass_b_2048") == b and cav.get_option("pass_c_2048") == c
            out[b, c] = cav.apply(x, "mixed").to(torch.complex128)
            assert rel(out[b, c], ref) < 1e-6, (b, c)
    for k in out:
        assert rel(out[k], out[0, 0]) < 1e-6, k
    cav.set_option("pass_b_2048", 0)
    cav.set_option("pass_c_2048", 0)


def test_group_widths_give_the_same_solution(gb, cav):
    rng = np.random.default_rng(6)
    th, ph, al = rng.uniform(0, 1, 8), rng.uniform(0, 6, 8), np.zeros(8)
    sol = {}
    for gw in (16, 8, 4, 1):
        cav.set_option("group_width", gw)
        ap, _, it, res = cav.solve(KAPPA0, LAYERS, th, ph, al, field=False)
        assert np.all(res <= 1e-10), (gw, res)
        sol[gw] = ap.clone()
    for gw in sol:
        assert rel(sol[gw], sol[16]) < 1e-8, gw
    cav.set_option("group_width", 16)
    with pytest.raises(gb.CavityError):
        cav.set_option("group_width", 17)


def test_autotune_chooses_and_caches(gb, cav, tmp_path):
    from paper_2008_01966_gb300 import autotune
    rng = np.random.default_rng(7)
    th, ph, al = rng.uniform(0, 1, 8), rng.uniform(0, 6, 8), np.zeros(8)
    cache = str(tmp_path / "tune.json")
    out = autotune.tune(cav, KAPPA0, LAYERS, th, ph, al, cache=cache, reps=2)
    assert set(out["choice"]) == {"pass_b_2048", "pass_c_2048", "group_width", "field_fused"}
    for name, v in out["choice"].items():
        assert cav.get_option(name) == v
        assert min(out["ms"][name].values()) == out["ms"][name][str(v)]
    again = autotune.tune(cav, KAPPA0, LAYERS, th, ph, al, cache=cache, reps=2)
    assert again["cached"] and again["choice"] == out["choice"]
    for name in ("pass_b_2048", "pass_c_2048", "field_fused"):
        cav.set_option(name, 0)
    cav.set_option("group_width", 16)
    cav.prepare(KAPPA0, LAYERS)


def test_field_paths_agree(gb):
    """The complex64 field of a square grid from the fused kernel (option 1)
    and from the two-pass kernels (option 2) agree to FP32 rounding; the
    default takes the two-pass kernels below 512 points per side.  The option
    re-prepares the context (the FP32 profiles change layout)."""
    g = gb.Cavity(1.0, 1.0, 0.5, 128, 128, 16, precision="mixed", gmres_tol=1e-10)
    rng = np.random.default_rng(9)
    th, ph, al = rng.uniform(0, 1, 4), rng.uniform(0, 6, 4), np.zeros(4)
    fields = {}
    for o in (0, 1, 2):
        g.set_option("field_fused", o)
        assert g.get_option("field_fused") == o
        ap, fl, it, res = g.solve(KAPPA0, LAYERS, th, ph, al)
        assert np.all(np.asarray(res) <= 1e-10)
        fields[o] = fl.to(torch.complex128)
    assert rel(fields[1], fields[2]) < 1e-6
    assert rel(fields[0], fields[2]) < 1e-12
