"""The serving loop on the GPU: requests for three contexts arrive together,
so later ones are answered by batches that mix several requests on one
context while the contexts' streams overlap.  Every request's aperture
solution and RCS equal those of the same request solved alone, within the
solver tolerance (mixed precision, tolerance 1e-10)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from paper_2008_01966_gb300.serving import GpuBackend, Request, Server

pytestmark = pytest.mark.gpu

KEYS = [
    ((1.0, 1.0, 0.5, 16, 16, 21), 2 * np.pi * 2, ((21, 1.0 + 0j),)),
    ((1.0, 1.0, 0.5, 16, 16, 23), 7.5, ((7, 4 + 1j), (9, 2 + 0.5j), (7, 1.0 + 0j))),
    ((1.0, 0.75, 0.4, 16, 8, 13), 9.0, ((13, 2.0 + 0.3j),)),
]


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01966_gb300 as gb
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return gb


def test_each_result_alone_and_in_the_mix(gb):
    reqs = []
    rid = 0
    for k, (geom, kappa0, layers) in enumerate(KEYS):
        for j in range(4):
            th, ph, al = workloads.directions(1 + (j % 3), 100 * k + j)
            reqs.append(Request(rid, 0.0, geom, kappa0, layers, th, ph, al, keep_aperture=True))
            rid += 1
    srv = Server(GpuBackend("mixed", tol=1e-10), budget_bytes=16 << 30, max_dirs=16)
    res = srv.run(reqs)
    assert all(res[r.rid].status == 0 for r in reqs)
    assert max(b[1] for b in srv.batches) > 1          # requests shared a batch
    assert len({b[0] for b in srv.batches}) == 3
    for r in reqs:
        (a, b, c, nx, ny, nz), kappa0, layers = r.key
        g = gb.Cavity(a, b, c, nx, ny, nz, precision="mixed", gmres_tol=1e-10)
        ap, _, _, _ = g.solve(kappa0, list(layers), r.theta, r.phi, r.alpha, field=False)
        sig = g.rcs(ap, r.theta, r.phi, "theta")
        got = res[r.rid].aperture.cpu().numpy()
        ref = ap.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref), r.rid
        assert np.all(np.abs(res[r.rid].rcs - sig) <= 1e-8 * np.abs(sig).max()), r.rid
        g.close()
