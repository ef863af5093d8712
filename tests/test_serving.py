"""The serving loop's scheduling on the host, with a backend that needs no
GPU: continuous batching of requests that share a context, the split of a
batch's results back to its requests, admission by footprint with least
recently used eviction, rejection of unsupported grids and of contexts that
can never fit, and the seeded request stream."""

import threading
import time

import numpy as np

from paper_2008_01966_gb300.serving import Request, Server, summary, workload_requests


class FakeBackend:
    """solve() answers per direction with values that identify the direction
    and sleeps in proportion to the batch; tracks concurrently open handles."""

    def __init__(self, dt=0.02):
        self.dt = dt
        self.open_now = 0
        self.max_open = 0
        self.opened = []
        self.lock = threading.Lock()

    def open(self, key):
        with self.lock:
            self.open_now += 1
            self.max_open = max(self.max_open, self.open_now)
            self.opened.append(key)
        return {"key": key}

    def solve(self, handle, key, theta, phi, alpha, want_field, keep_aperture):
        time.sleep(self.dt * (1 + 0.1 * len(theta)))
        sig = 1000 * theta + phi
        return sig, np.full(len(theta), 7), np.full(len(theta), 1e-9), None, 10

    def close(self, handle):
        with self.lock:
            self.open_now -= 1


def req(rid, t, nx, nd, kappa0=5.0, seed=0):
    rng = np.random.Generator(np.random.PCG64(1000 + rid + seed))
    return Request(rid, t, (1.0, 1.0, 0.5, nx, nx, 8), kappa0, ((8, 1 + 0j),),
                   rng.uniform(0, 1, nd), rng.uniform(0, 6, nd), np.zeros(nd))


def foot(geom, ndir, precision, layered, want_field):
    return geom[3]  # one unit of "memory" per grid point along x


def test_batching_split_and_eviction():
    be = FakeBackend()
    srv = Server(be, budget_bytes=40, footprint=foot, max_dirs=16)
    reqs = [req(0, 0.0, 16, 3)]
    # while request 0 runs, four more arrive for the same key: one batch
    reqs += [req(i, 0.005 + 0.001 * i, 16, 2) for i in range(1, 5)]
    # two other keys of 16 "bytes" each: the budget (40) holds two contexts
    reqs += [req(5, 0.2, 16, 1, kappa0=6.0), req(6, 0.4, 16, 1, kappa0=7.0)]
    res = srv.run(reqs)
    assert len(res) == 7 and all(r.status == 0 for r in res.values())
    for r in reqs:
        out = res[r.rid]
        assert np.array_equal(out.rcs, 1000 * r.theta + r.phi)   # its own directions
        assert out.latency >= 0 and out.done >= out.start >= out.arrival - 1e-9
    sizes = sorted(b[1] for b in srv.batches)
    assert sizes[-1] == 4                                      # requests 1-4 batched
    assert srv.peak <= 40 and be.max_open <= 2                 # admission held
    assert len(be.opened) == 3                                 # third key evicted the first
    s = summary(res, 1.0)
    assert s["answered"] == 7 and s["latency_ms"]["p99"] >= s["latency_ms"]["p50"]


def test_rejections():
    be = FakeBackend()
    srv = Server(be, budget_bytes=100, footprint=lambda g, *a: 10 * g[3], max_dirs=8)
    reqs = [req(0, 0.0, 1024, 2), req(1, 0.0, 16, 2), req(2, 0.0, 8, 2)]
    res = srv.run(reqs)
    assert res[0].status == 1            # grid above the library's limit
    assert res[1].status == 2            # footprint 160 > budget 100
    assert res[2].status == 0


def test_request_stream_is_seeded_and_has_the_mix():
    a = workload_requests(200, 2.0, seed=5)
    b = workload_requests(200, 2.0, seed=5)
    assert [(r.arrival, r.geom, r.ndir) for r in a] == [(r.arrival, r.geom, r.ndir) for r in b]
    assert {r.geom[3] for r in a} == {128, 256, 512, 1024}
    assert all(1 <= r.ndir <= 32 for r in a)
    assert all(len(r.layers) == 4 and sum(l[0] for l in r.layers) == r.geom[5] for r in a)
    assert all(r.want_field == (r.geom[3] <= 256) for r in a)
    gaps = np.diff([r.arrival for r in a])
    assert abs(gaps.mean() - 0.5) < 0.1   # rate 2 per second
