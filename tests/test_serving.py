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


def _run_bounded(srv, reqs, limit=20.0):
    """Server.run in a thread: a stalled scheduler fails the test instead of
    hanging it."""
    out = {}

    def go():
        out["res"] = srv.run(reqs)
    t = threading.Thread(target=go, daemon=True)
    t.start()
    t.join(limit)
    assert not t.is_alive(), "the scheduler stalled"
    return out["res"]


class TrackingBackend(FakeBackend):
    """Records the order in which contexts close and whether a context was
    closed while one of its solves was running."""

    def __init__(self, dt=0.02):
        super().__init__(dt)
        self.active = set()
        self.closed = []
        self.closed_while_busy = False

    def solve(self, handle, key, *args):
        with self.lock:
            self.active.add(id(handle))
        try:
            return super().solve(handle, key, *args)
        finally:
            with self.lock:
                self.active.discard(id(handle))

    def close(self, handle):
        with self.lock:
            if id(handle) in self.active:
                self.closed_while_busy = True
            self.closed.append(handle["key"])
        super().close(handle)


def test_batch_fills_max_dirs_exactly_and_oversized_requests_run_alone():
    """Requests queued behind a busy context are batched while their
    directions fit max_dirs, up to and including exactly max_dirs; a request
    larger than max_dirs is still served, as a batch of its own."""
    be = FakeBackend(dt=0.05)
    srv = Server(be, budget_bytes=100, footprint=foot, max_dirs=8)
    reqs = [req(0, 0.0, 16, 1)]
    reqs += [req(1, 0.010, 16, 4), req(2, 0.011, 16, 4), req(3, 0.012, 16, 4)]
    reqs += [req(4, 0.6, 16, 11)]
    res = _run_bounded(srv, reqs)
    assert all(r.status == 0 for r in res.values())
    assert [b[2] for b in srv.batches] == [1, 8, 4, 11]
    for r in reqs:
        assert res[r.rid].dof == 10 * r.ndir          # dof per direction x directions


def test_admission_at_the_budget_and_grid_at_the_size_limit():
    """A context whose footprint equals the budget is admitted, and a grid at
    exactly the largest supported side is served."""
    srv = Server(FakeBackend(dt=0.0), budget_bytes=16, footprint=foot, max_dirs=8, max_side=16)
    res = _run_bounded(srv, [req(0, 0.0, 16, 2)])
    assert res[0].status == 0


def test_least_recently_used_context_is_evicted_first():
    """Budget for two contexts: A and B are used in that order, then A again;
    a third key C must evict B (least recently used), not A."""
    be = TrackingBackend(dt=0.01)
    srv = Server(be, budget_bytes=32, footprint=foot, max_dirs=8)
    reqs = [req(0, 0.0, 16, 1, kappa0=5.0), req(1, 0.15, 16, 1, kappa0=6.0),
            req(2, 0.30, 16, 1, kappa0=5.0), req(3, 0.45, 16, 1, kappa0=7.0)]
    res = _run_bounded(srv, reqs)
    assert all(r.status == 0 for r in res.values())
    assert be.closed[0][1] == 6.0
    assert len(be.opened) == 3


def test_busy_context_is_never_evicted():
    """Budget for one context: a second key arriving while the first is
    solving waits for it instead of closing it under the running solve."""
    be = TrackingBackend(dt=0.3)
    srv = Server(be, budget_bytes=16, footprint=foot, max_dirs=8)
    res = _run_bounded(srv, [req(0, 0.0, 16, 1, kappa0=5.0), req(1, 0.05, 16, 1, kappa0=6.0)])
    assert all(r.status == 0 for r in res.values())
    assert not be.closed_while_busy
    assert res[1].start >= res[0].done - 1e-6


def test_rejections():
    be = FakeBackend()
    srv = Server(be, budget_bytes=100, footprint=lambda g, *a: 10 * g[3], max_dirs=8)
    reqs = [req(0, 0.0, 2048, 2), req(1, 0.0, 16, 2), req(2, 0.0, 8, 2)]
    res = srv.run(reqs)
    assert res[0].status == 1            # grid above the library's limit (1024)
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


class OomBackend(FakeBackend):
    """solve() of one key fails the way the library does when the device has
    no memory left for the batch (an exception carrying CAVITY_ENOMEM)."""

    class Err(RuntimeError):
        status = 2

    def solve(self, handle, key, theta, phi, alpha, want_field, keep_aperture):
        if key[1] == 6.0:
            raise OomBackend.Err("out of memory")
        return super().solve(handle, key, theta, phi, alpha, want_field, keep_aperture)


def test_out_of_memory_batch_is_answered_and_the_server_carries_on():
    be = OomBackend()
    srv = Server(be, budget_bytes=100, footprint=foot, max_dirs=16)
    reqs = [req(0, 0.0, 16, 2), req(1, 0.01, 16, 2, kappa0=6.0), req(2, 0.02, 16, 2, kappa0=6.0),
            req(3, 0.05, 16, 3)]
    res = srv.run(reqs)
    assert [res[i].status for i in range(4)] == [0, 2, 2, 0]
    assert srv.enomem >= 1
    assert np.allclose(res[3].rcs, 1000 * reqs[3].theta + reqs[3].phi)
