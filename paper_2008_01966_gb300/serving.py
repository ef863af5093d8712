"""Serving loop: cavity solve requests arriving over time, answered by
continuous batching on device-resident contexts.

A request names a cavity (a, b, c and its grid), a wavenumber kappa0, a layered
fill eps(z) and 1..32 incident directions; it asks for the aperture solution
and the backscatter RCS (optionally the interior field).  Requests that share
(cavity, kappa0, eps) share a context: its per-mode elimination, kernel table
and preconditioner are computed once (cavity_prepare) and stay resident, and
all requests queued for it while it is busy are solved together as one batch
of right-hand sides when it becomes free (continuous batching: a request that
arrives while its context is on the GPU joins the next batch, not a queue of
single solves).  Each context has its own CUDA stream and worker thread, so
batches of different contexts overlap on the device.  Contexts are admitted by
their HBM footprint (an upper estimate from the data layout) against a budget;
idle contexts are evicted least recently used first.  Per request the loop
records arrival, start and completion times; p50/p99 latency and DOF/s
(field degrees of freedom Nz * n_ap per direction) summarise a run.

    python -m paper_2008_01966_gb300.serving --requests 100 --precision mixed

runs a seeded Poisson stream with the mix of the serving workload (grids
128^2 x 64, 256^2 x 128, 512^2 x 256 and 1024^2 x 512; four-layer fills;
1-32 directions; field kept for grids up to 256^2).
"""

import argparse
import collections
import json
import math
import threading
import time
from dataclasses import dataclass

import numpy as np

LAYER_EPS = (4 + 1j, 2 + 0.5j, 6 + 0.1j, 1 + 0j)
GRIDS = ((128, 64), (256, 128), (512, 256), (1024, 512))
MAX_SIDE = 1024


@dataclass
class Request:
    rid: int
    arrival: float                  # seconds after the start of the run
    geom: tuple                     # (a, b, c, nx, ny, nz)
    kappa0: float
    layers: tuple                   # ((levels, eps), ...) top to bottom
    theta: np.ndarray
    phi: np.ndarray
    alpha: np.ndarray
    want_field: bool = False
    keep_aperture: bool = False

    @property
    def key(self):
        return (self.geom, float(self.kappa0), tuple(self.layers))

    @property
    def ndir(self):
        return len(self.theta)


@dataclass
class Result:
    rid: int
    status: int
    arrival: float
    start: float = math.nan
    done: float = math.nan
    batch: int = 0                  # requests in the batch that answered it
    rcs: np.ndarray = None
    iters: np.ndarray = None
    resid: np.ndarray = None
    aperture: object = None         # host tensor when keep_aperture
    dof: int = 0

    @property
    def latency(self):
        return self.done - self.arrival


def workload_requests(n, rate, seed=5, a=1.0, c=0.5, catalogue=0, keep_every=0):
    """Seeded Poisson stream with the serving workload's mix: grid drawn from
    GRIDS, four equal layers with a seeded permutation of LAYER_EPS, kappa0 at
    10 points per wavelength in the densest layer, 1-32 directions (theta in
    [0, pi/3], phi in [0, 2 pi), theta polarisation), field for grids up to
    256^2.  catalogue > 0: the cavities (grid and fill) are drawn once, that
    many, and every request names one of them (clients asking about the same
    cavities again, so contexts are reused and requests batch); 0: a fresh
    draw per request.  keep_every > 0: every keep_every-th request keeps its
    aperture solution (for checks against a reference)."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def cavity():
        nx, nz = GRIDS[rng.integers(len(GRIDS))]
        eps = [LAYER_EPS[i] for i in rng.permutation(len(LAYER_EPS))]
        return nx, nz, eps

    cat = [cavity() for _ in range(catalogue)]
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate)
        nx, nz, eps = cat[rng.integers(len(cat))] if cat else cavity()
        layers = tuple((nz // 4, e) for e in eps)
        h = c / nz
        nmax = max(np.sqrt(e).real for e in eps)
        kappa0 = 2 * np.pi / (10 * h * nmax)
        nd = int(rng.integers(1, 33))
        th = rng.uniform(0.0, np.pi / 3, nd)
        ph = rng.uniform(0.0, 2 * np.pi, nd)
        out.append(Request(rid, t, (a, a, c, nx, nx, nz), kappa0, layers, th, ph, np.zeros(nd),
                           want_field=nx <= 256,
                           keep_aperture=keep_every > 0 and rid % keep_every == 0))
    return out


def footprint_bytes(geom, ndir, precision, layered, want_field):
    """Upper estimate of a context's device memory for batches of up to ndir
    directions, from the library's data layout: profiles (FP64 and FP32
    copies, E3-driven ones when layered), kernel tables, operator scratch,
    Krylov bases and vectors, the pair-of-FP32 residual work, the field
    intermediate and output."""
    a, b, c, nx, ny, nz = geom
    M, N = nx - 1, ny - 1
    nap = 3 * M * N + M + N
    n12 = (M + 1) * N + M * (N + 1)
    Px, Py = 4 * nx, 4 * ny
    mixed = precision == "mixed"
    by = (nz - 1) * nap * (16 + (8 if mixed else 0))
    if layered:
        by += (nz - 1) * n12 * (16 + (8 if mixed else 0))
    by += (Px // 2) * (Py // 2) * 48 + 64 * nap
    el = 8 if mixed else 16
    scratch = 2 * ndir * 3 * (nx + 1) * Py * el
    by += scratch
    vec = ndir * nap
    if mixed:
        groups = -(-ndir // 16)
        by += groups * 31 * 16 * nap * 8 + 4 * vec * 8 + 6 * vec * 16 + 2 * scratch
        by += 608 * 31 * 16 * 16 * 16
    else:
        by += vec * 41 * 16 + 4 * vec * 16
    if want_field:
        fpd = (nx + 1) * (ny - 1) + (nx - 1) * (ny + 1) + (nx - 1) * (ny - 1)
        by += ndir * fpd * nz * el + (512 << 20)
    return int(by * 1.1) + (64 << 20)


class GpuBackend:
    """Contexts on the GPU through the library (one CUDA stream each)."""

    def __init__(self, precision="mixed", tol=1e-7):
        import torch
        import paper_2008_01966_gb300 as gb
        self.torch, self.gb = torch, gb
        self.precision, self.tol = precision, tol

    def open(self, key):
        torch, gb = self.torch, self.gb
        (a, b, c, nx, ny, nz), kappa0, layers = key
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            cav = gb.Cavity(a, b, c, nx, ny, nz, precision=self.precision, gmres_tol=self.tol,
                            stream=stream)
            cav.prepare(kappa0, list(layers))
        stream.synchronize()
        return (cav, stream)

    def solve(self, handle, key, theta, phi, alpha, want_field, keep_aperture):
        torch = self.torch
        cav, stream = handle
        _, kappa0, layers = key
        with torch.cuda.stream(stream):
            ap, fl, it, res = cav.solve(kappa0, list(layers), theta, phi, alpha, field=want_field)
            sig = cav.rcs(ap, theta, phi, "theta")
        stream.synchronize()
        out = (sig, it, res, (ap.cpu() if keep_aperture else None), cav.nz * cav.n_ap)
        if want_field:
            # the field (up to tens of GB per batch) goes back to the caching
            # allocator; hand it to the device so that the library's own
            # allocations, which the admission budget counts, find it
            del fl, ap
            torch.cuda.empty_cache()
        return out

    def close(self, handle):
        cav, stream = handle
        stream.synchronize()
        cav.close()


class _Ctx:
    def __init__(self, key, nbytes):
        self.key = key
        self.nbytes = nbytes
        self.handle = None
        self.busy = False
        self.last_used = 0.0
        self.closing = False


class Server:
    """Admission, continuous batching and eviction over a backend.

    backend: open(key) -> handle; solve(handle, key, theta, phi, alpha,
    want_field, keep_aperture) -> (rcs, iters, resid, aperture, dof per
    direction); close(handle).
    """

    def __init__(self, backend, budget_bytes, precision="mixed", max_dirs=64,
                 footprint=footprint_bytes, max_side=MAX_SIDE, clock=time.perf_counter):
        self.backend = backend
        self.budget = budget_bytes
        self.precision = precision
        self.max_dirs = max_dirs
        self.footprint = footprint
        self.max_side = max_side
        self.clock = clock
        self.lock = threading.Condition()
        self.pending = collections.OrderedDict()     # key -> deque of requests
        self.ctxs = {}                               # key -> _Ctx
        self.results = {}
        self.used = 0
        self.peak = 0
        self.batches = []                            # (key, number of requests, directions)
        self.t0 = None
        self.errors = []
        self.enomem = 0                              # batches answered CAVITY_ENOMEM

    # ---------------------------------------------------------------- public
    def run(self, requests, time_scale=1.0):
        """Replay the requests at their arrival times (scaled) and block until
        all are answered; returns the results by request id."""
        self.t0 = self.clock()
        todo = sorted(requests, key=lambda r: r.arrival)
        for r in todo:
            wait = r.arrival * time_scale - (self.clock() - self.t0)
            if wait > 0:
                time.sleep(wait)
            self.submit(r, now=self.clock() - self.t0)
        with self.lock:
            while len(self.results) < len(todo) and not self.errors:
                self.lock.wait(timeout=1.0)
            self._close_all_idle()
        if self.errors:
            raise self.errors[0]
        return self.results

    def submit(self, r, now):
        with self.lock:
            a, b, c, nx, ny, nz = r.geom
            if max(nx, ny) > self.max_side:
                self.results[r.rid] = Result(r.rid, 1, now, now, now, 0)
                self.lock.notify_all()
                return
            r._arr = now
            self.pending.setdefault(r.key, collections.deque()).append(r)
            self._dispatch()

    # ------------------------------------------------------------- internals
    def _dispatch(self):
        # called with the lock held: start a batch on every idle context with
        # pending work; admit contexts for keys without one while memory lasts
        for key in list(self.pending):
            q = self.pending[key]
            if not q:
                continue
            ctx = self.ctxs.get(key)
            if ctx is None:
                r0 = q[0]
                layered = len(r0.layers) > 1
                need = self.footprint(r0.geom, self.max_dirs, self.precision, layered,
                                      any(r.want_field for r in q))
                if need > self.budget:
                    # can never fit: CAVITY_ENOMEM for every request of the key
                    while q:
                        r = q.popleft()
                        self.results[r.rid] = Result(r.rid, 2, r._arr, r._arr, r._arr, 0)
                    self.lock.notify_all()
                    continue
                if not self._admit(need):
                    continue
                ctx = _Ctx(key, need)
                self.ctxs[key] = ctx
                self.used += need
                self.peak = max(self.peak, self.used)
            if ctx.busy or ctx.closing:
                continue
            batch, nd = [], 0
            while q and (not batch or nd + q[0].ndir <= self.max_dirs):
                r = q.popleft()
                batch.append(r)
                nd += r.ndir
            ctx.busy = True
            threading.Thread(target=self._work, args=(ctx, batch), daemon=True).start()

    def _admit(self, need):
        if self.used + need <= self.budget:
            return True
        # evict idle contexts, least recently used first, while that helps
        idle = sorted((c for c in self.ctxs.values() if not c.busy and not c.closing
                       and not self.pending.get(c.key)), key=lambda c: c.last_used)
        for c in idle:
            if self.used + need <= self.budget:
                break
            self._close(c)
        return self.used + need <= self.budget

    def _close(self, c):
        c.closing = True
        del self.ctxs[c.key]
        self.used -= c.nbytes
        if c.handle is not None:
            self.backend.close(c.handle)

    def _close_all_idle(self):
        for c in list(self.ctxs.values()):
            if not c.busy:
                self._close(c)

    def _work(self, ctx, batch):
        try:
            if ctx.handle is None:
                ctx.handle = self.backend.open(ctx.key)
            start = self.clock() - self.t0
            th = np.concatenate([r.theta for r in batch])
            ph = np.concatenate([r.phi for r in batch])
            al = np.concatenate([r.alpha for r in batch])
            wf = any(r.want_field for r in batch)
            ka = any(r.keep_aperture for r in batch)
            sig, it, res, ap, dof = self.backend.solve(ctx.handle, ctx.key, th, ph, al, wf, ka)
            done = self.clock() - self.t0
            with self.lock:
                o = 0
                for r in batch:
                    s = slice(o, o + r.ndir)
                    self.results[r.rid] = Result(
                        r.rid, 0, r._arr, start, done, len(batch), rcs=np.asarray(sig[s]),
                        iters=np.asarray(it[s]), resid=np.asarray(res[s]),
                        aperture=(ap[s] if (ap is not None and r.keep_aperture) else None),
                        dof=dof * r.ndir)
                    o += r.ndir
                self.batches.append((ctx.key, len(batch), o))
                ctx.busy = False
                ctx.last_used = done
                self._dispatch()
                self.lock.notify_all()
        except Exception as e:
            status = getattr(e, "status", None)
            with self.lock:
                if status == 2:
                    # the device ran out of memory for this batch (the
                    # footprint is an estimate): CAVITY_ENOMEM for its
                    # requests, the server carries on
                    now = self.clock() - self.t0
                    for r in batch:
                        self.results[r.rid] = Result(r.rid, 2, r._arr, now, now, len(batch))
                    self.enomem += 1
                    ctx.busy = False
                    self._dispatch()
                else:  # surface other backend failures to run()
                    self.errors.append(e)
                    ctx.busy = False
                self.lock.notify_all()


def summary(results, wall):
    ok = [r for r in results.values() if r.status == 0]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    dof = sum(r.dof for r in ok)
    return {"answered": len(ok), "rejected": len(results) - len(ok),
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                           "p99": 1e3 * float(np.percentile(lat, 99))},
            "dof_per_s": dof / wall if wall > 0 else 0.0, "wall_s": wall}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=100)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--rate", type=float, default=0.0,
                    help="arrivals per second; 0: 0.7 x the FP64 path's measured capacity")
    ap.add_argument("--budget-gb", type=float, default=200.0)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--catalogue", type=int, default=0,
                    help="number of distinct cavities the requests draw from (0: one per request)")
    ap.add_argument("--keep-every", type=int, default=0,
                    help="keep the aperture of every n-th request and write it to --dump")
    ap.add_argument("--dump", default="",
                    help=".npz file for the kept requests (inputs, first direction's aperture, RCS)")
    ap.add_argument("--rate-of", default="fp64", choices=["mixed", "fp64"],
                    help="with --rate 0: the path whose measured capacity sets the rate")
    ap.add_argument("--load", type=float, default=0.7,
                    help="with --rate 0: arrivals as this fraction of that capacity")
    args = ap.parse_args()
    rate = args.rate
    cap = None
    if rate <= 0:
        # capacity of a path: requests per second when a stream of the same
        # mix is solved one request at a time (on contexts of the catalogue
        # when there is one, else each on a new context)
        probe = [r for r in workload_requests(12, 1.0, seed=args.seed + 1000, catalogue=args.catalogue)
                 if max(r.geom[3], r.geom[4]) <= MAX_SIDE][:8]
        for r in probe:
            r.arrival = 0.0
            r.keep_aperture = False
        srv = Server(GpuBackend(args.rate_of), int(args.budget_gb * 2**30), precision=args.rate_of,
                     max_dirs=32)
        t0 = time.perf_counter()
        for r in probe:
            srv.run([r])
        cap = len(probe) / (time.perf_counter() - t0)
        rate = args.load * cap
    reqs = workload_requests(args.requests, rate, seed=args.seed, catalogue=args.catalogue,
                             keep_every=args.keep_every)
    srv = Server(GpuBackend(args.precision), int(args.budget_gb * 2**30),
                 precision=args.precision, max_dirs=64)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    out = summary(res, wall)
    by = collections.Counter(b[1] for b in srv.batches)
    out.update({"precision": args.precision, "requests": args.requests, "rate_per_s": rate,
                "capacity_per_s": cap, "rate_of": args.rate_of if cap else None,
                "seed": args.seed, "catalogue": args.catalogue, "batches": len(srv.batches),
                "mean_requests_per_batch": float(np.mean([b[1] for b in srv.batches])),
                "batch_sizes": {str(k): v for k, v in sorted(by.items())},
                "contexts_opened": len({b[0] for b in srv.batches}),
                "enomem_batches": srv.enomem,
                "peak_admitted_gb": srv.peak / 2**30})
    print(json.dumps(out))
    if args.dump:
        # grids above 512 points per side are kept by RCS only (a 1024^2
        # aperture vector is 50 MB, and no reference checks it)
        kept = [r for r in reqs if r.keep_aperture and res[r.rid].status == 0 and r.geom[3] <= 512]
        # one aperture array per kept request (their grids differ)
        aps = {"aperture_%d" % i: res[r.rid].aperture[0].numpy() for i, r in enumerate(kept)}
        np.savez(args.dump, precision=args.precision, tol=1e-7,
                 rid=np.array([r.rid for r in kept]),
                 geom=np.array([r.geom for r in kept], dtype=float),
                 kappa0=np.array([r.kappa0 for r in kept]),
                 layers=np.array([[(n, e) for n, e in r.layers] for r in kept], dtype=complex),
                 theta=np.array([r.theta[0] for r in kept]), phi=np.array([r.phi[0] for r in kept]),
                 alpha=np.array([r.alpha[0] for r in kept]),
                 rcs=np.array([res[r.rid].rcs[0] for r in kept]),
                 resid=np.array([res[r.rid].resid[0] for r in kept]), **aps)


if __name__ == "__main__":
    main()
