"""The 48-cavity backscatter sweep: cavities of uneven sides 64..512 (Nz =
side / 2), homogeneous and 2-4 layer fills, four wavenumbers each and 64
incident directions per wavenumber, 12,288 solves in all (the seeded inputs
are `workloads.rcs_sweep48()`).

The sweep runs cavity by cavity through the library: one context per cavity,
one prepare (kernel table, per-mode elimination, preconditioner) and one
batched 64-direction solve per wavenumber, the backscatter RCS sigma_theta
of every direction, and the interior field for sides up to 128 (larger
fields are not materialised: their DOF are the system's, counted as
Nz x n_ap per direction).  The mixed solve synchronises with the host once
per block step, so the sweep is not one captured launch.

    python -m paper_2008_01966_gb300.sweep48 [--subset K] [--precision mixed]
                                             [--tune CACHE.json]

prints one JSON line: solves, wall time, solves/s, DOF/s, and per side class
the solves, setup and solve seconds and the largest residual.  With --tune,
the implementation options (include/cavity.h, CAVITY_OPT_*) are chosen by the
autotuner on the first cavity of each side class (its first wavenumber, all
64 directions), cached in CACHE.json and applied to every cavity of the
class; the tuning time counts in the wall time and the choices are printed.
"""

import argparse
import json
import time

FIELD_MAX_SIDE = 128


def n_ap(nx, ny):
    """Aperture unknowns 3MN + M + N with M = nx - 1, N = ny - 1."""
    M, N = nx - 1, ny - 1
    return 3 * M * N + M + N


class GpuBackend:
    """Contexts on the GPU through the library (the current CUDA stream)."""

    def __init__(self, precision="mixed", tol=1e-7):
        import torch
        import paper_2008_01966_gb300 as gb
        self.torch, self.gb = torch, gb
        self.precision, self.tol = precision, tol

    def open(self, cv):
        return self.gb.Cavity(cv['a'], cv['b'], cv['c'], cv['nx'], cv['ny'], cv['nz'],
                              precision=self.precision, gmres_tol=self.tol)

    def prepare(self, cav, cv, kappa0):
        cav.prepare(kappa0, cv['layers'])
        self.torch.cuda.synchronize()

    def tune(self, cav, cv, kappa0, cache):
        from . import autotune
        out = autotune.tune(cav, kappa0, cv['layers'], cv['theta'], cv['phi'], cv['alpha'],
                            cache=cache)
        self.torch.cuda.synchronize()
        return out["choice"]

    def apply_choice(self, cav, choice):
        for name, v in choice.items():
            cav.set_option(name, v)

    def solve(self, cav, cv, kappa0, want_field):
        ap, _, it, res = cav.solve(kappa0, cv['layers'], cv['theta'], cv['phi'], cv['alpha'],
                                   field=want_field)
        sig = cav.rcs(ap, cv['theta'], cv['phi'], "theta")
        self.torch.cuda.synchronize()
        return sig, it, res

    def close(self, cav):
        cav.close()


def run(backend, cavities, clock=time.perf_counter, tune_cache=None, choices=None):
    """Solve every (cavity, wavenumber) pair; one record per pair.  With
    tune_cache, options are tuned once per side class (first cavity, first
    wavenumber) and applied to the class; `choices` receives them by side."""
    records = []
    chosen = {} if choices is None else choices
    for ci, cv in enumerate(cavities):
        cav = backend.open(cv)
        try:
            if tune_cache is not None:
                side = str(cv['nx'])
                if side not in chosen:
                    chosen[side] = backend.tune(cav, cv, cv['kappas'][0], tune_cache)
                backend.apply_choice(cav, chosen[side])
            for ki, kappa0 in enumerate(cv['kappas']):
                t0 = clock()
                backend.prepare(cav, cv, kappa0)
                t1 = clock()
                want_field = cv['nx'] <= FIELD_MAX_SIDE
                sig, it, res = backend.solve(cav, cv, kappa0, want_field)
                t2 = clock()
                ndir = len(cv['theta'])
                records.append(dict(cavity=ci, kappa=ki, side=cv['nx'], ndir=ndir,
                                    field=want_field, setup_s=t1 - t0, solve_s=t2 - t1,
                                    iters=int(max(it)), resid=float(max(res)),
                                    sigma_min=float(min(sig)),
                                    dof=ndir * cv['nz'] * n_ap(cv['nx'], cv['ny'])))
        finally:
            backend.close(cav)
    return records


def summary(records, wall_s):
    solves = sum(r['ndir'] for r in records)
    dof = sum(r['dof'] for r in records)
    by_side = {}
    for r in records:
        c = by_side.setdefault(str(r['side']), dict(solves=0, setup_s=0.0, solve_s=0.0,
                                                    max_resid=0.0, max_iters=0, field=r['field']))
        c['solves'] += r['ndir']
        c['setup_s'] += r['setup_s']
        c['solve_s'] += r['solve_s']
        c['max_resid'] = max(c['max_resid'], r['resid'])
        c['max_iters'] = max(c['max_iters'], r['iters'])
    return dict(solves=solves, wall_s=wall_s,
                solves_per_s=solves / wall_s if wall_s > 0 else None,
                dof_per_s=dof / wall_s if wall_s > 0 else None,
                dof_note="system DOF, Nz x n_ap per direction; the field is written "
                         "for sides <= %d only" % FIELD_MAX_SIDE,
                by_side=dict(sorted(by_side.items(), key=lambda kv: int(kv[0]))))


def main(argv=None):
    import workloads
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--subset", type=int, default=0,
                    help="only the first K cavities of the sweep (0: all 48)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--tune", default=None, metavar="CACHE.json",
                    help="autotune the implementation options per side class")
    args = ap.parse_args(argv)
    cavities = workloads.rcs_sweep48()
    if args.subset:
        cavities = cavities[:args.subset]
    backend = GpuBackend(args.precision, args.tol)
    t0 = time.perf_counter()
    choices = {}
    records = run(backend, cavities, tune_cache=args.tune, choices=choices)
    wall = time.perf_counter() - t0
    out = summary(records, wall)
    out.update(precision=args.precision, tol=args.tol, cavities=len(cavities))
    if args.tune:
        out["tuned_options"] = choices
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
