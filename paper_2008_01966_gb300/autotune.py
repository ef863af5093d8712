"""Autotuner of the library's implementation options (include/cavity.h,
CAVITY_OPT_*): for a context's shape it times every candidate value of each
option on the work that option affects, keeps the fastest, and caches the
choice in a JSON file keyed by shape and precision, so later contexts of the
same shape reuse it without timing.

    from paper_2008_01966_gb300 import autotune
    choice = autotune.tune(cav, kappa0, layers, theta, phi, alpha, cache="tune.json")

Options and what is timed:
  pass_b_2048, pass_c_2048  (512-point grid sides, mixed precision): one
      application of the FP32 operator to the batch (cavity_apply), per value;
  group_width (mixed precision): the aperture solve of the batch (cavity_solve
      without the field), per value among GROUP_WIDTHS; a width is kept only if
      every direction converged;
  field_fused (mixed precision, square grids of 32..512 points per side): one
      field synthesis of the batch (cavity_field) with the fused kernel (1)
      and with the two-pass kernels (2), each after a prepare (the option
      changes the layout of the FP32 profiles).
Values are compared by the median of `reps` timed repetitions after one
warm-up, measured with CUDA events on the context's stream.
"""

import json
import os

GROUP_WIDTHS = (16, 8, 4)
FIELD_PATHS = (1, 2)   # fused kernel, two-pass kernels


def shape_key(cav, ndir, layered):
    return "%dx%dx%d/%s/%s/ndir%d" % (cav.nx, cav.ny, cav.nz,
                                      "fp64" if cav.precision == 0 else "mixed",
                                      "layered" if layered else "homogeneous", ndir)


def candidates(cav):
    """{option: candidate values} that apply to this context."""
    out = {}
    if cav.precision != 0 and (cav.nx == 512 or cav.ny == 512):
        if cav.nx == 512:
            out["pass_b_2048"] = (0, 1)
        if cav.ny == 512:
            out["pass_c_2048"] = (0, 1)
    if cav.precision != 0:
        out["group_width"] = GROUP_WIDTHS
    if cav.precision != 0 and cav.nx == cav.ny and 32 <= cav.nx <= 512:
        out["field_fused"] = FIELD_PATHS
    return out


def _median(v):
    v = sorted(v)
    return v[len(v) // 2]


class _Timer:
    """CUDA-event timing of a callable on the context's stream."""

    def __init__(self, cav):
        import torch
        self.torch, self.stream = torch, cav.stream

    def __call__(self, fn, reps):
        torch = self.torch
        fn()
        out = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(self.stream)
            fn()
            b.record(self.stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return _median(out)


def load_cache(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(path, cache):
    if not path:
        return
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(cav, kappa0, layers, theta, phi, alpha, cache=None, reps=3, timer=None):
    """Choose and set every applicable option of `cav` for this batch; returns
    {"key": shape key, "choice": {option: value}, "ms": {option: {value: ms}},
    "cached": bool}."""
    layered = len(layers) > 1
    key = shape_key(cav, len(theta), layered)
    store = load_cache(cache)
    if key in store:
        for name, v in store[key]["choice"].items():
            cav.set_option(name, v)
        return {"key": key, "choice": store[key]["choice"], "ms": store[key].get("ms", {}),
                "cached": True}
    timer = timer or _Timer(cav)
    cands = candidates(cav)
    choice, ms = {}, {}
    if "field_fused" in cands:
        res = {}
        for v in cands["field_fused"]:
            cav.set_option("field_fused", v)
            cav.prepare(kappa0, layers)
            ap = cav.rhs(theta, phi, alpha)
            res[v] = timer(lambda: cav.field(ap), reps)
        best = min(res, key=res.get)
        cav.set_option("field_fused", best)
        choice["field_fused"], ms["field_fused"] = best, {str(k): t for k, t in res.items()}
    cav.prepare(kappa0, layers)
    x = None
    for name in ("pass_b_2048", "pass_c_2048"):
        if name not in cands:
            continue
        if x is None:
            x = cav.rhs(theta, phi, alpha).to(dtype=_complex64(cav))
        res = {}
        for v in cands[name]:
            cav.set_option(name, v)
            res[v] = timer(lambda: cav.apply(x, "mixed"), reps)
        best = min(res, key=res.get)
        cav.set_option(name, best)
        choice[name], ms[name] = best, {str(k): t for k, t in res.items()}
    if "group_width" in cands:
        res = {}
        for v in cands["group_width"]:
            cav.set_option("group_width", v)
            ok = []

            def solve():
                _, _, it, r = cav.solve(kappa0, layers, theta, phi, alpha, field=False)
                ok.append(cav.last_status == 0)
            t = timer(solve, reps)
            if all(ok):
                res[v] = t
        best = min(res, key=res.get) if res else 16
        cav.set_option("group_width", best)
        choice["group_width"], ms["group_width"] = best, {str(k): t for k, t in res.items()}
    store = load_cache(cache)
    store[key] = {"choice": choice, "ms": ms}
    save_cache(cache, store)
    return {"key": key, "choice": choice, "ms": ms, "cached": False}


def apply_choice(cav, choice):
    for name, v in choice.items():
        cav.set_option(name, v)


def _complex64(cav):
    import torch
    return torch.complex64
