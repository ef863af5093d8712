"""Host logic of the 48-cavity sweep driver on the CPU, with a stand-in
backend: every (cavity, wavenumber) pair is prepared and solved once, one
context per cavity is opened and closed, the field is requested exactly for
sides up to 128, and the solve and DOF counts of the summary are those of the
seeded sweep (12,288 solves)."""

import numpy as np

import workloads
from paper_2008_01966_gb300 import sweep48


class FakeBackend:
    def __init__(self):
        self.events = []

    def open(self, cv):
        self.events.append(("open", cv['nx']))
        return {"cv": cv, "open": True}

    def prepare(self, cav, cv, kappa0):
        assert cav["open"]
        self.events.append(("prepare", kappa0))

    def solve(self, cav, cv, kappa0, want_field):
        self.events.append(("solve", cv['nx'], want_field))
        n = len(cv['theta'])
        return np.ones(n), np.full(n, 12), np.full(n, 5e-8)

    def close(self, cav):
        cav["open"] = False
        self.events.append(("close",))


def test_full_sweep_bookkeeping():
    cavities = workloads.rcs_sweep48()
    fb = FakeBackend()
    t = iter(np.arange(0.0, 1e6, 0.5))
    records = sweep48.run(fb, cavities, clock=lambda: next(t))
    assert len(records) == 48 * 4
    kinds = [e[0] for e in fb.events]
    assert kinds.count("open") == 48 and kinds.count("close") == 48
    assert kinds.count("prepare") == 192 and kinds.count("solve") == 192
    for e in fb.events:
        if e[0] == "solve":
            assert e[2] == (e[1] <= 128)
    s = sweep48.summary(records, wall_s=100.0)
    assert s["solves"] == 12288
    want_dof = sum(64 * 4 * cv['nz'] * (3 * (cv['nx'] - 1) ** 2 + 2 * (cv['nx'] - 1))
                   for cv in cavities)
    assert s["dof_per_s"] == want_dof / 100.0
    sides = {int(k) for k in s["by_side"]}
    assert sides <= {64, 128, 256, 512}
    assert sum(c["solves"] for c in s["by_side"].values()) == 12288
    assert all(c["max_resid"] == 5e-8 and c["max_iters"] == 12 for c in s["by_side"].values())
    assert all(c["field"] == (int(k) <= 128) for k, c in s["by_side"].items())
    # each pair's setup and solve times come from the clock (0.5 s apart here)
    assert all(r["setup_s"] == 0.5 and r["solve_s"] == 0.5 for r in records)


def test_context_closed_when_a_solve_fails():
    class Failing(FakeBackend):
        def solve(self, cav, cv, kappa0, want_field):
            raise RuntimeError("solve failed")

    fb = Failing()
    try:
        sweep48.run(fb, workloads.rcs_sweep48()[:1])
    except RuntimeError:
        pass
    assert fb.events[-1] == ("close",)


def test_tuning_once_per_side_class():
    """With a tuning cache, the options are tuned on the first cavity of each
    side class (its first wavenumber) and applied to every cavity of that
    class before its solves."""
    class Tuning(FakeBackend):
        def tune(self, cav, cv, kappa0, cache):
            self.events.append(("tune", cv['nx'], kappa0, cache))
            return {"group_width": cv['nx'] // 64}

        def apply_choice(self, cav, choice):
            self.events.append(("apply", cav["cv"]['nx'], choice["group_width"]))

    cavities = workloads.rcs_sweep48()
    fb = Tuning()
    choices = {}
    sweep48.run(fb, cavities, tune_cache="c.json", choices=choices)
    tunes = [e for e in fb.events if e[0] == "tune"]
    assert sorted(e[1] for e in tunes) == sorted({cv['nx'] for cv in cavities})
    first = {}
    for cv in cavities:
        first.setdefault(cv['nx'], cv['kappas'][0])
    assert all(e[2] == first[e[1]] and e[3] == "c.json" for e in tunes)
    applies = [e for e in fb.events if e[0] == "apply"]
    assert len(applies) == 48 and all(e[2] == e[1] // 64 for e in applies)
    assert choices == {str(s): {"group_width": s // 64} for s in first}
    # every apply precedes the cavity's first solve
    last = None
    for e in fb.events:
        if e[0] == "apply":
            last = "apply"
        elif e[0] == "solve":
            assert last in ("apply", "solve")
            last = "solve"
        elif e[0] == "open":
            last = "open"
