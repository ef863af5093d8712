"""The autotuner's bookkeeping on the CPU with a stand-in context and timer:
the candidates that apply to a shape, the fastest value kept and set, widths
whose solve did not converge skipped, the JSON cache keyed by shape and
precision, and a cached choice applied without timing."""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2008_01966_gb300 import autotune


class FakeCav:
    def __init__(self, n=512, nz=16, precision=1):
        self.nx = self.ny = n
        self.nz = nz
        self.precision = precision
        self.opts = {"pass_b_2048": 0, "pass_c_2048": 0, "group_width": 16, "field_fused": 0}
        self.last_status = 0
        self.prepared = 0

    def set_option(self, name, v):
        self.opts[name] = v

    def prepare(self, kappa0, layers):
        self.prepared += 1

    def rhs(self, th, ph, al):
        class X:
            def to(self, dtype=None):
                return self
        return X()

    def apply(self, x, prec):
        pass

    def field(self, ap):
        pass

    def solve(self, *a, **k):
        # width 4 does not converge in this stand-in
        self.last_status = 4 if self.opts["group_width"] == 4 else 0
        return None, None, [1], [0.0]


class FakeTimer:
    """Time = a table lookup of the option values in force."""

    def __init__(self, cav, table):
        self.cav, self.table, self.calls = cav, table, 0

    def __call__(self, fn, reps):
        fn()
        self.calls += 1
        o = self.cav.opts
        return (self.table["b"][o["pass_b_2048"]] + self.table["c"][o["pass_c_2048"]] +
                self.table["g"][o["group_width"]] + self.table.get("f", {}).get(o["field_fused"], 0.0))


def test_candidates_by_shape_and_precision():
    assert autotune.candidates(FakeCav(512)) == {"pass_b_2048": (0, 1), "pass_c_2048": (0, 1),
                                                 "group_width": autotune.GROUP_WIDTHS,
                                                 "field_fused": autotune.FIELD_PATHS}
    assert autotune.candidates(FakeCav(256)) == {"group_width": autotune.GROUP_WIDTHS,
                                                 "field_fused": autotune.FIELD_PATHS}
    assert autotune.candidates(FakeCav(16)) == {"group_width": autotune.GROUP_WIDTHS}
    assert autotune.candidates(FakeCav(512, precision=0)) == {}


def test_tune_keeps_the_fastest_skips_unconverged_and_caches(tmp_path):
    cav = FakeCav()
    table = {"b": {0: 5.0, 1: 7.0}, "c": {0: 3.0, 1: 1.0}, "g": {16: 9.0, 8: 4.0, 4: 0.5},
             "f": {1: 2.0, 2: 6.0}}
    timer = FakeTimer(cav, table)
    cache = str(tmp_path / "tune.json")
    out = autotune.tune(cav, 1.0, [(8, 1.0), (8, 2.0)], [0.1, 0.2], [0.0, 1.0], [0.0, 0.0],
                        cache=cache, reps=1, timer=timer)
    # pass B: 0 faster; pass C: 1 faster; width 4 fastest but unconverged -> 8;
    # the fused field faster
    assert out["choice"] == {"pass_b_2048": 0, "pass_c_2048": 1, "group_width": 8,
                             "field_fused": 1}
    assert cav.opts == out["choice"] and not out["cached"]
    assert out["key"] == "512x512x16/mixed/layered/ndir2"
    stored = json.load(open(cache))
    assert stored[out["key"]]["choice"] == out["choice"]
    assert set(stored[out["key"]]["ms"]["group_width"]) == {"16", "8"}
    # a second context of the same shape: the cached choice, no timing
    cav2 = FakeCav()
    t2 = FakeTimer(cav2, table)
    out2 = autotune.tune(cav2, 1.0, [(8, 1.0), (8, 2.0)], [0.3, 0.4], [0.0, 1.0], [0.0, 0.0],
                         cache=cache, reps=1, timer=t2)
    assert out2["cached"] and out2["choice"] == out["choice"] and t2.calls == 0
    assert cav2.opts == out["choice"] and cav2.prepared == 0
    # another shape is tuned on its own
    cav3 = FakeCav(256)
    out3 = autotune.tune(cav3, 1.0, [(16, 1.0)], [0.1], [0.0], [0.0], cache=cache, reps=1,
                         timer=FakeTimer(cav3, table))
    assert out3["key"] == "256x256x16/mixed/homogeneous/ndir1"
    assert len(json.load(open(cache))) == 2
