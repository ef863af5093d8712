"""The oracle against its stored regression values (tests/golden/, written by
tests/golden/make_golden.py from oracle/ only).  The paper prints no solution
values, so these are not pins: they fix the oracle's current results so that
any change of its arithmetic comes with a changed fixture."""

import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


@pytest.mark.parametrize("name", make_golden.CASES)
def test_oracle_reproduces_golden(name):
    want = make_golden.read(os.path.join(HERE, "golden", "%s_oracle.txt" % name))
    got = make_golden.compute(name)
    assert got['n_ap'] == want['n_ap']
    assert got['resid'] < 1e-12 and want['resid'] < 1e-12
    assert got['norm'] == pytest.approx(want['norm'], rel=1e-10)
    # one polarisation can vanish by symmetry (rounding-level values)
    rs = max(want['rcs_theta'], want['rcs_phi'])
    for k in ('rcs_theta', 'rcs_phi'):
        assert abs(got[k] - want[k]) <= 1e-10 * rs, k
    scale = want['norm']
    for (i, v), (i2, v2) in zip(got['aperture'], want['aperture']):
        assert i == i2 and abs(v - v2) <= 1e-10 * scale
    fscale = max(abs(v) for *_, v in want['field'])
    for a, b in zip(got['field'], want['field']):
        assert a[:4] == b[:4] and abs(a[4] - b[4]) <= 1e-10 * fscale
