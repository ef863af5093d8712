"""The serving-sample checker (tests/check_serving_sample.py) on a dump made
on the CPU: the oracle's own solution passes, a perturbed one fails, and
grids above 512 points per side are listed as skipped."""

import os
import sys

import numpy as np

from oracle.aperture import ApertureSystem
from oracle.excitation import rhs
from oracle.geometry import Cavity, Layer
from oracle.rcs import backscatter

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import check_serving_sample  # noqa: E402


def dump(path, aperture, rcs, geom=(1.0, 1.0, 0.5, 8, 8, 8), extra=None):
    layers = [(4, 2.0 + 0.5j), (4, 1.0 + 0j)]
    rec = dict(precision="mixed", tol=1e-7, rid=np.array([0]), geom=np.array([geom]),
               kappa0=np.array([9.0]), layers=np.array([layers], dtype=complex),
               theta=np.array([0.3]), phi=np.array([0.7]), alpha=np.array([0.0]),
               rcs=np.array([rcs]), resid=np.array([1e-8]), aperture_0=aperture)
    np.savez(path, **rec)


def reference():
    cav = Cavity(1.0, 1.0, 0.5, 8, 8, 8, 9.0, layers=[Layer(4, 2.0 + 0.5j), Layer(4, 1.0 + 0j)])
    sysm = ApertureSystem(cav)
    b = rhs(cav, 0.3, 0.7, 0.0)
    x = sysm.solve_dense(b[None, :])[0]
    return x, backscatter(cav, x, 0.3, 0.7, "theta")


def test_checker_accepts_the_reference_and_rejects_a_perturbation(tmp_path, capsys):
    x, sig = reference()
    good = str(tmp_path / "good.npz")
    dump(good, x, sig)
    assert check_serving_sample.main(good) == 0
    bad = str(tmp_path / "bad.npz")
    dump(bad, x * (1 + 1e-3), sig)
    assert check_serving_sample.main(bad) == 1
    assert "FAIL" in capsys.readouterr().out


def test_checker_skips_grids_beyond_its_limit(tmp_path, capsys):
    big = str(tmp_path / "big.npz")
    dump(big, np.zeros(3, dtype=complex), 1.0, geom=(1.0, 1.0, 0.5, 1024, 1024, 512))
    assert check_serving_sample.main(big) == 0
    assert "skipped" in capsys.readouterr().out
