"""The seeded input recipe (workloads.py) against the workloads it is meant
to produce: grid sizes, direction ranges, permittivity sets, ten points per
wavelength, repeatability of the seeds, and scaled versions that keep the
points per wavelength."""

import numpy as np

import workloads


def _ppw(kappa0, h, eps_re=1.0):
    """Grid points per wavelength in a medium of relative permittivity eps_re."""
    return 2 * np.pi / (kappa0 * np.sqrt(eps_re)) / h


def test_small_workload():
    w = workloads.workload('small')
    assert (w['nx'], w['ny'], w['nz']) == (32, 32, 32)
    assert w['kappa0'] == 8 * np.pi                       # aperture of 4 wavelengths
    assert w['a'] * w['kappa0'] / (2 * np.pi) == 4.0
    assert np.all(w['theta'] == 0) and np.all(w['phi'] == 0) and np.all(w['alpha'] == 0)


def test_benchmark_workload_dirs16():
    w = workloads.workload('dirs16')
    assert (w['nx'], w['ny'], w['nz']) == (256, 256, 128)
    assert len(w['theta']) == 16 and np.all(w['alpha'] == 0)
    assert np.all((0 <= w['theta']) & (w['theta'] < np.pi / 3))
    assert np.all((0 <= w['phi']) & (w['phi'] < 2 * np.pi))
    # ten points per wavelength horizontally and vertically
    assert abs(_ppw(w['kappa0'], w['a'] / w['nx']) - 10.0) < 1e-12
    assert abs(_ppw(w['kappa0'], w['c'] / w['nz']) - 10.0) < 1e-12
    w2 = workloads.workload('dirs16')
    assert np.array_equal(w['theta'], w2['theta']) and np.array_equal(w['phi'], w2['phi'])


def test_layered_workload():
    w = workloads.workload('layered4')
    assert (w['nx'], w['ny'], w['nz']) == (512, 512, 256)
    assert [n for n, _ in w['layers']] == [64, 64, 64, 64]
    key = lambda e: (e.real, e.imag)  # noqa: E731
    assert sorted((e for _, e in w['layers']), key=key) == sorted(workloads.EPS_SET, key=key)
    assert len(w['theta']) == 8
    # ten points per wavelength in the densest layer (Re eps = 6)
    assert abs(_ppw(w['kappa0'], w['c'] / w['nz'], 6.0) - 10.0) < 1e-12


def test_scaled_workloads_keep_points_per_wavelength():
    for name in ('dirs16', 'layered4'):
        w = workloads.workload(name)
        for nx in (16, 64):
            s = workloads.scaled(name, nx, ndir=3)
            assert s['nx'] == nx and len(s['theta']) == 3
            assert sum(n for n, _ in s['layers']) == s['nz']
            eps = max(e.real for _, e in w['layers'])
            assert abs(_ppw(s['kappa0'], s['c'] / s['nz'], eps)
                       - _ppw(w['kappa0'], w['c'] / w['nz'], eps)) < 0.6
            assert [e for _, e in s['layers']] == [e for _, e in w['layers']]


def test_rcs_sweep48_recipe():
    cs = workloads.rcs_sweep48()
    assert len(cs) == 48
    assert {c['nx'] for c in cs} == {64, 128, 256, 512}
    nl = set()
    for c in cs:
        assert c['ny'] == c['nx'] and c['nz'] == c['nx'] // 2
        assert sum(n for n, _ in c['layers']) == c['nz']
        L = len(c['layers'])
        nl.add(L)
        assert L == 1 or 2 <= L <= 4
        if L == 1:
            assert c['layers'][0][1] == 1.0
        else:
            assert all(1 <= e.real <= 6 and 0 <= e.imag <= 1 for _, e in c['layers'])
        eps = max(e.real for _, e in c['layers'])
        k10 = c['kappas'][-1]
        assert abs(_ppw(k10, c['c'] / c['nz'], eps) - 10.0) < 1e-9
        assert np.allclose(np.array(c['kappas']) / k10, [0.25, 0.5, 0.75, 1.0])
        assert len(c['theta']) == 64
    assert 1 in nl and len(nl) > 1                      # both homogeneous and layered fills
    cs2 = workloads.rcs_sweep48()
    assert all(np.array_equal(a['theta'], b['theta']) and a['layers'] == b['layers']
               for a, b in zip(cs, cs2))
