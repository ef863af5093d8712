"""The C-ABI library builds for sm_103a and exports every entry point that
include/cavity.h declares (no compute call: this runs without a GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "cavity.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cavity_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_2008_01966_gb300 import _lib
    assert declared_symbols() == sorted(_lib.EXPORTS)


def test_every_cuda_unit_is_built():
    """build.py compiles every .cu file under csrc/ (a unit left out would
    leave its kernels' explicit instantiations unresolved only at load time)."""
    from paper_2008_01966_gb300 import build
    csrc = os.path.join(ROOT, "paper_2008_01966_gb300", "csrc")
    units = sorted(f for f in os.listdir(csrc) if f.endswith(".cu"))
    assert sorted(os.path.basename(s) for s in build.SOURCES) == units
    assert set(os.path.basename(s) for s in build.SPLIT) <= set(units)


def test_library_builds_and_exports_every_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_01966_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_setup_rejects_bad_descriptors_without_a_gpu():
    """Argument validation happens on the host before any device work."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2008_01966_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    for bad in (dict(nx=12), dict(nz=1), dict(a=-1.0), dict(precision=7), dict(pad_factor=3),
                dict(a=1.0, b=0.3), dict(restart=121), dict(khat_scheme=2), dict(modes_m=-1),
                dict(modes_m=16), dict(modes_n=16), dict(a=1.0, b=0.05),
                dict(a=1.0, b=0.25, pad_factor=4)):
        kw = dict(a=1.0, b=1.0, c=0.5, nx=16, ny=16, nz=8, precision=0, pad_factor=0,
                  restart=0, khat_scheme=0, modes_m=0, modes_n=0)
        kw.update(bad)
        d = _lib.CavityDesc(kw['a'], kw['b'], kw['c'], kw['nx'], kw['ny'], kw['nz'],
                            kw['precision'], kw['pad_factor'], 0.0, kw['restart'], 0, 0.0,
                            kw['khat_scheme'], kw['modes_m'], kw['modes_n'])
        st = lib.cavity_setup(ctypes.byref(d), None, ctypes.byref(h))
        assert st == _lib.CAVITY_EINVAL, bad
        assert lib.cavity_last_error(None)
    assert lib.cavity_setup(None, None, ctypes.byref(h)) == _lib.CAVITY_EINVAL


def test_operator_io_checks_raise_before_the_library_is_called():
    """The binding checks y (and x) before it hands raw pointers to the
    library: wrong device, dtype, shape, stride, or y overlapping x."""
    torch = pytest.importorskip("torch")
    import paper_2008_01966_gb300 as gb
    cpu = torch.device("cpu")
    n = 10
    x = torch.zeros((2, n), dtype=torch.complex128)
    gb.check_operator_io(x, torch.empty_like(x), torch.complex128, n, cpu)
    bad_y = [torch.zeros((2, n), dtype=torch.complex64),          # dtype
             torch.zeros((3, n), dtype=torch.complex128),         # shape
             torch.zeros((2, n + 1), dtype=torch.complex128),     # n_ap
             torch.zeros((n, 2), dtype=torch.complex128).t(),     # not contiguous
             torch.zeros((2, n), dtype=torch.complex128, device="meta"),  # device
             x,                                                   # y is x
             torch.zeros((3, n), dtype=torch.complex128)[1:],     # ok on its own ...
             "not a tensor"]
    big = torch.zeros((3, n), dtype=torch.complex128)
    x_in_big = big[:2]
    for k, y in enumerate(bad_y):
        xx = x
        if k == 6:
            xx, y = x_in_big, big[1:]                             # ... but overlaps x
        with pytest.raises(ValueError):
            gb.check_operator_io(xx, y, torch.complex128, n, cpu)
    with pytest.raises(ValueError):
        gb.check_operator_io(x.to(torch.complex64), torch.empty_like(x), torch.complex128, n,
                             cpu)


def test_lu_io_checks_raise_before_the_library_is_called():
    """The binding checks lu, ipiv and b before the LU solve gets their raw
    pointers: device, dtype, shape, stride, and b overlapping lu or ipiv."""
    torch = pytest.importorskip("torch")
    import paper_2008_01966_gb300 as gb
    cpu = torch.device("cpu")
    n = 6
    lu = torch.zeros((n, n), dtype=torch.complex64)
    ipiv = torch.zeros(n, dtype=torch.int32)
    b = torch.zeros((2, n), dtype=torch.complex64)
    gb.check_lu_io(lu, ipiv, b, cpu)
    bad = [
        (lu.to(torch.complex128), ipiv, b),                          # lu dtype
        (torch.zeros((n, n + 1), dtype=torch.complex64), ipiv, b),   # lu not square
        (lu.t(), ipiv, b),                                           # lu not contiguous
        (lu, ipiv.to(torch.int64), b),                               # ipiv dtype
        (lu, torch.zeros(n - 1, dtype=torch.int32), b),              # ipiv length
        (lu, ipiv, b.to(torch.complex128)),                          # b dtype
        (lu, ipiv, torch.zeros((2, n + 1), dtype=torch.complex64)),  # b width
        (lu, ipiv, torch.zeros((n, 2), dtype=torch.complex64).t()),  # b not contiguous
        (lu, ipiv, torch.zeros((2, n), dtype=torch.complex64, device="meta")),  # device
        (lu, ipiv, lu[:2]),                                          # b inside lu
        (lu, ipiv, "not a tensor"),
    ]
    for args in bad:
        with pytest.raises(ValueError):
            gb.check_lu_io(*args, cpu)


def test_noalloc_precision_names_are_checked():
    """Only 'fp64' and 'mixed' reach the allocation-free entry point; any
    other name raises in the binding (no silent mapping to mixed)."""
    torch = pytest.importorskip("torch")
    import paper_2008_01966_gb300 as gb

    class NoLib:
        def __getattr__(self, name):
            raise AssertionError("library called: " + name)
    g = object.__new__(gb.Cavity)
    g.lib, g.h, g.n_ap, g.precision = NoLib(), None, 4, 0
    g.device = torch.device("cpu")
    x = torch.zeros((1, 4), dtype=torch.complex128)
    for name in ("pair32", "fp32", "FP64", ""):
        with pytest.raises(ValueError):
            g.apply_noalloc(x, name)
    with pytest.raises(ValueError):          # a CPU context never reaches the library
        g.apply_noalloc(x, "fp64")
    g.h = None


def test_solve_outputs_and_angles_are_checked_before_the_library():
    """solve's caller-supplied output tensors (shape, dtype, place,
    contiguity, no overlap) and the per-direction angle arrays of solve, rhs
    and rcs (one length) are checked in the binding; a bad one never reaches
    the library."""
    torch = pytest.importorskip("torch")
    import paper_2008_01966_gb300 as gb

    class NoLib:
        def __getattr__(self, name):
            raise AssertionError("library called: " + name)
    g = object.__new__(gb.Cavity)
    g.lib, g.h, g.n_ap, g.precision, g.field_per_dir = NoLib(), None, 4, gb._lib.CAVITY_MIXED, 6
    g.device = torch.device("meta")          # the "device" side of the checks
    lay = [(2, 1.0)]
    th = ph = al = [0.1, 0.2]
    dev = dict(dtype=torch.complex128, device="meta")
    good_ap = torch.empty((2, 4), **dev)
    bad = [
        dict(aperture_out=torch.empty((1, 4), **dev)),                       # ndir
        dict(aperture_out=torch.empty((2, 5), **dev)),                       # n_ap
        dict(aperture_out=torch.empty((2, 4), dtype=torch.complex64, device="meta")),
        dict(aperture_out=torch.empty((4, 2), **dev).t()),                   # stride
        dict(aperture_out=torch.empty((2, 4), dtype=torch.complex128)),      # host tensor
        dict(aperture_out=good_ap, field_out=torch.empty((2, 6), **dev)),    # field dtype
        dict(aperture_out=good_ap, field_out=torch.empty((2, 7), dtype=torch.complex64,
                                                         device="meta")),
    ]
    for kw in bad:
        with pytest.raises(ValueError):
            g.solve(1.0, lay, th, ph, al, field=True, **kw)
    with pytest.raises(ValueError):          # a device tensor for a host solve
        g.solve(1.0, lay, th, ph, al, field=False, host=True, aperture_out=good_ap)
    cpu_ap = torch.zeros((2, 4), dtype=torch.complex128)
    with pytest.raises(ValueError):          # the two outputs share memory
        big = torch.zeros(40, dtype=torch.complex128)
        g.solve(1.0, lay, th, ph, al, field=True, host=True, aperture_out=big[:8].view(2, 4),
                field_out=big[4:10].view(torch.complex64).view(2, 6))
    for f in (lambda: g.solve(1.0, lay, [0.1, 0.2], [0.3], [0.0, 0.0], field=False),
              lambda: g.rhs([0.1, 0.2], [0.3, 0.4], [0.0]),
              lambda: g.rcs(cpu_ap, [0.1, 0.2], [0.3])):
        with pytest.raises(ValueError):
            f()
    g.h = None
