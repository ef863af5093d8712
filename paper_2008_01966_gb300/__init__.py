"""GB300 solver for electromagnetic scattering by an open rectangular cavity in
a perfectly conducting ground plane (Chen, Jiang, Lai, Li: fast algorithm for
the electromagnetic scattering from a large rectangular cavity in 3D).

The Python layer only marshals arguments to the C ABI of include/cavity.h
(libcavity.so, CUDA for sm_103a).  PyTorch provides device memory and the
current CUDA stream; every step of the solver runs in the library's kernels.

    cav = Cavity(a=1, b=1, c=0.5, nx=256, ny=256, nz=128, precision="mixed")
    ap, field, iters, resid = cav.solve(kappa0, [(128, 1+0j)], theta, phi, alpha)
"""

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import CavityError

__all__ = ["Cavity", "CavityError"]


def _dptr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _layers(layers):
    lev = np.ascontiguousarray([int(l[0]) for l in layers], dtype=np.int32)
    er = np.ascontiguousarray([complex(l[1]).real for l in layers], dtype=np.float64)
    ei = np.ascontiguousarray([complex(l[1]).imag for l in layers], dtype=np.float64)
    return (lev, er, ei, lev.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            er.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            ei.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


_NOALLOC_PRECISION = {"fp64": _lib.CAVITY_FP64, "mixed": _lib.CAVITY_MIXED}


def check_operator_io(x, y, dtype, n_ap, device):
    """Argument checks of an operator call y = A x that writes through y's raw
    pointer: both tensors on `device`, of `dtype`, shaped (ndir, n_ap) alike,
    contiguous, and y not overlapping x.  Raises ValueError before anything
    reaches the library."""
    for name, t in (("x", x), ("y", y)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a tensor" % name)
        if t.device != device:
            raise ValueError("%s must be on %s, not %s" % (name, device, t.device))
        if t.dtype != dtype:
            raise ValueError("%s must be %s, not %s" % (name, dtype, t.dtype))
        if t.dim() != 2 or t.shape[1] != n_ap or t.shape[0] < 1:
            raise ValueError("%s must have shape (ndir, %d), not %s" % (name, n_ap,
                                                                        tuple(t.shape)))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if y.shape != x.shape:
        raise ValueError("y must have x's shape %s, not %s" % (tuple(x.shape), tuple(y.shape)))
    nb = x.numel() * x.element_size()
    x0, y0 = x.data_ptr(), y.data_ptr()
    if x0 < y0 + nb and y0 < x0 + nb:
        raise ValueError("y must not overlap x (the operator reads x while it writes y)")


def _angles(*arrays):
    """Host float64 copies of per-direction angle arrays, all of one length."""
    out = [_dptr(a) for a in arrays]
    if len({len(a) for a, _ in out}) != 1:
        raise ValueError("the per-direction angle arrays differ in length: %s"
                         % [len(a) for a, _ in out])
    return out


def check_out(name, t, shape, dtype, host, device):
    """Argument checks of an output tensor the library writes through its raw
    pointer: exactly `shape` and `dtype`, contiguous, and on the host (host
    True) or on `device`.  Raises ValueError."""
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s must be a tensor" % name)
    where = torch.device("cpu") if host else device
    if t.device != where:
        raise ValueError("%s must be on %s, not %s" % (name, where, t.device))
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError("%s must be %s of shape %s, not %s of shape %s" % (
            name, dtype, tuple(shape), t.dtype, tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def _overlap(s, t):
    s0, t0 = s.data_ptr(), t.data_ptr()
    return s0 < t0 + t.numel() * t.element_size() and t0 < s0 + s.numel() * s.element_size()


def check_lu_io(lu, ipiv, b, device):
    """Argument checks of an LU solve that writes b through its raw pointer:
    lu a contiguous square complex64 tensor, ipiv a contiguous int32 tensor of
    n entries, b a contiguous nrhs x n complex64 tensor, all on `device`, and b
    overlapping neither lu nor ipiv.  Raises ValueError before anything reaches
    the library (the library checks ipiv's values itself)."""
    for name, t in (("lu", lu), ("ipiv", ipiv), ("b", b)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a tensor" % name)
        if t.device != device:
            raise ValueError("%s must be on %s, not %s" % (name, device, t.device))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if lu.dtype != torch.complex64 or lu.dim() != 2 or lu.shape[0] != lu.shape[1] or \
            lu.shape[0] < 1:
        raise ValueError("lu must be a square complex64 tensor")
    n = lu.shape[0]
    if ipiv.dtype != torch.int32 or ipiv.dim() != 1 or ipiv.shape[0] != n:
        raise ValueError("ipiv must be an int32 tensor of %d entries" % n)
    if b.dtype != torch.complex64 or b.dim() != 2 or b.shape[1] != n or b.shape[0] < 1:
        raise ValueError("b must be an nrhs x %d complex64 tensor" % n)
    if _overlap(b, lu) or _overlap(b, ipiv):
        raise ValueError("b must not overlap lu or ipiv")


class Cavity:
    """One cavity geometry and grid with its resident device state."""

    def __init__(self, a, b, c, nx, ny, nz, precision="fp64", gmres_tol=0.0, gmres_restart=0,
                 gmres_max_iter=0, pivot_tol=0.0, stream=None, device=None,
                 khat_scheme="quadrature", modes_m=0, modes_n=0, aperture_solver="krylov",
                 outer_rule="trapezoid"):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.precision = _lib.CAVITY_FP64 if precision == "fp64" else _lib.CAVITY_MIXED
        d = _lib.CavityDesc(a, b, c, nx, ny, nz, self.precision, 0, gmres_tol, gmres_restart,
                            gmres_max_iter, pivot_tol,
                            {"quadrature": 0, "paper": 1}[khat_scheme], modes_m, modes_n,
                            _lib.SOLVERS[aperture_solver], _lib.OUTER_RULES[outer_rule])
        h = ctypes.c_void_p()
        st = self.lib.cavity_setup(ctypes.byref(d), ctypes.c_void_p(self.stream.cuda_stream),
                                   ctypes.byref(h))
        if st != 0:
            raise CavityError(st, self.lib.cavity_last_error(None).decode())
        self.h = h
        self.nx, self.ny, self.nz = nx, ny, nz
        n_ap = ctypes.c_longlong()
        fpd = ctypes.c_longlong()
        self.lib.cavity_sizes(self.h, ctypes.byref(n_ap), ctypes.byref(fpd))
        self.n_ap, self.field_per_dir = n_ap.value, fpd.value
        self.n1 = nx * (ny - 1)
        self.n2 = (nx - 1) * ny
        px, py = ctypes.c_int(), ctypes.c_int()
        self.lib.cavity_periods(self.h, ctypes.byref(px), ctypes.byref(py))
        self.pad_x, self.pad_y = px.value, py.value

    def _check(self, st, allow_noconv=False):
        if st == 0 or (allow_noconv and st == _lib.CAVITY_ENOCONV):
            return st
        raise CavityError(st, self.lib.cavity_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.cavity_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def field_dtype(self):
        return torch.complex128 if self.precision == _lib.CAVITY_FP64 else torch.complex64

    # ------------------------------------------------------------ hot path
    def prepare(self, kappa0, layers):
        lev, er, ei, pl, pr, pim = _layers(layers)
        self._check(self.lib.cavity_prepare(self.h, float(kappa0), len(lev), pl, pr, pim))

    def solve(self, kappa0, layers, theta, phi, alpha, field=True, host=False,
              aperture_out=None, field_out=None):
        """Aperture coefficients (ndir x n_ap complex128) and, if `field`, the
        interior field (ndir x field_per_dir), with per-direction Krylov
        iterations and relative residuals.  host=True returns pinned host
        tensors filled through the library's own device-to-host copies."""
        lev, er, ei, pl, pr, pim = _layers(layers)
        (th, pth), (ph, pph), (al, pal) = _angles(theta, phi, alpha)
        ndir = len(th)
        if host:
            ap = aperture_out if aperture_out is not None else torch.empty(
                (ndir, self.n_ap), dtype=torch.complex128, pin_memory=True)
            fl = None
            if field:
                fl = field_out if field_out is not None else torch.empty(
                    (ndir, self.field_per_dir), dtype=self.field_dtype, pin_memory=True)
        else:
            ap = aperture_out if aperture_out is not None else torch.empty(
                (ndir, self.n_ap), dtype=torch.complex128, device=self.device)
            fl = None
            if field:
                fl = field_out if field_out is not None else torch.empty(
                    (ndir, self.field_per_dir), dtype=self.field_dtype, device=self.device)
        check_out("aperture_out", ap, (ndir, self.n_ap), torch.complex128, host, self.device)
        if fl is not None:
            check_out("field_out", fl, (ndir, self.field_per_dir), self.field_dtype, host,
                      self.device)
            if _overlap(ap, fl):
                raise ValueError("aperture_out and field_out must not overlap")
        iters = np.zeros(ndir, dtype=np.int32)
        res = np.zeros(ndir, dtype=np.float64)
        st = self.lib.cavity_solve(
            self.h, float(kappa0), len(lev), pl, pr, pim, ndir, pth, pph, pal,
            _lib.CAVITY_OUT_FIELD if field else _lib.CAVITY_OUT_APERTURE,
            _lib.CAVITY_MEM_HOST if host else _lib.CAVITY_MEM_DEVICE,
            ctypes.c_void_p(ap.data_ptr()), ctypes.c_void_p(fl.data_ptr() if fl is not None else 0),
            iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        self.last_status = self._check(st, allow_noconv=True)
        return ap, fl, iters, res

    def rcs(self, aperture, theta, phi, pol="theta"):
        (th, pth), (ph, pph) = _angles(theta, phi)
        out = np.zeros(len(th))
        aperture = aperture.contiguous()
        if aperture.dtype != torch.complex128 or aperture.shape != (len(th), self.n_ap) or \
                (aperture.is_cuda and aperture.device != self.device):
            raise ValueError("aperture must be a (ndir, n_ap) complex128 tensor on the host "
                             "or on %s" % self.device)
        mem = _lib.CAVITY_MEM_DEVICE if aperture.is_cuda else _lib.CAVITY_MEM_HOST
        self._check(self.lib.cavity_rcs(
            self.h, len(th), ctypes.c_void_p(aperture.data_ptr()), mem, pth, pph,
            _lib.CAVITY_POL_THETA if pol == "theta" else _lib.CAVITY_POL_PHI,
            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    # ------------------------------------------------------------ step level
    def rhs(self, theta, phi, alpha):
        (th, pth), (ph, pph), (al, pal) = _angles(theta, phi, alpha)
        out = torch.empty((len(th), self.n_ap), dtype=torch.complex128, device=self.device)
        self._check(self.lib.cavity_rhs(self.h, len(th), pth, pph, pal, ctypes.c_void_p(out.data_ptr())))
        return out

    def apply(self, x, precision=None):
        """y = A x.  precision: None (the context's), "fp64", "mixed" (FP32
        operator, complex64 vectors) or "pair32" (pair-of-FP32 arithmetic,
        complex128 vectors: the residual operator of the mixed solve)."""
        prec = self.precision if precision is None else {
            "fp64": _lib.CAVITY_FP64, "mixed": _lib.CAVITY_MIXED,
            "pair32": _lib.CAVITY_PAIR32}[precision]
        x = x.contiguous()
        want = torch.complex64 if prec == _lib.CAVITY_MIXED else torch.complex128
        if x.dtype != want or x.device != self.device or x.dim() != 2 or \
                x.shape[1] != self.n_ap:
            raise ValueError("x must be a (ndir, n_ap) tensor of %s on %s" % (want, self.device))
        y = torch.empty_like(x)
        self._check(self.lib.cavity_apply(self.h, x.shape[0], prec, ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(y.data_ptr())))
        return y

    def apply_noalloc(self, x, precision=None, y=None):
        """y = A x through the allocation-free entry point: the library uses
        its own fixed scratch array and allocates nothing.  precision: None
        (the context's), "fp64" (complex128 vectors) or "mixed" (FP32
        operator, complex64 vectors); the pair-of-FP32 operator has no
        allocation-free form.  y, if given, must be a contiguous CUDA tensor
        of x's shape and dtype on the context's device that does not overlap
        x; otherwise a new tensor is returned (allocated here by torch, not
        by the library)."""
        if precision is None:
            prec = self.precision
        elif precision in _NOALLOC_PRECISION:
            prec = _NOALLOC_PRECISION[precision]
        else:
            raise ValueError("apply_noalloc precision must be 'fp64' or 'mixed', not %r"
                             % (precision,))
        want = torch.complex128 if prec == _lib.CAVITY_FP64 else torch.complex64
        if self.device.type != "cuda":
            raise ValueError("apply_noalloc needs a CUDA context")
        x = x.contiguous()
        if y is None:
            y = torch.empty_like(x)
        check_operator_io(x, y, want, self.n_ap, self.device)
        self._check(self.lib.cavity_apply_noalloc(self.h, x.shape[0], prec,
                                                  ctypes.c_void_p(x.data_ptr()),
                                                  ctypes.c_void_p(y.data_ptr())))
        return y

    def field(self, aperture):
        aperture = aperture.contiguous()
        if aperture.dtype != torch.complex128 or aperture.device != self.device or \
                aperture.dim() != 2 or aperture.shape[1] != self.n_ap:
            raise ValueError("aperture must be a (ndir, n_ap) complex128 tensor on %s"
                             % self.device)
        out = torch.empty((aperture.shape[0], self.field_per_dir), dtype=self.field_dtype,
                          device=self.device)
        self._check(self.lib.cavity_field(self.h, aperture.shape[0],
                                          ctypes.c_void_p(aperture.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr())))
        return out

    def export_elimination(self):
        top = torch.empty(self.n_ap + self.n1 + self.n2, dtype=torch.complex128, device=self.device)
        prof = torch.empty((self.nz - 1, self.n_ap), dtype=torch.complex128, device=self.device)
        profq = torch.empty((self.nz - 1, self.n1 + self.n2), dtype=torch.complex128,
                            device=self.device)
        self._check(self.lib.cavity_export_elimination(
            self.h, ctypes.c_void_p(top.data_ptr()), ctypes.c_void_p(prof.data_ptr()),
            ctypes.c_void_p(profq.data_ptr())))
        return top, prof, profq

    def export_khat(self):
        out = torch.empty((self.pad_x * self.nx // 2, self.pad_y * self.ny // 2), dtype=torch.complex128,
                          device=self.device)
        self._check(self.lib.cavity_export_khat(self.h, ctypes.c_void_p(out.data_ptr())))
        return out

    # ------------------------------------------------------------ dense solve steps
    def dense_size(self):
        """Number of kept unknowns (rows of the kept block)."""
        n = ctypes.c_int()
        self._check(self.lib.cavity_dense_size(self.h, ctypes.byref(n)))
        return n.value

    def dense_assemble(self):
        """The kept block of the aperture matrix (after prepare) as an n x n
        complex64 device tensor."""
        n = self.dense_size()
        a = torch.empty((n, n), dtype=torch.complex64, device=self.device)
        self._check(self.lib.cavity_dense_assemble(self.h, ctypes.c_void_p(a.data_ptr()), n))
        return a

    def lu_factor(self, a):
        """In-place LU with partial pivoting of the square complex64 device
        tensor a (row-major); returns (ipiv, info) with ipiv an int32 device
        tensor of row exchanges (info -1 unless a pivot column was zero)."""
        if a.dtype != torch.complex64 or a.dim() != 2 or a.shape[0] != a.shape[1] or \
                not a.is_contiguous() or a.device != self.device:
            raise ValueError("a must be a contiguous square complex64 tensor on %s" % self.device)
        n = a.shape[0]
        ipiv = torch.empty(n, dtype=torch.int32, device=self.device)
        info = ctypes.c_int(-1)
        st = self.lib.cavity_lu_factor(self.h, ctypes.c_void_p(a.data_ptr()), n, n,
                                       ctypes.c_void_p(ipiv.data_ptr()), ctypes.byref(info))
        if st not in (0, _lib.CAVITY_ESINGULAR):
            self._check(st)
        return ipiv, info.value

    def lu_solve(self, lu, ipiv, b):
        """Solve with lu_factor's output for the rows of b (nrhs x n
        complex64 device tensor, overwritten and returned)."""
        check_lu_io(lu, ipiv, b, self.device)
        n = lu.shape[0]
        self._check(self.lib.cavity_lu_solve(self.h, ctypes.c_void_p(lu.data_ptr()), n, n,
                                             ctypes.c_void_p(ipiv.data_ptr()), b.shape[0],
                                             ctypes.c_void_p(b.data_ptr()), n))
        return b

    # ------------------------------------------------------------ options
    def set_option(self, name, value):
        """Implementation option (include/cavity.h, CAVITY_OPT_*): "pass_b_2048",
        "pass_c_2048" (0 warp pairs, 1 block transform), "group_width"
        (1..16 directions per block Krylov group), "coarse_modes" (0, or
        mc > 0: the mixed solve's two-level preconditioner with the exact
        solve of the modes m, n <= mc as its coarse level) or "field_fused"
        (complex64 field synthesis: 0 the default per grid, 1 the fused
        kernel where the grid allows it, 2 the two passes)."""
        self._check(self.lib.cavity_set_option(self.h, _lib.OPTIONS[name], int(value)))

    def get_option(self, name):
        v = ctypes.c_int()
        self._check(self.lib.cavity_get_option(self.h, _lib.OPTIONS[name], ctypes.byref(v)))
        return v.value

    # ------------------------------------------------------------ instrumentation
    def timing(self, enable=True):
        """Reset launch counters; with enable, time every launch with events."""
        self._check(self.lib.cavity_timing(self.h, 1 if enable else 0))

    def timing_read(self):
        """{class name: (ms, launches)} since the last timing() call."""
        n = _lib.NUM_KCLASS
        ms = np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        self._check(self.lib.cavity_timing_read(
            self.h, n, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))))
        return {self.lib.cavity_kernel_class(k).decode(): (float(ms[k]), int(cnt[k]))
                for k in range(n)}
