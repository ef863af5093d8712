"""ctypes declarations of the C ABI in include/cavity.h.

Loading fails loudly when the library has not been built: there is no other
implementation of the solver in this package.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcavity.so")

CAVITY_OK, CAVITY_EINVAL, CAVITY_ENOMEM, CAVITY_ESINGULAR, CAVITY_ENOCONV, CAVITY_ETIMEOUT, \
    CAVITY_ECUDA = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ESINGULAR", 4: "ENOCONV", 5: "ETIMEOUT",
                6: "ECUDA"}
CAVITY_FP64, CAVITY_MIXED, CAVITY_PAIR32 = 0, 1, 2
CAVITY_OUT_APERTURE, CAVITY_OUT_FIELD = 0, 1
CAVITY_MEM_DEVICE, CAVITY_MEM_HOST = 0, 1
CAVITY_POL_THETA, CAVITY_POL_PHI = 0, 1

# every entry point that include/cavity.h declares
EXPORTS = ["cavity_setup", "cavity_prepare", "cavity_solve", "cavity_rcs", "cavity_destroy",
           "cavity_last_error", "cavity_sizes", "cavity_export_elimination",
           "cavity_export_khat", "cavity_rhs", "cavity_apply", "cavity_field",
           "cavity_timing", "cavity_timing_read", "cavity_kernel_class",
           "cavity_apply_noalloc", "cavity_set_option", "cavity_get_option",
           "cavity_dense_size", "cavity_dense_assemble", "cavity_lu_factor", "cavity_lu_solve",
           "cavity_periods"]
CAVITY_SOLVER_KRYLOV, CAVITY_SOLVER_DENSE = 0, 1
SOLVERS = {"krylov": CAVITY_SOLVER_KRYLOV, "dense": CAVITY_SOLVER_DENSE}
OUTER_RULES = {"trapezoid": 0, "parseval": 1}
DENSE_MAX_N = 16384
CAVITY_OPT_PASS_B_2048, CAVITY_OPT_PASS_C_2048, CAVITY_OPT_GROUP_WIDTH, \
    CAVITY_OPT_COARSE_MODES, CAVITY_OPT_FIELD_FUSED = range(5)
OPTIONS = {"pass_b_2048": CAVITY_OPT_PASS_B_2048, "pass_c_2048": CAVITY_OPT_PASS_C_2048,
           "group_width": CAVITY_OPT_GROUP_WIDTH, "coarse_modes": CAVITY_OPT_COARSE_MODES,
           "field_fused": CAVITY_OPT_FIELD_FUSED}
NUM_KCLASS = 24


class CavityDesc(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("precision", ctypes.c_int), ("pad_factor", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("gmres_restart", ctypes.c_int),
                ("gmres_max_iter", ctypes.c_int), ("pivot_tol", ctypes.c_double),
                ("khat_scheme", ctypes.c_int), ("modes_m", ctypes.c_int), ("modes_n", ctypes.c_int),
                ("aperture_solver", ctypes.c_int), ("outer_rule", ctypes.c_int)]


class CavityError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def load():
    """Load libcavity.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError("libcavity.so is not built (run __graft_entry__.build() or "
                      "python paper_2008_01966_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    pd = ctypes.POINTER(ctypes.c_double)
    pi = ctypes.POINTER(ctypes.c_int)
    pll = ctypes.POINTER(ctypes.c_longlong)
    lib.cavity_setup.argtypes = [ctypes.POINTER(CavityDesc), P, ctypes.POINTER(P)]
    lib.cavity_prepare.argtypes = [P, D, I, pi, pd, pd]
    lib.cavity_solve.argtypes = [P, D, I, pi, pd, pd, I, pd, pd, pd, I, I, P, P, pi, pd]
    lib.cavity_rcs.argtypes = [P, I, P, I, pd, pd, I, pd]
    lib.cavity_destroy.argtypes = [P]
    lib.cavity_destroy.restype = None
    lib.cavity_last_error.argtypes = [P]
    lib.cavity_last_error.restype = ctypes.c_char_p
    lib.cavity_sizes.argtypes = [P, pll, pll]
    lib.cavity_export_elimination.argtypes = [P, P, P, P]
    lib.cavity_export_khat.argtypes = [P, P]
    lib.cavity_rhs.argtypes = [P, I, pd, pd, pd, P]
    lib.cavity_apply.argtypes = [P, I, I, P, P]
    lib.cavity_field.argtypes = [P, I, P, P]
    lib.cavity_apply_noalloc.argtypes = [P, I, I, P, P]
    lib.cavity_set_option.argtypes = [P, I, I]
    lib.cavity_get_option.argtypes = [P, I, ctypes.POINTER(I)]
    lib.cavity_periods.argtypes = [P, pi, pi]
    lib.cavity_dense_size.argtypes = [P, pi]
    lib.cavity_dense_assemble.argtypes = [P, P, I]
    lib.cavity_lu_factor.argtypes = [P, P, I, I, P, pi]
    lib.cavity_lu_solve.argtypes = [P, P, I, I, P, I, P, I]
    lib.cavity_timing.argtypes = [P, I]
    lib.cavity_timing_read.argtypes = [P, I, pd, pll]
    lib.cavity_kernel_class.argtypes = [I]
    lib.cavity_kernel_class.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("cavity_destroy", "cavity_last_error", "cavity_kernel_class"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib
