"""ctypes declarations of the C ABI in include/recon.h (argument marshalling
only: every step of the solve runs in librecon.so's CUDA kernels)."""
import ctypes as C
import os

from . import build as _build

RECON_OK, RECON_NOT_CONVERGED, RECON_STALLED = 0, 1, 2
RECON_E_INVALID, RECON_E_OOM, RECON_E_CUDA, RECON_E_NONFINITE = -1, -2, -3, -4
RECON_E_LIMITER, RECON_E_TIMEOUT, RECON_E_STATE, RECON_E_UNSUPPORTED = -5, -6, -7, -8
RECON_FP64, RECON_MIXED = 0, 1
RECON_CLIM_SOFT, RECON_CLIM_LITERAL, RECON_CLIM_STEP = 0, 1, 2
RECON_PARTICLES, RECON_GRID = 0, 1
FIELDS = {"phi": 0, "delta_r": 1, "mesh_x": 2, "mass": 3, "det": 4, "lambda0": 5, "density": 6}

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)

# Every function the header declares, with (restype, argtypes).
SYMBOLS = {
    "recon_default_params": (C.c_int, None),
    "recon_resolve_params": (C.c_int, None),
    "recon_create": (C.c_int, None),
    "recon_deposit": (C.c_int, None),
    "recon_solve": (C.c_int, None),
    "recon_solve_batch": (C.c_int, None),
    "recon_field": (C.c_int, None),
    "recon_adjoint": (C.c_int, None),
    "recon_destroy": (None, None),
    "recon_last_error": (C.c_char_p, None),
    "recon_deposit_cic_noalloc": (C.c_int, None),
}


class recon_params(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3), ("box", C.c_double * 3), ("precision", C.c_int),
        ("xi_m", C.c_double), ("v_m", C.c_double), ("a_min", C.c_double),
        ("climiter", C.c_int), ("s_side", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
        ("tol_in", C.c_double), ("max_vcycles", C.c_int), ("tol_out", C.c_double),
        ("k_max", C.c_int), ("d_max", C.c_double), ("alpha_min", C.c_double),
        ("lambda_floor", C.c_double), ("replay_alpha", _D), ("profile", C.c_int),
        ("inner_vcycles", C.c_int), ("density_update", C.c_int), ("device_loop", C.c_int),
        ("checkpoint", C.c_int), ("stream_planes", C.c_int), ("restrict_planes", C.c_int),
        ("coarse_faces", C.c_int), ("tune_inner", C.c_int), ("group_max", C.c_int),
        ("tma", C.c_int), ("warm_start", C.c_int),
    ]


class recon_stats(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("steps", C.c_int), ("vcycles", C.c_int), ("R0", C.c_double),
        ("R", C.c_double), ("min_det", C.c_double), ("min_lambda0", C.c_double),
        ("max_delta_r", C.c_double), ("mass_error", C.c_double), ("ms", C.c_double),
        ("alpha", _D), ("Rk", _D), ("ncycles", _I), ("relres", _D),
        ("launches", C.c_longlong), ("smooth_ms", C.c_double), ("smooth_sweeps", C.c_int),
        ("smooth_bytes", C.c_double), ("inner_vcycles", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
    ]


_lib = None


def _checked() -> bool:
    """RECON_BUILD=checked selects the bounds-checked library."""
    return os.environ.get("RECON_BUILD", "") == "checked"


def lib_path():
    return _build.lib_path(_checked())


def load(build_if_missing: bool = True):
    """Load librecon.so, or librecon_checked.so under RECON_BUILD=checked
    (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    checked = _checked()
    path = _build.build(checked=checked) if build_if_missing else _build.lib_path(checked)
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not built at {path}")
    lib = C.CDLL(path)
    lib.recon_default_params.restype = C.c_int
    lib.recon_default_params.argtypes = [C.POINTER(recon_params), C.c_int, C.c_int, C.c_int]
    lib.recon_resolve_params.restype = C.c_int
    lib.recon_resolve_params.argtypes = [C.POINTER(recon_params)]
    lib.recon_create.restype = C.c_int
    lib.recon_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(recon_params), C.c_void_p]
    lib.recon_deposit.restype = C.c_int
    lib.recon_deposit.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int64]
    lib.recon_solve.restype = C.c_int
    lib.recon_solve.argtypes = [C.c_void_p, C.POINTER(recon_stats)]
    lib.recon_solve_batch.restype = C.c_int
    lib.recon_solve_batch.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(recon_stats)]
    lib.recon_field.restype = C.c_int
    lib.recon_field.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]
    lib.recon_adjoint.restype = C.c_int
    lib.recon_adjoint.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.recon_destroy.restype = None
    lib.recon_destroy.argtypes = [C.c_void_p]
    lib.recon_last_error.restype = C.c_char_p
    lib.recon_last_error.argtypes = []
    lib.recon_deposit_cic_noalloc.restype = C.c_int
    lib.recon_deposit_cic_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p,
                                              C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    _lib = lib
    return lib


def last_error() -> str:
    return load().recon_last_error().decode(errors="replace")


class ReconError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where} failed with status {status}: {last_error()}")


def check(status, where):
    if status < 0:
        raise ReconError(status, where)
    return status
