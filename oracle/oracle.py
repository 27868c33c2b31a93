"""ctypes wrapper of the C oracle (oracle/recon_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's
CPU-baseline leg.  Arrays are numpy float64, C order, grid units, masses in
units of the mean density.  Every function mirrors the C function of the same
name; see recon_oracle.h for the paper passage each step follows.
"""
import ctypes as C
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from .build import build

__all__ = [
    "OracleParams", "CLIM_SOFT", "CLIM_LITERAL", "CLIM_STEP", "cic_deposit", "apply_L",
    "rbgs_sweep", "restrict", "prolong_add", "apply_S", "vcycle", "mg_solve", "geometry",
    "source", "step_limiter", "advance", "solve", "delta_r", "mesh_x", "min_eig_sym3", "mass_change",
    "coarse_dims", "levels", "adjoint", "set_threads",
]

CLIM_SOFT, CLIM_LITERAL, CLIM_STEP = 0, 1, 2

_lib = None
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


class _Params(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3), ("xi_m", C.c_double), ("v_m", C.c_double), ("a_min", C.c_double),
        ("climiter", C.c_int), ("s_side", C.c_double),
        ("nu1", C.c_int), ("nu2", C.c_int), ("tol_in", C.c_double), ("max_vcycles", C.c_int),
        ("tol_out", C.c_double), ("k_max", C.c_int), ("d_max", C.c_double),
        ("alpha_min", C.c_double), ("lambda_floor", C.c_double), ("density_update", C.c_int),
        ("warm_start", C.c_int),
    ]


class _Trace(C.Structure):
    _fields_ = [("alpha", _D), ("R", _D), ("ncycles", _I), ("relres", _D), ("min_det", _D),
                ("min_lam", _D), ("mass", _D)]


@dataclass
class OracleParams:
    """Parameters of the solve; defaults are the readings of App. A stated in
    the oracle header (xi_m = 1/10, v_m = 10, S = (1/4, 1/2, 1/4) per axis,
    V(2,2) cycles, 1e-8 relative inner tolerance)."""
    n: Sequence[int] = (32, 32, 32)
    xi_m: float = 0.1
    v_m: float = 10.0
    a_min: float = 0.01
    climiter: int = CLIM_SOFT
    s_side: float = 0.25
    nu1: int = 2
    nu2: int = 2
    tol_in: float = 1e-8
    max_vcycles: int = 50
    tol_out: float = 1e-3
    k_max: int = 200
    d_max: float = 0.5
    alpha_min: float = 2.0 ** -20
    lambda_floor: float = 0.01
    density_update: int = 0
    warm_start: int = 2

    def _c(self) -> _Params:
        p = _Params()
        p.n[:] = [int(v) for v in self.n]
        for f in ("xi_m", "v_m", "a_min", "climiter", "s_side", "nu1", "nu2",
                  "tol_in", "max_vcycles", "tol_out", "k_max", "d_max", "alpha_min",
                  "lambda_floor", "density_update", "warm_start"):
            setattr(p, f, getattr(self, f))
        return p


def _load():
    """Load (building if needed) the oracle library.  It runs one thread unless
    ORACLE_THREADS or set_threads() asks for more; idle threads sleep instead
    of spinning, so a busy host is not slowed further."""
    global _lib
    if _lib is None:
        import os

        os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
        _lib = C.CDLL(build())
        _lib.orc_set_threads(C.c_int(int(os.environ.get("ORACLE_THREADS", "1"))))
        for name in ("orc_cic_deposit", "orc_apply_L", "orc_rbgs_sweep", "orc_restrict",
                     "orc_prolong_add", "orc_apply_S", "orc_vcycle", "orc_mg_solve",
                     "orc_geometry", "orc_source", "orc_step_limiter", "orc_advance",
                     "orc_solve", "orc_delta_r", "orc_mesh_x", "orc_mass_change", "orc_adjoint"):
            getattr(_lib, name).restype = C.c_int
        _lib.orc_min_eig_sym3.restype = C.c_double
        _lib.orc_set_threads.restype = C.c_int
    return _lib


def set_threads(nthreads=0):
    """Threads of the plane-split loops (OpenMP build; the results do not
    depend on it).  nthreads > 0 sets the count; returns the count in use."""
    return int(_load().orc_set_threads(C.c_int(int(nthreads))))


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _n3(n):
    return (C.c_int * 3)(*[int(v) for v in n])


def _h3(h):
    return (C.c_double * 3)(*[float(v) for v in h])


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")
    return rc


def coarse_dims(n):
    """Dims of the next multigrid level: axes longer than 4 are halved."""
    return tuple(v // 2 if v > 4 else v for v in n)


def levels(n):
    """(dims, spacing) of every multigrid level, finest first."""
    out, h = [(tuple(n), (1.0, 1.0, 1.0))], [1.0, 1.0, 1.0]
    while any(v > 4 for v in out[-1][0]):
        d = out[-1][0]
        h = [hh * 2 if v > 4 else hh for hh, v in zip(h, d)]
        out.append((coarse_dims(d), tuple(h)))
    return out


def cic_deposit(n, x, w=None):
    x = _f64(x).reshape(-1, 3)
    w = None if w is None else _f64(w)
    out = np.empty(tuple(n))
    _check(_load().orc_cic_deposit(_n3(n), _dp(x), _dp(w), C.c_int64(x.shape[0]), _dp(out)),
           "cic_deposit")
    return out


def apply_L(a, u, h=(1.0, 1.0, 1.0)):
    a, u = _f64(a), _f64(u)
    out = np.empty_like(u)
    _check(_load().orc_apply_L(_n3(u.shape), _h3(h), _dp(a), _dp(u), _dp(out)), "apply_L")
    return out


def rbgs_sweep(a, f, u, h=(1.0, 1.0, 1.0)):
    a, f, u = _f64(a), _f64(f), _f64(u).copy()
    _check(_load().orc_rbgs_sweep(_n3(u.shape), _h3(h), _dp(a), _dp(f), _dp(u)), "rbgs_sweep")
    return u


def restrict(fine):
    fine = _f64(fine)
    out = np.empty(coarse_dims(fine.shape))
    _check(_load().orc_restrict(_n3(fine.shape), _dp(fine), _dp(out)), "restrict")
    return out


def prolong_add(coarse, fine):
    coarse, fine = _f64(coarse), _f64(fine).copy()
    _check(_load().orc_prolong_add(_n3(fine.shape), _dp(coarse), _dp(fine)), "prolong_add")
    return fine


def apply_S(u, s_side=0.25):
    u = _f64(u)
    out = np.empty_like(u)
    _check(_load().orc_apply_S(_n3(u.shape), C.c_double(s_side), _dp(u), _dp(out)), "apply_S")
    return out


def vcycle(params: OracleParams, a, f, u):
    a, f, u = _f64(a), _f64(f), _f64(u).copy()
    p = params._c()
    _check(_load().orc_vcycle(C.byref(p), _dp(a), _dp(f), _dp(u)), "vcycle")
    return u


def mg_solve(params: OracleParams, a, s):
    a, s = _f64(a), _f64(s)
    u = np.empty_like(s)
    nc, rel = C.c_int(0), C.c_double(0.0)
    p = params._c()
    _check(_load().orc_mg_solve(C.byref(p), _dp(a), _dp(s), _dp(u), C.byref(nc), C.byref(rel)),
           "mg_solve")
    return u, nc.value, rel.value


def geometry(phi):
    phi = _f64(phi)
    g, lam = np.empty_like(phi), np.empty_like(phi)
    _check(_load().orc_geometry(_n3(phi.shape), _dp(phi), _dp(g), _dp(lam)), "geometry")
    return g, lam


def source(params: OracleParams, phi, m):
    phi, m = _f64(phi), _f64(m)
    s, t = np.empty_like(phi), np.empty_like(phi)
    p = params._c()
    _check(_load().orc_source(C.byref(p), _dp(phi), _dp(m), _dp(s), _dp(t)), "source")
    return s, t


def step_limiter(params: OracleParams, phi, dphi):
    phi, dphi = _f64(phi), _f64(dphi)
    al = C.c_double(0.0)
    p = params._c()
    rc = _load().orc_step_limiter(C.byref(p), _dp(phi), _dp(dphi), C.byref(al))
    if rc == -5:
        return None
    _check(rc, "step_limiter")
    return al.value


def advance(alpha, dphi, phi, xi):
    dphi, phi, xi = _f64(dphi), _f64(phi).copy(), _f64(xi).reshape(-1, 3).copy()
    _check(_load().orc_advance(_n3(phi.shape), C.c_double(alpha), _dp(dphi), _dp(phi), _dp(xi),
                               C.c_int64(xi.shape[0])), "advance")
    return phi, xi


def mass_change(phi, m, v):
    phi, m, v = _f64(phi), _f64(m), _f64(v)
    out = np.empty_like(phi)
    _check(_load().orc_mass_change(_n3(phi.shape), _dp(phi), _dp(m), _dp(v), _dp(out)),
           "mass_change")
    return out


def delta_r(phi):
    phi = _f64(phi)
    out = np.empty_like(phi)
    _check(_load().orc_delta_r(_n3(phi.shape), _dp(phi), _dp(out)), "delta_r")
    return out


def mesh_x(phi):
    phi = _f64(phi)
    out = np.empty(phi.shape + (3,))
    _check(_load().orc_mesh_x(_n3(phi.shape), _dp(phi), _dp(out)), "mesh_x")
    return out


def min_eig_sym3(A):
    A = _f64(A)
    return _load().orc_min_eig_sym3((C.c_double * 9)(*A.ravel().tolist()))


@dataclass
class SolveResult:
    status: int
    steps: int
    phi: np.ndarray
    xi: np.ndarray
    m: np.ndarray
    alpha: np.ndarray = field(default=None)
    R: np.ndarray = field(default=None)
    ncycles: np.ndarray = field(default=None)
    relres: np.ndarray = field(default=None)
    min_det: np.ndarray = field(default=None)
    min_lam: np.ndarray = field(default=None)
    mass: np.ndarray = field(default=None)


def solve(params: OracleParams, rho, replay_alpha=None) -> SolveResult:
    """Whole moving-mesh solve (Sec. II, App. A) on a density grid rho."""
    rho = _f64(rho)
    assert tuple(rho.shape) == tuple(params.n)
    K = max(int(params.k_max), 1)
    phi, xi, m = np.empty_like(rho), np.empty(rho.shape + (3,)), np.empty_like(rho)
    arrs = {k: np.zeros(K) for k in ("alpha", "R", "relres", "min_det", "min_lam", "mass")}
    ncyc = np.zeros(K, dtype=np.int32)
    tr = _Trace(_dp(arrs["alpha"]), _dp(arrs["R"]), ncyc.ctypes.data_as(_I), _dp(arrs["relres"]),
                _dp(arrs["min_det"]), _dp(arrs["min_lam"]), _dp(arrs["mass"]))
    ra = None if replay_alpha is None else _f64(replay_alpha)
    steps = C.c_int(0)
    p = params._c()
    rc = _check(_load().orc_solve(C.byref(p), _dp(rho), _dp(ra), _dp(phi), _dp(xi), _dp(m),
                                  C.byref(steps), C.byref(tr)), "solve")
    k = steps.value
    nrec = min(k + 1, K)
    return SolveResult(rc, k, phi, xi, m, arrs["alpha"][:k], arrs["R"][:nrec], ncyc[:k],
                       arrs["relres"][:k], arrs["min_det"][:nrec], arrs["min_lam"][:nrec],
                       arrs["mass"][:nrec])


def adjoint(params: OracleParams, rho, alpha, gbar):
    """dL/d rho from gbar = dL/d delta_r for the solve's len(alpha) advances
    with those step lengths held fixed (orc_adjoint)."""
    rho = _f64(rho)
    assert tuple(rho.shape) == tuple(params.n)
    al = _f64(np.asarray(alpha, dtype=np.float64).reshape(-1))
    g = _f64(gbar)
    out = np.empty_like(rho)
    p = params._c()
    _check(_load().orc_adjoint(C.byref(p), _dp(rho), _dp(al) if al.size else None, int(al.size),
                               _dp(g), _dp(out)), "adjoint")
    return out
