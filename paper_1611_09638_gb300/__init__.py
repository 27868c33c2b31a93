"""GB300 (sm_103a) nonlinear reconstruction: the displacement-potential solve of
Zhu, Yu, Pen, Chen & Yu 2016 (arXiv:1611.09638) behind the C ABI of
include/recon.h.

``Recon`` is a thin wrapper: it marshals torch tensors (device memory, the
current CUDA stream) into librecon.so calls; every step of the solve runs in
the library's CUDA kernels.  There is no CPU path: without the compiled library
or a CUDA device the calls raise.
"""
import ctypes as C
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import _abi
from ._abi import (RECON_FP64, RECON_MIXED, RECON_OK, RECON_NOT_CONVERGED, ReconError,  # noqa: F401
                   FIELDS)

__all__ = ["Recon", "SolveStats", "default_params", "resolved_params", "solve_batch", "reconstruct", "RECON_FP64", "RECON_MIXED", "ReconError"]


def default_params(n, box=None, precision="fp64", **overrides):
    """recon_params filled by recon_default_params, then overridden."""
    lib = _abi.load()
    p = _abi.recon_params()
    _abi.check(lib.recon_default_params(C.byref(p), int(n[0]), int(n[1]), int(n[2])),
               "recon_default_params")
    if box is not None:
        b = [float(box)] * 3 if np.isscalar(box) else [float(v) for v in box]
        p.box[:] = b
    p.precision = {"fp64": RECON_FP64, "mixed": RECON_MIXED}[precision]
    for k, v in overrides.items():
        if k == "replay_alpha":
            continue
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def resolved_params(n, box=None, precision="fp64", **overrides):
    """default_params with the multigrid settings left at -1 replaced by the
    values recon_create uses for the precision (recon_resolve_params)."""
    p = default_params(n, box=box, precision=precision, **overrides)
    _abi.check(_abi.load().recon_resolve_params(C.byref(p)), "recon_resolve_params")
    return p


@dataclass
class SolveStats:
    status: int
    steps: int
    vcycles: int
    R0: float
    R: float
    min_det: float
    min_lambda0: float
    max_delta_r: float
    mass_error: float
    ms: float
    launches: int = 0
    smooth_ms: float = 0.0
    smooth_sweeps: int = 0
    smooth_bytes: float = 0.0
    inner_vcycles: int = 0
    nu1: int = 0
    nu2: int = 0
    alpha: np.ndarray = field(default=None)
    Rk: np.ndarray = field(default=None)
    ncycles: np.ndarray = field(default=None)
    relres: np.ndarray = field(default=None)


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (C-contiguous float64)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous() and str(x.dtype) == "torch.float64", "need contiguous float64"
        return C.c_void_p(x.data_ptr())
    assert x.dtype == np.float64 and x.flags.c_contiguous, "need contiguous float64"
    return C.c_void_p(x.ctypes.data)


class Recon:
    """One solver handle for an n[0] x n[1] x n[2] periodic grid of side box."""

    def __init__(self, n, box=None, precision="fp64", stream=None, replay_alpha=None, **params):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_1611_09638_gb300 needs a CUDA device (no CPU path)")
        self._lib = _abi.load()
        self.n = tuple(int(v) for v in n)
        self.cells = int(np.prod(self.n))
        self.params = default_params(self.n, box, precision, **params)
        self._replay = None
        if replay_alpha is not None:
            ra = np.zeros(self.params.k_max)
            ra[:len(replay_alpha)] = replay_alpha
            self._replay = np.ascontiguousarray(ra, dtype=np.float64)
            self.params.replay_alpha = self._replay.ctypes.data_as(C.POINTER(C.c_double))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _abi.check(self._lib.recon_create(C.byref(h), C.byref(self.params),
                                          C.c_void_p(self.stream.cuda_stream)), "recon_create")
        self._h = h

    # -- inputs ------------------------------------------------------------
    def deposit_particles(self, pos, mass=None):
        """Grid particles (np x 3 positions in box units; host or device)."""
        n_p = int(pos.shape[0])
        return _abi.check(self._lib.recon_deposit(self._h, _abi.RECON_PARTICLES, _ptr(pos),
                                                  _ptr(mass), n_p), "recon_deposit")

    def deposit_grid(self, rho):
        """Take a density grid (host or device, n cells, float64)."""
        return _abi.check(self._lib.recon_deposit(self._h, _abi.RECON_GRID, _ptr(rho), None,
                                                  int(np.prod(rho.shape))), "recon_deposit")

    # -- solve -------------------------------------------------------------
    def _stats_record(self, st, record):
        """Attach per-step host arrays of length k_max to a recon_stats."""
        K = max(int(self.params.k_max), 1)
        arrs = {}
        if record:
            for k in ("alpha", "Rk", "relres"):
                arrs[k] = np.zeros(K)
                setattr(st, k, arrs[k].ctypes.data_as(C.POINTER(C.c_double)))
            arrs["ncycles"] = np.zeros(K, dtype=np.int32)
            st.ncycles = arrs["ncycles"].ctypes.data_as(C.POINTER(C.c_int))
        return arrs

    def _stats_out(self, rc, st, arrs, record):
        K = max(int(self.params.k_max), 1)
        k = st.steps
        out = SolveStats(rc, k, st.vcycles, st.R0, st.R, st.min_det, st.min_lambda0,
                         st.max_delta_r, st.mass_error, st.ms, st.launches, st.smooth_ms,
                         st.smooth_sweeps, st.smooth_bytes, st.inner_vcycles, st.nu1, st.nu2)
        if record:
            out.alpha, out.ncycles, out.relres = arrs["alpha"][:k], arrs["ncycles"][:k], arrs["relres"][:k]
            stopped = rc in (RECON_OK, _abi.RECON_STALLED)
            out.Rk = arrs["Rk"][:min(k + 1, K)] if stopped else arrs["Rk"][:k]
        return out

    def solve(self, record=True) -> SolveStats:
        st = _abi.recon_stats()
        arrs = self._stats_record(st, record)
        rc = self._lib.recon_solve(self._h, C.byref(st))
        _abi.check(rc, "recon_solve")
        return self._stats_out(rc, st, arrs, record)

    # -- outputs -----------------------------------------------------------
    def field(self, which, out=None):
        """Copy an output field into ``out`` (a float64 tensor or array, host or
        device) or into a new device tensor."""
        import torch

        code = FIELDS[which]
        shape = self.n + (3,) if which == "mesh_x" else self.n
        if out is None:
            out = torch.empty(shape, dtype=torch.float64, device="cuda")
        nbytes = int(np.prod(shape)) * 8
        _abi.check(self._lib.recon_field(self._h, code, _ptr(out), nbytes), "recon_field")
        return out

    def adjoint(self, grad_delta_r, grad_rho=None):
        """dL/d rho of the last solve from dL/d delta_r (recon_adjoint; the
        handle needs checkpoint=1).  Returns grad_rho (a new device tensor if
        none is given)."""
        import torch

        if grad_rho is None:
            grad_rho = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _abi.check(self._lib.recon_adjoint(self._h, _ptr(grad_delta_r), _ptr(grad_rho)),
                   "recon_adjoint")
        return grad_rho

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.recon_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve_batch(recons, record=True):
    """Solve several independent problems at once (recon_solve_batch): every
    handle's solve is launched on its own stream before any is waited for, so
    handles created on distinct streams run concurrently.  Returns one
    SolveStats per handle; raises if any solve failed."""
    recons = list(recons)
    if not recons:
        return []
    lib = recons[0]._lib
    sts = (_abi.recon_stats * len(recons))()
    arrs = [r._stats_record(sts[b], record) for b, r in enumerate(recons)]
    hs = (C.c_void_p * len(recons))(*[r._h.value for r in recons])
    rc = lib.recon_solve_batch(hs, len(recons), sts)
    _abi.check(rc, "recon_solve_batch")
    return [r._stats_out(sts[b].status, sts[b], arrs[b], record) for b, r in enumerate(recons)]


def reconstruct(recon, rho):
    """delta_r of a density grid as a differentiable torch operation: the
    forward pass deposits rho on the handle and solves; the backward pass is
    recon_adjoint (the step lengths held fixed).  The handle must have been
    created with checkpoint=1."""
    import torch

    class _Reconstruct(torch.autograd.Function):
        @staticmethod
        def forward(ctx, r):
            recon.deposit_grid(r.detach().contiguous())
            recon.solve(record=False)
            return recon.field("delta_r")

        @staticmethod
        def backward(ctx, g):
            return recon.adjoint(g.detach().contiguous())

    return _Reconstruct.apply(rho)
