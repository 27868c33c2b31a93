"""Seeded synthetic inputs shaped like the paper's simulation fields.

The paper reconstructs the z = 0 density of a 2048^3-particle N-body run gridded
to 512^3 (Sec. III).  Those snapshots are not available, so inputs are drawn
here: a Gaussian random field with the BBKS transfer function (Bardeen et al.
1986; Gamma = 0.2, n_s = 1, sigma_8 = 0.8), and one particle per grid node moved
by the Zel'dovich (first-order) or second-order Lagrangian displacement at
growth D = 1 (Sec. IV, x = q + Psi(q)).

This module holds none of the reconstruction's arithmetic (no deposit, no
solve): it only produces particle positions and the seed's linear field.  Both
the oracle and the CUDA library are fed from it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

try:  # multithreaded FFTs when scipy is present
    import scipy.fft as _fft

    def _rfftn(a):
        return _fft.rfftn(a, workers=-1)

    def _irfftn(a, s):
        return _fft.irfftn(a, s=s, workers=-1)
except ImportError:  # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, s):
        return np.fft.irfftn(a, s=s)

__all__ = ["bbks_transfer", "power_bbks", "sigma_R", "linear_field", "lpt_particles",
           "Workload", "WORKLOADS"]


def bbks_transfer(k, gamma=0.2):
    """BBKS transfer function T(q), q = k / Gamma, k in h/Mpc."""
    q = np.asarray(k, dtype=np.float64) / gamma
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.log1p(2.34 * q) / (2.34 * q) * (
            1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25
    return np.where(q > 0, t, 1.0)


def power_bbks(k, amp=1.0, gamma=0.2, ns=1.0):
    """Linear power P(k) = amp k^ns T^2(k) in (Mpc/h)^3."""
    k = np.asarray(k, dtype=np.float64)
    return amp * k ** ns * bbks_transfer(k, gamma) ** 2


def sigma_R(R=8.0, amp=1.0, gamma=0.2, ns=1.0):
    """rms of the linear field in top-hat spheres of radius R (Mpc/h)."""
    lnk = np.linspace(np.log(1e-6), np.log(1e3), 40001)
    k = np.exp(lnk)
    x = k * R
    W = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    integrand = k ** 3 * power_bbks(k, amp, gamma, ns) * W ** 2 / (2.0 * np.pi ** 2)
    trap = getattr(np, "trapezoid", None) or np.trapz
    return float(np.sqrt(trap(integrand, lnk)))


def _kgrid(n, box):
    kf = 2.0 * np.pi / box
    k1 = np.fft.fftfreq(n, d=1.0 / n) * kf
    kr = np.fft.rfftfreq(n, d=1.0 / n) * kf
    return (k1[:, None, None], k1[None, :, None], kr[None, None, :])


def _nyquist_mask(n):
    i = np.fft.fftfreq(n, d=1.0 / n)
    ir = np.fft.rfftfreq(n, d=1.0 / n)
    ny = n // 2
    bad = (np.abs(i)[:, None, None] == ny) | (np.abs(i)[None, :, None] == ny) | \
          (np.abs(ir)[None, None, :] == ny)
    bad[0, 0, 0] = True
    return bad


def linear_field(n, box, seed, sigma8=0.8, gamma=0.2, ns=1.0, return_k=False):
    """Gaussian random field delta_L on an n^3 grid of side box (Mpc/h).

    White noise from numpy's PCG64(seed), Fourier-transformed and scaled by
    sqrt(P(k) n^3 / box^3) so the discrete field has power P(k); the k = 0 mode
    and the Nyquist planes are zeroed.  Amplitude fixed by sigma_8.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n, n, n))
    amp = (sigma8 / sigma_R(8.0, 1.0, gamma, ns)) ** 2
    kx, ky, kz = _kgrid(n, box)
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    dk = _rfftn(w)
    del w
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.sqrt(power_bbks(kk, amp, gamma, ns) * n ** 3 / box ** 3)
    scale[_nyquist_mask(n)] = 0.0
    dk *= scale
    del scale
    delta = _irfftn(dk, (n, n, n))
    if return_k:
        return delta, dk
    return delta


def lpt_particles(n, box, seed, order=1, growth=1.0, sigma8=0.8, gamma=0.2, ns=1.0):
    """One particle per node of an n^3 grid, displaced by Zel'dovich (order=1)
    or 2LPT (order=2) at linear growth D = growth.

    Returns (positions, delta_L): positions is (n^3, 3) float64 in box units,
    wrapped into [0, box), in C order of the Lagrangian node q; delta_L is the
    linear field scaled by D.
    x = q - D grad Phi1 + D2 grad Phi2 with lap Phi1 = delta_L,
    lap Phi2 = sum_{a<b} (Phi1_aa Phi1_bb - Phi1_ab^2), D2 = -3/7 D^2.
    """
    delta, dk = linear_field(n, box, seed, sigma8, gamma, ns, return_k=True)
    kx, ky, kz = _kgrid(n, box)
    kv = (kx, ky, kz)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2[0, 0, 0] = 1.0
    phi1 = -dk / k2  # lap Phi1 = delta  ->  Phi1_k = -delta_k / k^2
    del dk
    psi = np.empty((3, n, n, n))
    for a in range(3):  # -grad Phi1
        psi[a] = growth * _irfftn(-1j * kv[a] * phi1, (n, n, n))
    if order >= 2:
        d2 = -3.0 / 7.0 * growth ** 2
        diag = [_irfftn(-kv[a] * kv[a] * phi1, (n, n, n)) for a in range(3)]
        src = diag[0] * diag[1] + diag[0] * diag[2] + diag[1] * diag[2]
        del diag
        for a, b in ((0, 1), (0, 2), (1, 2)):
            pab = _irfftn(-kv[a] * kv[b] * phi1, (n, n, n))
            src -= pab * pab
            del pab
        sk = _rfftn(src)
        del src
        phi2 = -sk / k2
        phi2[0, 0, 0] = 0.0
        phi2[_nyquist_mask(n)] = 0.0
        del sk
        for a in range(3):  # + D2 grad Phi2
            psi[a] += d2 * _irfftn(1j * kv[a] * phi2, (n, n, n))
        del phi2
    h = box / n
    q = np.arange(n, dtype=np.float64) * h
    pos = np.empty((n, n, n, 3))
    pos[..., 0] = q[:, None, None] + psi[0]
    pos[..., 1] = q[None, :, None] + psi[1]
    pos[..., 2] = q[None, None, :] + psi[2]
    del psi
    pos = np.mod(pos, box).reshape(-1, 3)
    pos[pos >= box] -= box  # mod can round up to box
    return pos, delta * growth


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: grid n^3, box side (Mpc/h), displacement order,
    seed, and the precision mode it is run in."""
    name: str
    n: int
    box: float
    order: int
    seed: int
    precision: str

    @property
    def cell(self):
        return self.box / self.n

    def particles(self):
        return lpt_particles(self.n, self.box, self.seed, order=self.order)


# The configurations the solve is exercised and measured on.
WORKLOADS = {
    "za32": Workload("32^3 ZA, 100 Mpc/h, FP64", 32, 100.0, 1, 1000, "fp64"),
    "lpt256": Workload("256^3 2LPT, 400 Mpc/h, mixed vs FP64", 256, 400.0, 2, 1001, "mixed"),
    "lpt512": Workload("512^3 2LPT, 800 Mpc/h, mixed vs FP64", 512, 800.0, 2, 1002, "mixed"),
    "za128": Workload("128^3 ZA, 200 Mpc/h", 128, 200.0, 1, 1004, "fp64"),
}


def mock_batch(per_size=32, sizes=((32, 100.0), (64, 200.0), (128, 400.0)), seed0=2000):
    """Batched mock catalogues: per_size Zel'dovich realisations of each
    (n, box) pair (3.125 Mpc/h cells in the default sizes), with seeds
    seed0 + i in order; solved in mixed precision."""
    out = []
    for n, box in sizes:
        for _ in range(per_size):
            i = len(out)
            out.append(Workload(f"mock {i}: {n}^3 ZA, {box:g} Mpc/h", n, box, 1, seed0 + i, "mixed"))
    return out
