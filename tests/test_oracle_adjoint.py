"""Pins of the oracle's adjoint (vector-Jacobian product of rho -> delta_r
with the step lengths held fixed, Sec. II / App. A) against central finite
differences of the oracle's own forward solve, plus invariants the map has.

The forward map is piecewise smooth: the step lengths are frozen (replayed),
and tiny perturbations (1e-6 of the mean density) do not move a tracer across
a cell face or a node across a Heaviside switch.  Both solves run to a 1e-13
relative residual so that the finite differences resolve the derivative to
~1e-7.  The inputs are strongly nonlinear, so the compression limiter
(lambda0 < xi_m), the expansion limiter (sqrt g > v_m, with v_m = 2) and the
coefficient floor a_min all act in some of the cases.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_09638_gb300.inputs import lpt_particles


def _case(n, box, seed, K, **kw):
    pos, _ = lpt_particles(n, box, seed, order=2)
    rho = O.cic_deposit((n, n, n), pos / (box / n))
    p = O.OracleParams(n=(n, n, n), k_max=K, tol_in=1e-13, max_vcycles=200, **kw)
    f = O.solve(p, rho)
    return p, rho, f


def _loss(p, rho, alpha, gbar):
    ra = np.r_[alpha, np.zeros(p.k_max - len(alpha))]
    s = O.solve(p, rho, replay_alpha=ra)
    return float(np.sum(gbar * O.delta_r(s.phi)))


def _check_fd(p, rho, alpha, ncells, seed, rtol=1e-4):
    rng = np.random.default_rng(seed)
    gbar = rng.standard_normal(rho.shape)
    grad = O.adjoint(p, rho, alpha, gbar)
    eps = 1e-6 * rho.mean()
    scale = np.abs(grad).max()
    for c in rng.choice(np.flatnonzero(rho.ravel() > 1e-3), ncells, replace=False):
        e = np.zeros(rho.size)
        e[c] = eps
        e = e.reshape(rho.shape)
        fd = (_loss(p, rho + e, alpha, gbar) - _loss(p, rho - e, alpha, gbar)) / (2 * eps)
        assert abs(grad.ravel()[c] - fd) <= rtol * max(abs(fd), 1e-2 * scale), (c, grad.ravel()[c], fd)
    d = rng.random(rho.shape) * (rho > 1e-3)
    fd = (_loss(p, rho + eps * d, alpha, gbar) - _loss(p, rho - eps * d, alpha, gbar)) / (2 * eps)
    assert abs(np.sum(grad * d) - fd) <= rtol * abs(fd)
    return grad


def test_adjoint_matches_finite_differences_with_the_compression_limiter_active():
    p, rho, f = _case(8, 25.0, 3, 10)
    assert f.steps == 10 and f.min_lam.min() < p.xi_m  # C acts in the later steps
    _check_fd(p, rho, f.alpha, 12, 0)


def test_adjoint_matches_finite_differences_with_expansion_limiter_and_floor():
    p, rho, f = _case(16, 30.0, 5, 6, v_m=2.0)
    g, _ = O.geometry(f.phi)
    assert g.max() > p.v_m  # E acts
    assert (f.m < p.a_min).any()  # a = max(m, a_min) clamps
    _check_fd(p, rho, f.alpha, 6, 1)


@pytest.mark.parametrize("reading", [O.CLIM_LITERAL, O.CLIM_STEP])
def test_adjoint_matches_finite_differences_for_the_other_limiter_readings(reading):
    p, rho, f = _case(8, 25.0, 3, 4, climiter=reading)
    _check_fd(p, rho, f.alpha, 6, 2)


def test_adjoint_invariants():
    p, rho, f = _case(8, 25.0, 3, 5)
    rng = np.random.default_rng(3)
    g1 = rng.standard_normal(rho.shape)
    a1 = O.adjoint(p, rho, f.alpha, g1)
    # linear in gbar
    a2 = O.adjoint(p, rho, f.alpha, 2.0 * g1 + 1.0)
    assert np.allclose(a2, 2.0 * a1, rtol=0, atol=1e-9 * np.abs(a1).max())
    # delta_r depends on rho only through rho / mean(rho): zero along rho
    assert abs(np.sum(a1 * rho)) <= 1e-9 * np.abs(a1).max() * np.abs(rho).sum()
    # no steps: delta_r = 0 for every rho
    assert not O.adjoint(p, rho, [], g1).any()
    with pytest.raises(RuntimeError):
        O.adjoint(O.OracleParams(n=(8, 8, 8), density_update=1), rho, f.alpha, g1)
