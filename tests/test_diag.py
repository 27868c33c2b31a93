"""FFT diagnostics of Sec. III (off the solve path): cross-correlation r(k),
propagator C(k), mode-coupling power P_N(k) and delta_E = -div Psi."""
import numpy as np

from paper_1611_09638_gb300 import diag
from paper_1611_09638_gb300.inputs import linear_field, lpt_particles


def test_cross_correlation_limits():
    d = linear_field(32, 200.0, 1)
    k, r = diag.cross_correlation(d, d, 200.0)
    assert np.allclose(r, 1.0)
    _, r = diag.cross_correlation(d, -3.0 * d, 200.0)
    assert np.allclose(r, -1.0)
    e = linear_field(32, 200.0, 2)
    _, r = diag.cross_correlation(d, e, 200.0)
    assert np.abs(r[6:]).max() < 0.2  # independent fields: |r| ~ 1/sqrt(modes per shell)


def test_propagator_and_mode_coupling_of_a_scaled_field_plus_noise():
    d = linear_field(32, 200.0, 1)
    k, C = diag.propagator(0.7 * d, d, 200.0)
    assert np.allclose(C, 0.7)
    _, pn = diag.mode_coupling(0.7 * d, d, 200.0)
    _, pd = diag.power_spectrum(0.7 * d, 200.0)
    assert np.abs(pn).max() < 1e-10 * pd.max()
    # the power spectrum of the linear field follows the input spectrum's shape
    _, pl = diag.power_spectrum(d, 200.0)
    assert pl[1] > pl[-1]


def test_delta_E_of_zeldovich_displacement_is_the_linear_field():
    n, box = 32, 400.0
    pos, dL = lpt_particles(n, box, 5, order=1)
    psi = diag.displacement_from_positions(pos, n, box)
    dE = diag.delta_E(psi, box)
    assert np.linalg.norm(dE - dL) < 1e-8 * np.linalg.norm(dL)
