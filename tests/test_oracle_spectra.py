"""Pins of the oracle's r(k) estimator (oracle/spectra.py) by closed forms:
a field is perfectly correlated with any positive multiple of itself and
anti-correlated with a negative one, and two plane waves of the same wave
vector with phases differing by theta have r = cos(theta) in their shell."""
import numpy as np

from oracle.spectra import cross_correlation


def test_self_and_sign():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((16, 16, 16))
    k, r = cross_correlation(a, 3.0 * a, 50.0)
    assert len(k) == 8 and np.allclose(r, 1.0, atol=1e-12)
    _, r = cross_correlation(a, -a, 50.0)
    assert np.allclose(r, -1.0, atol=1e-12)
    assert np.allclose(k, 2 * np.pi / 50.0 * np.arange(1, 9))


def test_plane_waves_phase_shift():
    n, box = 16, 100.0
    i, j, l = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    ph = 2 * np.pi * (3 * i + 0 * j + 4 * l) / n  # |m| = 5
    for theta in (0.3, 1.2, 2.5):
        k, r = cross_correlation(np.cos(ph), np.cos(ph + theta), box)
        sel = np.abs(k - 5 * 2 * np.pi / box) < 1e-12
        assert sel.sum() == 1 and abs(r[sel][0] - np.cos(theta)) < 1e-12


def test_disjoint_shells_add_no_cross_power():
    """b = a + (a field whose modes lie only in other shells): the shells of a
    keep r = 1."""
    n = 16
    i, j, l = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    a = np.cos(2 * np.pi * 2 * i / n)            # shell 2
    c = np.sin(2 * np.pi * (6 * j + 0 * l) / n)  # shell 6
    k, r = cross_correlation(a, a + c, 10.0)
    sel = np.abs(k - 2 * 2 * np.pi / 10.0) < 1e-12
    assert sel.sum() == 1 and abs(r[sel][0] - 1.0) < 1e-12
