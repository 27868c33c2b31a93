"""Shell-averaged cross-correlation coefficient r(k) of two periodic fields,
written out from its definition (Sec. III of Zhu et al. 2016):
r(k) = P_ab(k) / sqrt(P_aa(k) P_bb(k)), with every power a sum over the
Fourier modes of one spherical shell.

TEST INFRASTRUCTURE ONLY (the tests and the scripts that write the stored
oracle values use it).  Shells are |k| / k_f rounded to the nearest integer,
k_f = 2 pi / box, from 1 to n/2; the full complex FFT is used, so every mode
is counted once with no half-space weights.
"""
import numpy as np


def cross_correlation(a, b, box):
    """(k of each non-empty shell, r(k)) for two real n^3 fields of side box."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.shape[0]
    fa, fb = np.fft.fftn(a), np.fft.fftn(b)
    m = np.fft.fftfreq(n, d=1.0 / n)
    kk = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    shell = np.rint(kk).astype(np.int64).ravel()
    nb = n // 2 + 1
    sel = (shell > 0) & (shell < nb)
    sh = shell[sel]
    fa, fb = fa.ravel()[sel], fb.ravel()[sel]
    pab = np.bincount(sh, np.real(fa * np.conj(fb)), nb)
    paa = np.bincount(sh, np.abs(fa) ** 2, nb)
    pbb = np.bincount(sh, np.abs(fb) ** 2, nb)
    good = (paa > 0) & (pbb > 0)
    k = np.arange(nb) * (2 * np.pi / box)
    return k[good], pab[good] / np.sqrt(paa[good] * pbb[good])
