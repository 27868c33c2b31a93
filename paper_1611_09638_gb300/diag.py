"""FFT diagnostics of the reconstruction (off the solve path): the
cross-correlation coefficient r(k) = P_ab / sqrt(P_aa P_bb) of Sec. III in
spherical shells of width k_f = 2 pi / box, without window deconvolution."""
import numpy as np


def cross_correlation(a, b, box):
    """(k_centres, r(k)) for two real fields on the same n^3 grid of side box."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.shape[0]
    fa, fb = np.fft.rfftn(a), np.fft.rfftn(b)
    kf = 2 * np.pi / box
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kr[None, None, :] ** 2)
    # rfft half-space: modes with 0 < k_z < n/2 stand for two conjugate modes
    wgt = np.where((kr[None, None, :] > 0) & (kr[None, None, :] < n / 2), 2.0, 1.0)
    wgt = np.broadcast_to(wgt, kk.shape)
    shell = np.rint(kk).astype(int).ravel()
    nb = n // 2 + 1
    sel = (shell > 0) & (shell < nb)
    w = wgt.ravel()[sel]
    sh = shell[sel]
    pab = np.bincount(sh, w * np.real(fa.ravel()[sel] * np.conj(fb.ravel()[sel])), nb)
    paa = np.bincount(sh, w * np.abs(fa.ravel()[sel]) ** 2, nb)
    pbb = np.bincount(sh, w * np.abs(fb.ravel()[sel]) ** 2, nb)
    good = (paa > 0) & (pbb > 0)
    ks = np.arange(nb) * kf
    r = np.zeros(nb)
    r[good] = pab[good] / np.sqrt(paa[good] * pbb[good])
    return ks[good], r[good]
