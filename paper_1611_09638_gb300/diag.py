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


def _shell_sums(fa, fb, n):
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kr[None, None, :] ** 2)
    wgt = np.where((kr[None, None, :] > 0) & (kr[None, None, :] < n / 2), 2.0, 1.0)
    wgt = np.broadcast_to(wgt, kk.shape).ravel()
    shell = np.rint(kk).astype(int).ravel()
    nb = n // 2 + 1
    sel = (shell > 0) & (shell < nb)
    s = np.bincount(shell[sel], wgt[sel] * np.real(fa.ravel()[sel] * np.conj(fb.ravel()[sel])), nb)
    cnt = np.bincount(shell[sel], wgt[sel], nb)
    return s, cnt


def cross_power(a, b, box):
    """(k, P_ab(k)) in (box units)^3, shells of width 2 pi / box: the
    estimator of the power spectra of Sec. III."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.shape[0]
    s, cnt = _shell_sums(np.fft.rfftn(a), np.fft.rfftn(b), n)
    good = cnt > 0
    vol = float(box) ** 3
    p = np.zeros_like(s)
    p[good] = s[good] / cnt[good] * vol / float(n) ** 6
    k = np.arange(len(s)) * 2 * np.pi / box
    return k[good], p[good]


def power_spectrum(a, box):
    return cross_power(a, a, box)


def propagator(delta, delta_L, box):
    """C(k) = P_{delta delta_L} / P_{delta_L} (Sec. III)."""
    k, pxl = cross_power(delta, delta_L, box)
    _, pl = power_spectrum(delta_L, box)
    return k, pxl / pl


def mode_coupling(delta, delta_L, box):
    """P_N(k) = P_delta - C^2 P_{delta_L}, the power not explained by the
    linear signal (Sec. III, P_delta = C^2 P_L + P_N)."""
    k, C = propagator(delta, delta_L, box)
    _, pd = power_spectrum(delta, box)
    _, pl = power_spectrum(delta_L, box)
    return k, pd - C ** 2 * pl


def delta_E(psi, box):
    """delta_E(q) = -div Psi(q) (Sec. III) of a displacement field psi of
    shape (3, n, n, n) in box units, by spectral differentiation."""
    psi = np.asarray(psi, dtype=np.float64)
    n = psi.shape[1]
    kf = 2 * np.pi / box
    k1 = np.fft.fftfreq(n, d=1.0 / n) * kf
    kr = np.fft.rfftfreq(n, d=1.0 / n) * kf
    kv = (k1[:, None, None], k1[None, :, None], kr[None, None, :])
    div = np.zeros((n, n, n // 2 + 1), dtype=complex)
    for a in range(3):
        div += 1j * kv[a] * np.fft.rfftn(psi[a])
    return -np.fft.irfftn(div, s=(n, n, n), axes=(0, 1, 2))


def displacement_from_positions(pos, n, box):
    """Psi(q) = x - q (minimum image) of one particle per node, (3, n, n, n)."""
    q = np.stack(np.meshgrid(*(np.arange(n) * (box / n),) * 3, indexing="ij"), -1).reshape(-1, 3)
    d = (np.asarray(pos) - q + box / 2) % box - box / 2
    return np.moveaxis(d.reshape(n, n, n, 3), -1, 0)
