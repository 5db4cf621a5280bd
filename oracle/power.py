"""Shell-averaged matter power spectrum of a periodic density mesh.

Oracle (test infrastructure only).  Float64.

Paper passage: Sec. 3.1 (power spectra P_i of the models; ensemble averages replaced by
averages in k-bins).  Readings of this library (the paper gives no estimator formula):
  * P(k) = (L^3 / N^6) |delta_k|^2 / W(k)^2, W the CIC window (no shot-noise subtraction);
  * shells b = 1, 2, ...: integer |n|^2 = m falls in shell b iff b(b-1) < m <= b(b+1), i.e.
    (b - 1/2) k_F <= |k| < (b + 1/2) k_F, k_F = 2 pi / L, decided exactly in integers;
  * over the r2c half spectrum, planes n_x = 0 and n_x = N/2 count once, others twice;
  * per shell: k_b = mean |k|, P_b = mean P, nmodes_b = the mode count (weights summed).
"""
import numpy as np
import scipy.fft

from .mesh import FFT_WORKERS, cic_window, mode_numbers


def shell_index(m):
    """Shell b of integer |n|^2 = m: the b >= 0 with b(b-1) < m <= b(b+1)."""
    m = np.asarray(m, dtype=np.int64)
    r = np.floor(np.sqrt(m.astype(np.float64))).astype(np.int64)
    r = np.where((r + 1) * (r + 1) <= m, r + 1, r)
    r = np.where(r * r > m, r - 1, r)
    return np.where(m <= r * (r + 1), r, r + 1)


def power_spectrum(delta, box, nbins, deconvolve=True):
    """Returns (k, P, nmodes) for shells b = 1..nbins (arrays of length nbins)."""
    ng = delta.shape[0]
    dk = scipy.fft.rfftn(np.asarray(delta, dtype=np.float64), workers=FFT_WORKERS)
    nz, ny, nx = mode_numbers(ng)
    m = (nx * nx + ny * ny + nz * nz)
    m = np.broadcast_to(m, dk.shape)
    b = shell_index(m)
    weight = np.where((nx == 0) | (nx == ng // 2), 1.0, 2.0)
    weight = np.broadcast_to(weight, dk.shape)
    p = np.abs(dk) ** 2 * (box**3 / float(ng) ** 6)
    if deconvolve:
        p = p / cic_window(ng) ** 2
    kmag = 2.0 * np.pi / box * np.sqrt(m.astype(np.float64))
    sel = (b >= 1) & (b <= nbins)
    idx = (b[sel] - 1).ravel()
    w = weight[sel].ravel()
    nmodes = np.bincount(idx, weights=w, minlength=nbins)
    ksum = np.bincount(idx, weights=w * kmag[sel].ravel(), minlength=nbins)
    psum = np.bincount(idx, weights=w * p[sel].ravel(), minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        kmean = np.where(nmodes > 0, ksum / nmodes, 0.0)
        pmean = np.where(nmodes > 0, psum / nmodes, 0.0)
    return kmean, pmean, nmodes.astype(np.int64)
