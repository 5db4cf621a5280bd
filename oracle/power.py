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


def n_max(rho):
    """eq. nmax: n_max = (2/3) rho / sqrt(1 - rho^2) (App. B; +inf at rho = 1)."""
    rho = np.asarray(rho, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return (2.0 / 3.0) * rho / np.sqrt(1.0 - rho * rho)


def cross_correlation(delta_a, delta_b, box, nbins):
    """Cross-correlation coefficient of two density meshes (Sec. 3.1) and n_max (eq. nmax).

    rho(k) = <delta_a delta_b^*> / sqrt(<|delta_a|^2> <|delta_b|^2>), the ensemble averages
    replaced by averages over the shells of power_spectrum (reading: the square root in the
    denominator, as in App. B; the real part of the cross term, which is what the Hermitian
    pairs +-k sum to).  The CIC window cancels in rho; the spectra are deconvolved as in
    power_spectrum.  Returns (k, P_a, P_b, P_ab, rho, n_max, nmodes) for shells b = 1..nbins."""
    ng = delta_a.shape[0]
    da = scipy.fft.rfftn(np.asarray(delta_a, dtype=np.float64), workers=FFT_WORKERS)
    db = scipy.fft.rfftn(np.asarray(delta_b, dtype=np.float64), workers=FFT_WORKERS)
    nz, ny, nx = mode_numbers(ng)
    m = np.broadcast_to(nx * nx + ny * ny + nz * nz, da.shape)
    b = shell_index(m)
    weight = np.broadcast_to(np.where((nx == 0) | (nx == ng // 2), 1.0, 2.0), da.shape)
    norm = box**3 / float(ng) ** 6 / cic_window(ng) ** 2
    sel = (b >= 1) & (b <= nbins)
    idx = (b[sel] - 1).ravel()
    w = weight[sel].ravel()

    def shell_mean(q):
        s = np.bincount(idx, weights=w * np.broadcast_to(q, da.shape)[sel].ravel(), minlength=nbins)
        with np.errstate(invalid="ignore", divide="ignore"):
            return np.where(nmodes > 0, s / nmodes, 0.0)

    nmodes = np.bincount(idx, weights=w, minlength=nbins)
    kmean = shell_mean(2.0 * np.pi / box * np.sqrt(m.astype(np.float64)))
    pa = shell_mean(np.abs(da) ** 2 * norm)
    pb = shell_mean(np.abs(db) ** 2 * norm)
    pab = shell_mean((da * np.conj(db)).real * norm)
    with np.errstate(invalid="ignore", divide="ignore"):
        rho = pab / np.sqrt(pa * pb)
    return kmean, pa, pb, pab, rho, n_max(rho), nmodes.astype(np.int64)
