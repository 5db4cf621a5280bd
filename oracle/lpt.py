"""Zel'dovich and second-order LPT displacement fields on the Lagrangian lattice.

Oracle (test infrastructure only).  Float64.

Paper passages: Sec. 2 (2LPT initial conditions at z_init = 9 from 2LPTic; x_LPT is 2LPT),
App. A.3 (s_res = s - D1 s1 - D2 s2 with s1, s2 the Zel'dovich and 2LPT displacement fields
at a = 1, D1(1) = D2(1) = 1; s1, s2 are a by-product of any 2LPT code, kept per particle).

Readings (the paper cites 2LPT, not its formulas):
  * linear density at a = 1 from unit white noise w on the n^3 lattice of side L:
        delta_k = w_k sqrt(P(k) n^3 / L^3),  delta_{k=0} = 0;
  * psi1 = -grad d^-2 delta, i.e. psi1_k = i k delta_k / k^2  (so div psi1 = -delta);
  * psi1_{i,j} = d_j psi1_i, source mu2 = sum_{i<j} (psi1_{i,i} psi1_{j,j} - psi1_{i,j}^2);
  * psi2 = grad d^-2 mu2, i.e. psi2_k = -i k mu2_k / k^2 (so div psi2 = mu2);
  * every first derivative i k_j is zero on the Nyquist plane |n_j| = n/2; second derivatives
    are products of first derivatives;
  * s1 = psi1 and s2 = D2u(1) psi2 (the normalisation D2(1) = 1 of App. A.3).
"""
import numpy as np
import scipy.fft

from .mesh import FFT_WORKERS, gradient_factor, mode_numbers


def linear_density_k(noise, box, cosmo):
    """delta_k = w_k sqrt(P(k) n^3 / L^3), zero at k = 0 (half spectrum, complex128)."""
    n = noise.shape[0]
    wk = scipy.fft.rfftn(np.asarray(noise, dtype=np.float64), workers=FFT_WORKERS)
    nz, ny, nx = mode_numbers(n)
    kf = 2.0 * np.pi / box
    kmag = kf * np.sqrt((nx * nx + ny * ny + nz * nz).astype(np.float64))
    kmag[0, 0, 0] = 1.0
    amp = np.sqrt(cosmo.pk_linear(kmag) * n**3 / box**3)
    amp[0, 0, 0] = 0.0
    return wk * amp


def lpt_fields(delta_k, n, box):
    """psi1 and psi2 (each (3, n^3) float64, components x, y, z) from the linear delta_k."""
    nz, ny, nx = mode_numbers(n)
    kf = 2.0 * np.pi / box
    k2 = kf * kf * (nx * nx + ny * ny + nz * nz).astype(np.float64)
    k2[0, 0, 0] = 1.0
    inv_k2 = 1.0 / k2
    inv_k2[0, 0, 0] = 0.0
    grad = [gradient_factor(a, n, box) for a in (nx, ny, nz)]
    shape = (n, n, n)

    def c2r(fk):
        return scipy.fft.irfftn(fk, s=shape, workers=FFT_WORKERS)

    base = delta_k * inv_k2
    psi1 = np.stack([c2r(grad[j] * base).reshape(-1) for j in range(3)])
    d = {}
    for i in range(3):
        for j in range(i, 3):
            d[i, j] = c2r(grad[i] * grad[j] * base)
    mu2 = (d[0, 0] * d[1, 1] + d[0, 0] * d[2, 2] + d[1, 1] * d[2, 2]
           - d[0, 1] ** 2 - d[0, 2] ** 2 - d[1, 2] ** 2)
    mu2_k = scipy.fft.rfftn(mu2, workers=FFT_WORKERS) * inv_k2
    psi2 = np.stack([c2r(-grad[j] * mu2_k).reshape(-1) for j in range(3)])
    return psi1, psi2


def ic_2lpt(noise, box, cosmo):
    """The paper's s1 and s2 (App. A.3) for white noise ``noise`` ([iz][iy][ix], n^3)."""
    n = noise.shape[0]
    psi1, psi2 = lpt_fields(linear_density_k(noise, box, cosmo), n, box)
    d2u1 = cosmo.growth([1.0])["d2u1"]
    return psi1, d2u1 * psi2
