"""Reverse-mode derivative (adjoint) of a COLA run with respect to the initial white noise.

Oracle (test infrastructure only).  Float64.  Nothing here is in the paper, which has no
derivatives; the adjoint is the exact transpose of the forward map the oracle implements
(oracle.lpt, oracle.mesh, oracle.cola), written out operator by operator and applied in the
reverse order of eq. ALCtimestep:

  forward, per step i:   K(a_i, a_i+1/2; a_i)  D(a_i, a_i+1; a_i+1/2)  K(a_i+1/2, a_i+1; a_i+1)
    Kick:  v += c (A g(s) - T2D1 s1 - T2D2 s2),  A = (3/2) Om a_c, g the unit PM force
    Drift: s += cD v + dD1 s1 + dD2 s2
  reverse:  Kick^T: lam_s += c A (dg/ds)^T lam_v, lam_s1 -= c T2D1 lam_v, lam_s2 -= c T2D2 lam_v
            Drift^T: lam_v += cD lam_s, lam_s1 += dD1 lam_s, lam_s2 += dD2 lam_s
            L+^T: lam_s1 += TD1 lam_v, lam_s2 += TD2 lam_v;  the 2LPT velocity and L- cancel.

PM force g_p = sum_c W(u_p - c) F(c), F_i = K_i delta, delta = rho/rho_bar - 1, rho_c =
sum_q W(u_q - c), u = x N/L, K_i the Fourier multiplier m_i = i k_i / (k^2 W^p) (inverse
scaled by 1/N^3).  Its vector-Jacobian product with lam (3, P):
  mu_q = (N/L) [ sum_i lam_q,i sum_c dW(u_q - c) F_i(c) + (1/rho_bar) sum_c dW(u_q - c) Phi(c) ],
  Phi = sum_i K_i^T Lam_i,  Lam_i(c) = sum_p W(u_p - c) lam_p,i,  K_i^T = multiplier conj(m_i),
with dW the gradient of the CIC kernel in cell units (a.e.; the kernel has kinks at cell faces).
"""
import numpy as np
import scipy.fft

from . import mesh
from .cola import evolve, quantise_positions
from .cosmology import time_grid
from .lpt import ic_2lpt, linear_density_k
from .mesh import FFT_WORKERS, cic_window, gradient_factor, mode_numbers


def _corners(pos, ng, box):
    u = np.asarray(pos, dtype=np.float64) * (ng / box)
    base = np.floor(u)
    frac = u - base
    return base.astype(np.int64), frac


def cic_gather_grad(field, pos, box):
    """(3, P): gradient with respect to x of the CIC interpolation of `field` at pos,
    sum_c dW(u_p - c)/dx field(c), for a scalar mesh field [iz][iy][ix]."""
    ng = field.shape[0]
    flat = field.reshape(-1)
    base, f = _corners(pos, ng, box)
    out = np.zeros((3, base.shape[1]))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = [f[0] if dx else 1 - f[0], f[1] if dy else 1 - f[1], f[2] if dz else 1 - f[2]]
                dw = [1.0 if dx else -1.0, 1.0 if dy else -1.0, 1.0 if dz else -1.0]
                cx, cy, cz = (base[0] + dx) % ng, (base[1] + dy) % ng, (base[2] + dz) % ng
                val = flat[(cz * ng + cy) * ng + cx]
                out[0] += dw[0] * w[1] * w[2] * val
                out[1] += w[0] * dw[1] * w[2] * val
                out[2] += w[0] * w[1] * dw[2] * val
    return out * (ng / box)


def cic_deposit_weighted(pos, values, ng, box):
    """sum_p W(u_p - c) values_p on the mesh (float64 CIC of arbitrary particle values)."""
    base, f = _corners(pos, ng, box)
    rho = np.zeros(ng**3)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                cx, cy, cz = (base[0] + dx) % ng, (base[1] + dy) % ng, (base[2] + dz) % ng
                rho += np.bincount((cz * ng + cy) * ng + cx, weights=w * values, minlength=ng**3)
    return rho.reshape(ng, ng, ng)


def force_multipliers(ng, box, deconv):
    """m_i(k) = i k_i / (k^2 W^p) on the half spectrum (zero at k = 0), i = x, y, z."""
    nz, ny, nx = mode_numbers(ng)
    kf = 2.0 * np.pi / box
    k2 = kf * kf * (nx * nx + ny * ny + nz * nz).astype(np.float64)
    k2[0, 0, 0] = 1.0
    green = 1.0 / k2
    if deconv:
        green = green / cic_window(ng) ** deconv
    green[0, 0, 0] = 0.0
    return [gradient_factor(n_axis, ng, box) * green for n_axis in (nx, ny, nz)]


def force_vjp(pos, lam, n_particles, ng, box, deconv=1):
    """(d g / d x)^T lam for the unit PM force g at positions pos (both (3, P))."""
    delta = mesh.overdensity(mesh.cic_deposit(pos, ng, box), n_particles)
    meshes = mesh.unit_force_mesh(delta, box, deconv)
    shape = (ng, ng, ng)
    # term A: the force meshes seen through the gradient of the gather weights
    term_a = np.zeros_like(np.asarray(pos, dtype=np.float64))
    for i in range(3):
        term_a += lam[i] * cic_gather_grad(meshes[i], pos, box)
    # term B: lam deposited, transposed force operator, gathered with the weight gradient
    mult = force_multipliers(ng, box, deconv)
    phi_k = np.zeros((ng, ng, ng // 2 + 1), dtype=np.complex128)
    for i in range(3):
        lam_mesh = cic_deposit_weighted(pos, lam[i], ng, box)
        phi_k += np.conj(mult[i]) * scipy.fft.rfftn(lam_mesh, workers=FFT_WORKERS)
    phi = scipy.fft.irfftn(phi_k, s=shape, workers=FFT_WORKERS)
    rho_bar = n_particles / ng**3
    return term_a + cic_gather_grad(phi, pos, box) / rho_bar


def density_vjp(pos, delta_bar, n_particles, box):
    """(d delta / d x)^T delta_bar for delta = rho / rho_bar - 1 (float64 CIC)."""
    ng = delta_bar.shape[0]
    return cic_gather_grad(delta_bar, pos, box) * (ng**3 / n_particles)


def ic_vjp(noise, lam_s1, lam_s2, box, cosmo):
    """Transpose of (noise -> s1, s2) of oracle.lpt.ic_2lpt applied to (lam_s1, lam_s2)."""
    n = noise.shape[0]
    shape = (n, n, n)
    nz, ny, nx = mode_numbers(n)
    kf = 2.0 * np.pi / box
    k2 = kf * kf * (nx * nx + ny * ny + nz * nz).astype(np.float64)
    k2[0, 0, 0] = 1.0
    inv_k2 = 1.0 / k2
    inv_k2[0, 0, 0] = 0.0
    grad = [gradient_factor(a, n, box) for a in (nx, ny, nz)]
    kmag = kf * np.sqrt((nx * nx + ny * ny + nz * nz).astype(np.float64))
    kmag[0, 0, 0] = 1.0
    amp = np.sqrt(cosmo.pk_linear(kmag) * n**3 / box**3)
    amp[0, 0, 0] = 0.0

    def r2c(f):
        return scipy.fft.rfftn(np.asarray(f).reshape(shape), workers=FFT_WORKERS)

    def c2r(fk):
        return scipy.fft.irfftn(fk, s=shape, workers=FFT_WORKERS)

    d2u1 = cosmo.growth([1.0])["d2u1"]
    # s2 = d2u1 psi2, psi2_j = IFFT((-i k_j / k^2) mu2_k): transpose multiplier (+i k_j / k^2)
    lam_mu2 = c2r(sum(np.conj(-grad[j] * inv_k2) * r2c(d2u1 * lam_s2[j]) for j in range(3)))
    # mu2 = sum_{i<j} (p_ii p_jj - p_ij^2), p_ij = IFFT(M_ij delta_k), M_ij = (i k_i)(i k_j) / k^2
    delta_k = linear_density_k(noise, box, cosmo)
    p = {(i, j): c2r(grad[i] * grad[j] * delta_k * inv_k2) for i in range(3) for j in range(i, 3)}
    lam_p = {}
    for i in range(3):
        lam_p[i, i] = lam_mu2 * sum(p[j, j] for j in range(3) if j != i)
    for (i, j) in ((0, 1), (0, 2), (1, 2)):
        lam_p[i, j] = -2.0 * lam_mu2 * p[i, j]
    lam_dk = sum(np.conj(grad[i] * grad[j] * inv_k2) * r2c(lam_p[i, j]) for (i, j) in lam_p)
    # s1_j = IFFT((i k_j / k^2) delta_k)
    lam_dk = lam_dk + sum(np.conj(grad[j] * inv_k2) * r2c(lam_s1[j]) for j in range(3))
    # delta_k = amp(k) FFT(noise): transpose = IFFT(amp * .) with the same 1/n^3 scaling
    return c2r(amp * lam_dk)


def forward_with_checkpoints(noise, cfg):
    """oracle.cola's forward run that also keeps the displacement of every force evaluation."""
    s1, s2 = ic_2lpt(np.asarray(noise, dtype=np.float64), cfg.box, cfg.cosmo)
    ckpt = []
    out = evolve(s1, s2, cfg, "cola", record=ckpt)
    return {"s": out["s"], "v": out["v"], "s1": s1, "s2": s2, "ckpt": ckpt}


def final_density(s, cfg):
    pos = np.mod(mesh.lattice_q(cfg.n_p, cfg.box) + s, cfg.box)
    if cfg.fixed_bits > 0:
        pos = quantise_positions(pos, cfg.n_g, cfg.box, cfg.fixed_bits)
    return mesh.overdensity(mesh.cic_deposit(pos, cfg.n_g, cfg.box), cfg.n_p**3)


def loss_and_gradient(noise, target, cfg):
    """L = sum_c (delta_c - target_c)^2 of the final CIC density, and dL/d noise (float64)."""
    fw = forward_with_checkpoints(noise, cfg)
    loss, grad = loss_and_gradient_along(noise, target, cfg, fw["ckpt"], fw["s"])
    return loss, grad, fw


def loss_and_gradient_along(noise, target, cfg, ckpt, s_final, positions=None):
    """The reverse sweep of loss_and_gradient along a given trajectory: ckpt = the displacement
    at each of the nsteps + 1 force evaluations, s_final = the final displacement.  The loss and
    the adjoint are evaluated at the particle positions positions(s) (default: x = q + s modulo
    L, rounded down to 2^-F cell when cfg.fixed_bits = F > 0, the reading oracle.cola applies to
    the force), so that a trajectory computed elsewhere is differentiated on the same side of
    every CIC kink as it was integrated.  Returns (loss, dL/d noise)."""
    cosmo = cfg.cosmo
    a, mid = time_grid(cfg.a_init, cfg.a_final, cfg.nsteps, cfg.spacing)
    g = cosmo.growth(a)
    q = mesh.lattice_q(cfg.n_p, cfg.box)
    npart = cfg.n_p**3
    am = 1.5 * cosmo.omega_m

    def pos_of(s):
        if positions is not None:
            return positions(s)
        pos = np.mod(q + s, cfg.box)
        if cfg.fixed_bits > 0:
            pos = quantise_positions(pos, cfg.n_g, cfg.box, cfg.fixed_bits)
        return pos

    pos_final = pos_of(s_final)
    delta = mesh.overdensity(mesh.cic_deposit(pos_final, cfg.n_g, cfg.box), npart)
    loss = float(np.sum((delta - target) ** 2))
    lam_s = density_vjp(pos_final, 2.0 * (delta - target), npart, cfg.box)
    lam_v = np.zeros_like(lam_s)
    lam_s1 = np.zeros_like(lam_s)
    lam_s2 = np.zeros_like(lam_s)
    # L+ (eq. Lops)
    lam_s1 += g["TD1"][-1] * lam_v
    lam_s2 += g["TD2"][-1] * lam_v
    for i in reversed(range(cfg.nsteps)):
        # K(a_i+1/2, a_i+1; a_i+1) with the force at the positions after the drift
        c = cosmo.kick_cola(mid[i], a[i + 1], a[i + 1], cfg.n_lpt)
        lam_s += c * am * a[i + 1] * force_vjp(pos_of(ckpt[i + 1]), lam_v, npart, cfg.n_g, cfg.box, cfg.deconv)
        lam_s1 -= c * g["T2D1"][i + 1] * lam_v
        lam_s2 -= c * g["T2D2"][i + 1] * lam_v
        # D(a_i, a_i+1; a_i+1/2)
        lam_v += cosmo.drift_cola(a[i], a[i + 1], mid[i], cfg.n_lpt) * lam_s
        lam_s1 += (g["D1"][i + 1] - g["D1"][i]) * lam_s
        lam_s2 += (g["D2"][i + 1] - g["D2"][i]) * lam_s
        # K(a_i, a_i+1/2; a_i)
        c = cosmo.kick_cola(a[i], mid[i], a[i], cfg.n_lpt)
        lam_s += c * am * a[i] * force_vjp(pos_of(ckpt[i]), lam_v, npart, cfg.n_g, cfg.box, cfg.deconv)
        lam_s1 -= c * g["T2D1"][i] * lam_v
        lam_s2 -= c * g["T2D2"][i] * lam_v
    # initial conditions: s = D1 s1 + D2 s2 (the 2LPT velocity and L- cancel exactly)
    lam_s1 += g["D1"][0] * lam_s
    lam_s2 += g["D2"][0] * lam_s
    grad = ic_vjp(np.asarray(noise, dtype=np.float64), lam_s1, lam_s2, cfg.box, cosmo)
    return loss, grad


def loss_only(noise, target, cfg):
    fw = forward_with_checkpoints(noise, cfg)
    return float(np.sum((final_density(fw["s"], cfg) - target) ** 2))
