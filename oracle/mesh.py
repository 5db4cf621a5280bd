"""Periodic particle-mesh pieces of the COLA force: CIC deposit, PM force, CIC gather.

Oracle (test infrastructure only).  Float64 except where a float32 decision is the definition.

Paper passages: Sec. 2 (a PM code with a 768^3 grid for 256^3 particles; forces on a PM grid),
App. A.1 eq. eom (the force -(3/2) Om a d_x d_x^-2 delta(x, a), with delta the fractional
overdensity).  The paper does not spell out the PM details; the readings used here are:

  * mass assignment and force interpolation: cloud-in-cell (CIC) with the same kernel;
    mesh node c sits at position c * H, H = L / Ng;
  * Fourier convention f_k = sum_x f(x) exp(-i k.x), inverse divided by Ng^3;
  * d^-2 -> -1/k^2 with the k = 0 mode set to zero; the gradient d_j -> i k_j, set to zero on
    the Nyquist plane |n_j| = Ng/2 of that component;
  * CIC deconvolution: divide by W(k)^p, W = prod_d sinc^2(pi n_d / Ng), p = 0, 1 or 2
    (default 1).

The "unit force" returned here is g = -d_x d_x^-2 delta (deconvolved), so the acceleration of
eq. eom is (3/2) Om a * g; in Fourier space g_j = i k_j delta_k / (k^2 W^p).
"""
import numpy as np
import scipy.fft

FFT_WORKERS = -1  # all host cores for the library FFT steps


def lattice_index(n):
    """(ix, iy, iz) lattice indices of particles p = (iz n + iy) n + ix, each int64 (n^3,)."""
    p = np.arange(n**3, dtype=np.int64)
    return p % n, (p // n) % n, p // (n * n)


def lattice_q(n, box):
    """Lagrangian positions q = L (ix, iy, iz) / n, shape (3, n^3), float64."""
    ix, iy, iz = lattice_index(n)
    return np.stack([ix, iy, iz]).astype(np.float64) * (box / n)


# ---- CIC deposit ------------------------------------------------------------------------
def cic_deposit(pos, ng, box):
    """Float64 CIC density (particle counts per cell), shape (ng, ng, ng) = [iz][iy][ix].

    Each particle adds prod_d max(0, 1 - |x_d / H - c_d|) to node c (periodic)."""
    u = np.asarray(pos, dtype=np.float64) * (ng / box)
    base = np.floor(u)
    frac = u - base
    base = base.astype(np.int64)
    rho = np.zeros(ng**3, dtype=np.float64)
    for dz in (0, 1):
        wz = frac[2] if dz else 1.0 - frac[2]
        cz = (base[2] + dz) % ng
        for dy in (0, 1):
            wy = frac[1] if dy else 1.0 - frac[1]
            cy = (base[1] + dy) % ng
            for dx in (0, 1):
                wx = frac[0] if dx else 1.0 - frac[0]
                cx = (base[0] + dx) % ng
                rho += np.bincount((cz * ng + cy) * ng + cx, weights=wz * wy * wx, minlength=ng**3)
    return rho.reshape(ng, ng, ng)


def fixed_point_coords(s32, n_p, ng, box, fbits):
    """Fixed-point CIC coordinates used by the integer deposit (a reading of this library).

    Per axis d, with lattice index i_d and float32 displacement s_d:
        q_fix = floor(i_d * ng * 2^F / n_p)                      (exact integer)
        w     = fl32(s_d * fl32(ng / box))                        (one float32 multiply)
        f     = (q_fix + floor(w * 2^F)) mod (ng * 2^F)
    The cell is f >> F and the upper-neighbour weight t = f mod 2^F (lower weight 2^F - t).
    Returns f as int64 array (3, n_p^3)."""
    s32 = np.asarray(s32, dtype=np.float32)
    scale32 = np.float32(ng / box)
    one = np.int64(1) << np.int64(fbits)
    lat = lattice_index(n_p)
    out = np.empty((3, n_p**3), dtype=np.int64)
    for d in range(3):
        qfix = (lat[d] * np.int64(ng) * one) // np.int64(n_p)
        w = s32[d] * scale32  # float32 * float32 -> float32, round to nearest
        dfix = np.floor(w * np.float32(2.0**fbits)).astype(np.int64)
        out[d] = np.mod(qfix + dfix, np.int64(ng) * one)
    return out


def cic_deposit_fixed(s32, n_p, ng, box, fbits=15):
    """Integer CIC deposit rho_fix (int64, [iz][iy][ix]); sum = n_p^3 * 2^(3F) exactly."""
    f = fixed_point_coords(s32, n_p, ng, box, fbits)
    one = np.int64(1) << np.int64(fbits)
    cell = f >> np.int64(fbits)
    t = f & (one - 1)
    rho = np.zeros(ng**3, dtype=np.int64)
    for dz in (0, 1):
        wz = t[2] if dz else one - t[2]
        cz = (cell[2] + dz) % ng
        for dy in (0, 1):
            wy = t[1] if dy else one - t[1]
            cy = (cell[1] + dy) % ng
            for dx in (0, 1):
                wx = t[0] if dx else one - t[0]
                cx = (cell[0] + dx) % ng
                np.add.at(rho, (cz * ng + cy) * ng + cx, wz * wy * wx)
    return rho.reshape(ng, ng, ng)


def overdensity(rho, n_particles):
    """delta = rho / rho_bar - 1 with rho_bar = n_particles / ng^3 (float64)."""
    ng3 = rho.size
    return rho * (ng3 / n_particles) - 1.0


# ---- CIC gather -------------------------------------------------------------------------
def cic_gather(field, pos, box):
    """Float64 CIC interpolation of a periodic mesh field ([iz][iy][ix]) at positions (3, P)."""
    ng = field.shape[0]
    flat = field.reshape(-1)
    u = np.asarray(pos, dtype=np.float64) * (ng / box)
    base = np.floor(u)
    frac = u - base
    base = base.astype(np.int64)
    out = np.zeros(u.shape[1], dtype=np.float64)
    for dz in (0, 1):
        wz = frac[2] if dz else 1.0 - frac[2]
        cz = (base[2] + dz) % ng
        for dy in (0, 1):
            wy = frac[1] if dy else 1.0 - frac[1]
            cy = (base[1] + dy) % ng
            for dx in (0, 1):
                wx = frac[0] if dx else 1.0 - frac[0]
                cx = (base[0] + dx) % ng
                out += wz * wy * wx * flat[(cz * ng + cy) * ng + cx]
    return out


# ---- Fourier-space operators ------------------------------------------------------------
def mode_numbers(ng, half_last=True):
    """Integer mode numbers (nz, ny, nx) broadcastable over the r2c half spectrum."""
    full = np.fft.fftfreq(ng, d=1.0 / ng).round().astype(np.int64)  # 0..ng/2-1, -ng/2..-1
    nx = np.arange(ng // 2 + 1, dtype=np.int64) if half_last else full
    return full[:, None, None], full[None, :, None], nx[None, None, :]


def cic_window(ng, half_last=True):
    """W(k) = prod_d sinc^2(pi n_d / ng) on the half spectrum."""
    nz, ny, nx = mode_numbers(ng, half_last)
    return (np.sinc(nz / ng) ** 2) * (np.sinc(ny / ng) ** 2) * (np.sinc(nx / ng) ** 2)


def gradient_factor(n_axis, ng, box):
    """i k_j with the Nyquist plane |n_j| = ng/2 set to zero (complex128, broadcastable)."""
    k = 2.0 * np.pi / box * n_axis.astype(np.float64)
    k = np.where(np.abs(n_axis) == ng // 2, 0.0, k)
    return 1j * k


def unit_force_mesh(delta, box, deconv=1):
    """g_j = IFFT(i k_j delta_k / (k^2 W^deconv)), j = x, y, z; i.e. -d_j d^-2 delta (eq. eom).

    Returns a list of three float64 meshes [iz][iy][ix]."""
    ng = delta.shape[0]
    dk = scipy.fft.rfftn(delta, workers=FFT_WORKERS)
    nz, ny, nx = mode_numbers(ng)
    kf = 2.0 * np.pi / box
    k2 = kf * kf * (nx * nx + ny * ny + nz * nz).astype(np.float64)
    k2[0, 0, 0] = 1.0
    green = 1.0 / k2
    if deconv:
        green = green / cic_window(ng) ** deconv
    green[0, 0, 0] = 0.0
    pot = dk * green  # -d^-2 delta in Fourier space (deconvolved)
    out = []
    for n_axis in (nx, ny, nz):
        out.append(scipy.fft.irfftn(pot * gradient_factor(n_axis, ng, box), s=delta.shape,
                                    workers=FFT_WORKERS))
    return out


def unit_force_particles(pos, n_particles, ng, box, deconv=1):
    """CIC deposit -> delta -> g mesh -> CIC gather at the same positions; shape (3, P)."""
    delta = overdensity(cic_deposit(pos, ng, box), n_particles)
    meshes = unit_force_mesh(delta, box, deconv)
    return np.stack([cic_gather(m, pos, box) for m in meshes])


def unit_force_axis_wave(s_line, axis, n_p, ng, box, deconv=1):
    """Unit force (the force mesh and gather above) on a lattice displaced along one axis only.

    Special case used where the mesh is too large for unit_force_particles: every particle
    (ix, iy, iz) is displaced by s_line[i_axis] along `axis` and not at all across it, and the
    mesh side is an integer multiple r = ng / n_p of the lattice side.  Then the particles of
    one lattice plane i_axis form a sheet sitting exactly on the mesh nodes c = 0 mod r of the
    two transverse axes, and the same PM definition reduces to one dimension:

      * deposit: rho(x, y, z) = rho_1(x) E(y) E(z), rho_1 the 1-D CIC deposit of the n_p sheet
        positions (one unit each) and E(c) = [c = 0 mod r] = (1/r) sum_j exp(2 pi i j c / r);
        so delta = r rho_1 sum_{j,l} exp(2 pi i (j y + l z) / r) - 1 and delta_1 = r rho_1 - 1;
      * every transverse pair (j, l) carries the same x spectrum delta_1k for k_x != 0, at
        transverse mode numbers (j ng / r, l ng / r);
      * on the sheets (y, z = 0 mod r) all transverse phases are 1, the CIC gather is 1-D, and
        g_axis(k_x) = i k_x delta_1k / W(k_x)^p * sum_{j,l} 1 / (W_j^p W_l^p (k_x^2 + k_j^2 + k_l^2)),
        with the Nyquist plane of the component and k = 0 set to zero as in unit_force_mesh;
      * the transverse components vanish: their gradient factor is zero at transverse mode 0
        and on the Nyquist plane, and the sum over j (and over l) of i k_j cancels in pairs
        (+-j) for the other modes.

    s_line: displacements of the n_p sheets (float64 values of the float32 inputs), shape (n_p,).
    Returns the axis component of g at each sheet, shape (n_p,), float64."""
    r = ng // n_p
    assert r * n_p == ng, "the mesh side must be a multiple of the lattice side"
    x = np.mod(np.arange(n_p) * (box / n_p) + np.asarray(s_line, dtype=np.float64), box)
    u = x * (ng / box)
    base = np.floor(u).astype(np.int64)
    frac = u - np.floor(u)
    rho1 = np.zeros(ng)
    np.add.at(rho1, base % ng, 1.0 - frac)
    np.add.at(rho1, (base + 1) % ng, frac)
    delta1 = r * rho1 - 1.0
    dk = np.fft.rfft(delta1)
    kf = 2.0 * np.pi / box
    nx = np.arange(ng // 2 + 1)
    kx = kf * nx
    w1 = np.sinc(nx / ng) ** 2
    trans = [((j * ng // r + ng // 2) % ng) - ng // 2 for j in range(r)]  # signed mode numbers
    green = np.zeros(nx.size)
    for j in trans:
        for l in trans:
            wt = (np.sinc(j / ng) ** 2 * np.sinc(l / ng) ** 2) ** deconv
            k2 = kx**2 + (kf * j) ** 2 + (kf * l) ** 2
            with np.errstate(divide="ignore"):
                green += np.where(k2 > 0, 1.0 / (wt * k2), 0.0)
    grad = np.where(nx == ng // 2, 0.0, kx)
    gk = 1j * grad * dk * green / (w1**deconv)
    gk[0] = 0.0
    g = np.fft.irfft(gk, n=ng)
    # 1-D CIC gather at the sheets
    return g[base % ng] * (1.0 - frac) + g[(base + 1) % ng] * frac
