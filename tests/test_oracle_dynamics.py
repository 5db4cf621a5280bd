"""Dynamics pins of the oracle (App. A: eqs. eom, eomALC, ALCtimestep, Lops, KDKALC; Sec. 2).

* Continuum check of the 2LPT solution: the Lagrangian form of eq. eom,
  J div_x(T^2 s) + (3/2) Om a (1 - J) = 0, J = det(1 + d s / d q), has a residual of third
  order in the amplitude for s = D1 s1 + D2 s2 and T^2 s = T^2[D1] s1 + T^2[D2] s2 (App. A.3),
  evaluated with exact spectral derivatives on band-limited fields.
* The COLA operators with the exact 2LPT force reproduce the 2LPT trajectory exactly for any
  number of steps (eqs. eomALC, KDKALC, Lops: the residual force then vanishes).
* Linear regime on a mesh: COLA recovers D1(1) s1 after 1, 2 or 10 steps up to mesh error,
  the standard leapfrog (eq. KDKStd) does not with 2 steps (Sec. 2: "exact to second order
  for any number of timesteps, even one"; App. A.2).
* Momentum conservation of a full run (zero-mean s1, s2 and an antisymmetric force).
"""
import numpy as np
import pytest
import scipy.fft

from oracle import lpt, mesh
from oracle.cola import ColaConfig, evolve, run
from oracle.cosmology import Cosmology
from oracle.philox import white_noise


def band_limited_delta_k(n, amp, seed=4, nmax=2):
    rng = np.random.default_rng(seed)
    nz, ny, nx = mesh.mode_numbers(n)
    m = np.broadcast_to(nx * nx + ny * ny + nz * nz, (n, n, n // 2 + 1))
    dk = np.zeros((n, n, n // 2 + 1), dtype=complex)
    sel = (m > 0) & (m <= nmax * nmax)
    dk[sel] = rng.standard_normal(sel.sum()) + 1j * rng.standard_normal(sel.sum())
    d = scipy.fft.irfftn(dk, s=(n, n, n))
    d *= amp / d.std()
    return scipy.fft.rfftn(d)


def spectral_jacobian(field3, n, box):
    """d field_i / d q_j on the lattice by exact spectral differentiation (full FFT)."""
    k1 = 2 * np.pi / box * np.fft.fftfreq(n, 1.0 / n)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    out = np.empty((n**3, 3, 3))
    for i in range(3):
        fk = np.fft.fftn(field3[i].reshape(n, n, n))
        for j, kj in enumerate((kx, ky, kz)):
            out[:, i, j] = np.real(np.fft.ifftn(1j * kj * fk)).reshape(-1)
    return out


def lagrangian_residual(amp, a, flip_s2=False):
    cosmo = Cosmology()
    n, box = 24, 300.0
    s1, psi2 = lpt.lpt_fields(band_limited_delta_k(n, amp), n, box)
    g = cosmo.growth([a])
    s2 = g["d2u1"] * psi2 * (-1.0 if flip_s2 else 1.0)
    s = g["D1"][0] * s1 + g["D2"][0] * s2
    acc = g["T2D1"][0] * s1 + g["T2D2"][0] * s2
    m = spectral_jacobian(s, n, box)
    da = spectral_jacobian(acc, n, box)
    eye = np.eye(3)[None]
    jac = np.linalg.det(eye + m)
    div_x = np.einsum("pji,pij->p", np.linalg.inv(eye + m), da)
    resid = jac * div_x + 1.5 * cosmo.omega_m * a * (1.0 - jac)
    scale = 1.5 * cosmo.omega_m * a * np.sqrt(np.mean((1.0 - jac) ** 2))
    return np.sqrt(np.mean(resid**2)), scale


@pytest.mark.parametrize("a", [0.1, 0.5, 1.0])
def test_2lpt_solves_lagrangian_eom_to_second_order(a):
    r1, sc1 = lagrangian_residual(0.01, a)
    r2, sc2 = lagrangian_residual(0.02, a)
    assert r1 < 1e-2 * sc1
    assert np.log2(r2 / r1) == pytest.approx(3.0, abs=0.15)  # third-order residual
    # with the second-order field of the wrong sign the residual is second order
    f1, _ = lagrangian_residual(0.01, a, flip_s2=True)
    f2, _ = lagrangian_residual(0.02, a, flip_s2=True)
    assert np.log2(f2 / f1) == pytest.approx(2.0, abs=0.15)


@pytest.mark.parametrize("nsteps", [1, 3, 10])
@pytest.mark.parametrize("scheme", ["cola", "cola_std", "cola_u1"])
def test_cola_operators_exact_with_2lpt_force(nsteps, scheme):
    cosmo = Cosmology()
    n, box = 8, 100.0
    s1, psi2 = lpt.lpt_fields(band_limited_delta_k(n, 0.3, seed=9), n, box)
    g1 = cosmo.growth([1.0])
    s2 = g1["d2u1"] * psi2
    cfg = ColaConfig(n_p=n, n_g=n, box=box, nsteps=nsteps)

    def exact(s_, a_):
        g = cosmo.growth([a_])
        return g["T2D1"][0] * s1 + g["T2D2"][0] * s2

    out = evolve(s1, s2, cfg, scheme, accel_fn=exact)
    assert np.allclose(out["s"], g1["D1"][0] * s1 + g1["D2"][0] * s2, atol=1e-12)
    assert np.allclose(out["v"], g1["TD1"][0] * s1 + g1["TD2"][0] * s2, atol=1e-12)
    if nsteps < 10:
        # the standard leapfrog (no LPT frame) is not exact for the same force
        pm = evolve(s1, s2, cfg, "pm_std", accel_fn=exact)
        assert np.abs(pm["s"] - out["s"]).max() > 1e-3 * np.abs(out["s"]).max()


def test_linear_regime_cola_exact_for_any_step_count():
    # ratio-1 mesh with the lattice on cell centres: the CIC response is then the symmetric
    # difference, and the mesh error is O((k H)^2) on these long modes.
    cosmo = Cosmology()
    n, box = 32, 200.0
    s1, psi2 = lpt.lpt_fields(band_limited_delta_k(n, 1e-3), n, box)
    g1 = cosmo.growth([1.0])
    s2 = g1["d2u1"] * psi2
    half = 0.5 * box / n
    rms = lambda x: float(np.sqrt(np.mean(x**2)))
    for nsteps in (1, 2, 10):
        cfg = ColaConfig(n_p=n, n_g=n, box=box, nsteps=nsteps, deconv=2)
        out = evolve(s1, s2, cfg, "cola", offset=half)
        assert rms(out["s"] - half - s1 - s2) < 1e-2 * rms(s1)
    cfg = ColaConfig(n_p=n, n_g=n, box=box, nsteps=2, deconv=2)
    pm = evolve(s1, s2, cfg, "pm_std", offset=half)
    assert rms(pm["s"] - half - s1 - s2) > 4e-2 * rms(s1)


def test_full_run_conserves_momentum():
    cfg = ColaConfig(n_p=16, n_g=32, box=100.0, nsteps=4)
    out = run(white_noise(16, 1), cfg)
    for key in ("s1", "s2"):
        assert np.abs(out[key].sum(axis=1)).max() < 1e-9 * np.abs(out[key]).sum()
    v = out["v"]
    assert np.abs(v.sum(axis=1)).max() < 1e-9 * np.abs(v).sum()


@pytest.mark.parametrize("scheme", ["cola", "cola_std", "cola_u1", "pm_std"])
@pytest.mark.parametrize("spacing", ["a", "loga"])
def test_scheme_coefficients_match_eds_closed_forms(scheme, spacing):
    # Einstein-de Sitter (Q = a^(3/2)), no LPT frame (s1 = s2 = 0) and a uniform acceleration c:
    # the run reduces to v += c_K c, s += c_D v with the closed forms
    #   eq. KDKALC:    c_K = (af^n - ai^n) / (n ac^(n+1/2)),  c_D = (af^(n-1/2) - ai^(n-1/2)) / ((n-1/2) ac^n)
    #   eq. KDKALCstd / KDKStd: c_K = 2 (af^(1/2) - ai^(1/2)) / ac,  c_D = 2 (ai^(-1/2) - af^(-1/2))
    # and "cola_u1" = the KDKALC Kick with the standard Drift (u = 1 in the Drift).
    n, nsteps, a0, a1 = -2.5, 4, 0.1, 1.0
    cfg = ColaConfig(n_p=2, n_g=4, box=10.0, cosmo=Cosmology(omega_m=1.0, omega_l=0.0), n_lpt=n, nsteps=nsteps,
                     a_init=a0, a_final=a1, spacing=spacing)
    zero = np.zeros((3, 8))
    c = np.array([1.0, -2.0, 0.5])[:, None] * np.ones((3, 8))
    out = evolve(zero, zero, cfg, scheme=scheme, accel_fn=lambda s_, a_: c)
    if spacing == "a":
        a = a0 + (a1 - a0) * np.arange(nsteps + 1) / nsteps
    else:
        a = a0 * (a1 / a0) ** (np.arange(nsteps + 1) / nsteps)
    mid = 0.5 * (a[:-1] + a[1:])

    def kick(ai, af, ac):
        if scheme in ("cola", "cola_u1"):
            return (af**n - ai**n) / (n * ac ** (n + 0.5))
        return 2.0 * (af**0.5 - ai**0.5) / ac

    def drift(ai, af, ac):
        if scheme == "cola":
            return (af ** (n - 0.5) - ai ** (n - 0.5)) / ((n - 0.5) * ac**n)
        return 2.0 * (ai**-0.5 - af**-0.5)

    s_ref, v_ref = np.zeros(3), np.zeros(3)
    for i in range(nsteps):
        v_ref = v_ref + kick(a[i], mid[i], a[i]) * c[:, 0]
        s_ref = s_ref + drift(a[i], a[i + 1], mid[i]) * v_ref
        v_ref = v_ref + kick(mid[i], a[i + 1], a[i + 1]) * c[:, 0]
    assert np.allclose(out["s"][:, 0], s_ref, rtol=1e-9, atol=0)
    assert np.allclose(out["v"][:, 0], v_ref, rtol=1e-9, atol=0)
