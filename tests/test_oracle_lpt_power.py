"""Pins of oracle.lpt (App. A.3: s1, s2) and oracle.power (Sec. 3.1: P(k) in k-bins)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest
import scipy.fft

from oracle import lpt, mesh, power
from oracle.cosmology import Cosmology


def grid(n, box):
    h = box / n
    return np.meshgrid(np.arange(n) * h, np.arange(n) * h, np.arange(n) * h, indexing="ij")


def test_plane_wave_zeldovich_and_no_second_order():
    # delta_L = A cos(k x): psi1 = -(A/k) sin(k x) x_hat, and mu2 = 0 so psi2 = 0.
    n, box, amp = 16, 50.0, 0.2
    z, y, x = grid(n, box)
    k = 2 * np.pi / box * 3
    delta = amp * np.cos(k * x)
    psi1, psi2 = lpt.lpt_fields(scipy.fft.rfftn(delta), n, box)
    assert np.allclose(psi1[0], (-amp / k * np.sin(k * x)).ravel(), atol=1e-12)
    assert np.abs(psi1[1:]).max() < 1e-13
    assert np.abs(psi2).max() < 1e-13


def test_crossed_plane_waves_second_order_closed_form():
    # delta_L = A cos(k1 x) + B cos(k2 y):  mu2 = A B cos(k1 x) cos(k2 y) and
    # psi2 = (A B / 2) sum_{+-} K sin(K.x) / |K|^2,  K = (k1, +-k2, 0).
    n, box, amp_a, amp_b = 16, 30.0, 0.3, -0.2
    z, y, x = grid(n, box)
    kf = 2 * np.pi / box
    k1, k2 = 2 * kf, 3 * kf
    delta = amp_a * np.cos(k1 * x) + amp_b * np.cos(k2 * y)
    psi1, psi2 = lpt.lpt_fields(scipy.fft.rfftn(delta), n, box)
    expect = np.zeros((3,) + x.shape)
    for sgn in (1, -1):
        kvec = np.array([k1, sgn * k2, 0.0])
        ph = kvec[0] * x + kvec[1] * y
        for j in range(3):
            expect[j] += 0.5 * amp_a * amp_b * kvec[j] * np.sin(ph) / (kvec @ kvec)
    assert np.allclose(psi2, expect.reshape(3, -1), atol=1e-13)
    assert np.allclose(psi1[1], (-amp_b / k2 * np.sin(k2 * y)).ravel(), atol=1e-13)


def test_linear_density_variance_matches_spectrum():
    # <delta^2> = (1/L^3) sum_k P(k) over the lattice modes (ensemble average over seeds)
    cosmo = Cosmology()
    n, box = 16, 200.0
    rng = np.random.default_rng(11)
    var = []
    for _ in range(20):
        dk = lpt.linear_density_k(rng.standard_normal((n, n, n)), box, cosmo)
        var.append(np.mean(scipy.fft.irfftn(dk, s=(n, n, n)) ** 2))
    nz, ny, nx = np.meshgrid(*(np.fft.fftfreq(n, 1.0 / n),) * 3, indexing="ij")
    kk = 2 * np.pi / box * np.sqrt(nx**2 + ny**2 + nz**2)
    expect = cosmo.pk_linear(kk[kk > 0]).sum() / box**3
    assert np.mean(var) == pytest.approx(expect, rel=0.05)


def test_ic_2lpt_normalisation():
    cosmo = Cosmology()
    rng = np.random.default_rng(2)
    w = rng.standard_normal((8, 8, 8))
    s1, s2 = lpt.ic_2lpt(w, 100.0, cosmo)
    p1, p2 = lpt.lpt_fields(lpt.linear_density_k(w, 100.0, cosmo), 8, 100.0)
    assert np.allclose(s1, p1) and np.allclose(s2, cosmo.growth([1.0])["d2u1"] * p2)


def test_shell_index_exact():
    for m in range(0, 5000):
        b = int(power.shell_index(np.array([m]))[0])
        # (b - 1/2)^2 <= m < (b + 1/2)^2 in exact arithmetic
        assert Fraction(2 * b - 1, 2) ** 2 <= m < Fraction(2 * b + 1, 2) ** 2 or (b == 0 and m == 0)


def test_mode_counts_brute_force():
    n, nbins = 10, 8
    _, _, nmodes = power.power_spectrum(np.zeros((n, n, n)), 1.0, nbins)
    count = np.zeros(nbins, dtype=np.int64)
    rng = range(-n // 2, n // 2)
    for v in itertools.product(rng, repeat=3):
        r = np.sqrt(sum(c * c for c in v))
        b = int(np.floor(r + 0.5))
        if 1 <= b <= nbins:
            count[b - 1] += 1
    assert np.array_equal(nmodes, count)


def test_power_single_mode():
    n, box, amp = 16, 64.0, 0.7
    z, y, x = grid(n, box)
    kf = 2 * np.pi / box
    modes = (2, 1, 0)
    delta = amp * np.cos(kf * (modes[0] * x + modes[1] * y + modes[2] * z))
    k, p, nm = power.power_spectrum(delta, box, 6)
    b = 2  # |n|^2 = 5: 2*1 < 5 <= 2*3
    w = np.prod([np.sinc(m / n) ** 2 for m in modes])
    assert p[b - 1] == pytest.approx(2 * box**3 * amp**2 / 4 / w**2 / nm[b - 1], rel=1e-12)
    assert np.allclose(np.delete(p, b - 1), 0.0, atol=1e-20)


def test_cross_correlation_limits_and_power_consistency():
    from oracle import power
    rng = np.random.default_rng(9)
    n, box = 16, 40.0
    d = rng.standard_normal((n, n, n))
    e = rng.standard_normal((n, n, n))
    k, pa, pb, pab, rho, nm, cnt = power.cross_correlation(d, d, box, 6)
    k0, p0, c0 = power.power_spectrum(d, box, 6)
    assert np.allclose(pa, p0, rtol=1e-12) and np.allclose(pab, p0, rtol=1e-12) and np.array_equal(cnt, c0)
    assert np.allclose(rho, 1.0, rtol=0, atol=1e-12)
    _, _, _, _, rho_neg, _, _ = power.cross_correlation(d, -2.0 * d, box, 6)
    assert np.allclose(rho_neg, -1.0, rtol=0, atol=1e-12)
    _, pa2, pb2, pab2, rho2, _, _ = power.cross_correlation(d, e, box, 6)
    _, pba2, _, pba_ab, _, _, _ = power.cross_correlation(e, d, box, 6)
    assert np.allclose(pab2, pba_ab, rtol=1e-12) and np.all(np.abs(rho2) < 1.0)


def test_n_max_calibration_on_orthogonal_fields():
    # App. B: with delta_NL = delta_M + eps, <delta_M eps*> = 0 and P_eps / P_NL = 10%, n_max = 2.
    # delta_M = A cos(k.x) and eps = B sin(k.x) are orthogonal in every shell; B^2 / (A^2 + B^2)
    # = 0.1 puts rho = sqrt(0.9) in the shell of k.
    from oracle import power
    n, box = 16, 40.0
    i = np.arange(n)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    ph = 2 * np.pi * (2 * x + 1 * y + 0 * z) / n  # |n|^2 = 5: shell 2
    A, B = 3.0, 1.0
    dm = A * np.cos(ph)
    dnl = dm + B * np.sin(ph)
    _, _, _, _, rho, nm, cnt = power.cross_correlation(dm, dnl, box, 4)
    assert rho[1] == pytest.approx(np.sqrt(0.9), rel=1e-12)
    assert nm[1] == pytest.approx(2.0, rel=1e-12)
    assert power.n_max(np.sqrt(0.9)) == pytest.approx(2.0, rel=1e-14)
