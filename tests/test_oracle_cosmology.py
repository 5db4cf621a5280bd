"""Pins of oracle.cosmology against closed forms, an independent integral and the toy model.

Paper passages: App. A.1 (eq. eom), App. A.3 (growth factors, eq. KDKALC), App. A.3.2 (eq.
toyKDK: the modified kick/drift integrate exactly when v_res / u and f / T[u] are constant).
"""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle.cosmology import Cosmology, time_grid

A_TEST = [0.02, 0.1, 0.37, 0.55, 1.0]


@pytest.fixture(scope="module")
def eds():
    return Cosmology(omega_m=1.0, omega_l=0.0)


@pytest.fixture(scope="module")
def lcdm():
    return Cosmology(omega_m=0.27, omega_l=0.73, h=0.7, sigma8=0.8, n_s=0.96)


def test_eds_growth_closed_forms(eds):
    # Einstein-de Sitter: Q = a^(3/2); D1 = a, D2u = -(3/7) a^2 so D2 = a^2 and D2u(1) = -3/7;
    # T[a^p] = p a^(p+1/2), T^2[a^p] = p (p + 1/2) a^(p+1).
    a = np.array(A_TEST)
    g = eds.growth(a)
    assert np.allclose(eds.Q(a), a**1.5, rtol=1e-15)
    assert np.allclose(g["D1"], a, rtol=1e-9)
    assert np.allclose(g["D2"], a**2, rtol=1e-8)
    assert g["d2u1"] == pytest.approx(-3.0 / 7.0, rel=1e-9)
    assert np.allclose(g["TD1"], a**1.5, rtol=1e-9)
    assert np.allclose(g["TD2"], 2.0 * a**2.5, rtol=1e-8)
    assert np.allclose(g["T2D1"], 1.5 * a**2, rtol=1e-9)
    assert np.allclose(g["T2D2"], 5.0 * a**3, rtol=1e-7)


def test_lcdm_d1_matches_heath_integral(lcdm):
    # For matter + Lambda (+ curvature) the growing mode is D1 ~ H(a) int_0^a da' / (a' H(a'))^3.
    def heath(a):
        integral, _ = scipy.integrate.quad(lambda x: 1.0 / (x * lcdm.hubble(x)) ** 3, 0.0, a,
                                           epsabs=0, epsrel=1e-13, limit=200)
        return float(lcdm.hubble(a)) * integral

    a = np.array(A_TEST)
    g = lcdm.growth(a)
    ref = np.array([heath(x) for x in a]) / heath(1.0)
    assert np.allclose(g["D1"], ref, rtol=1e-9)


def test_lcdm_d2_normalisation_matches_fit(lcdm):
    # Bouchet et al. (1995): D2u / D1^2 ~ -(3/7) Om^(-1/143) at a = 1 in flat LCDM (sub-percent).
    for om in (0.27, 0.5):
        c = Cosmology(omega_m=om, omega_l=1 - om)
        d2u1 = c.growth([1.0])["d2u1"]
        assert d2u1 == pytest.approx(-3.0 / 7.0 * om ** (-1.0 / 143.0), rel=2e-3)


def test_growth_time_derivatives_consistent(lcdm):
    # T[D] = Q dD/da and T^2[D] = Q d T[D] / da, checked by central differences.
    a = np.array([0.1, 0.3, 0.7])
    h = 1e-5
    gp, gm, g0 = lcdm.growth(a + h), lcdm.growth(a - h), lcdm.growth(a)
    q = lcdm.Q(a)
    for d, td, t2d in (("D1", "TD1", "T2D1"), ("D2", "TD2", "T2D2")):
        assert np.allclose(q * (gp[d] - gm[d]) / (2 * h), g0[td], rtol=1e-7)
        assert np.allclose(q * (gp[td] - gm[td]) / (2 * h), g0[t2d], rtol=1e-6)


def test_eds_step_coefficients_closed_forms(eds):
    n = -2.5
    for ai, af in ((0.1, 0.19), (0.5, 0.6), (0.9, 1.0)):
        ac = 0.5 * (ai + af)
        drift = (af ** (n - 0.5) - ai ** (n - 0.5)) / ((n - 0.5) * ac**n)
        kick = (af**n - ai**n) / (n * ac ** (n - 1.0) * ac**1.5)
        assert eds.drift_cola(ai, af, ac, n) == pytest.approx(drift, rel=1e-13)
        assert eds.kick_cola(ai, af, ac, n) == pytest.approx(kick, rel=1e-13)
        assert eds.drift_std(ai, af) == pytest.approx(2 * (ai**-0.5 - af**-0.5), rel=1e-13)
        assert eds.kick_std(ai, af, ac) == pytest.approx(2 * (af**0.5 - ai**0.5) / ac, rel=1e-13)


def test_kick_limit_nlpt_zero(lcdm):
    ai, af, ac = 0.3, 0.4, 0.35
    eps = 1e-7
    ref = 0.5 * (lcdm.kick_cola(ai, af, ac, eps) + lcdm.kick_cola(ai, af, ac, -eps))
    assert lcdm.kick_cola(ai, af, ac, 0.0) == pytest.approx(ref, rel=1e-6)


def test_modified_scheme_reduces_to_standard(lcdm):
    # eq. KDKALC with u = 1 in the Drift gives int da/Q; with u(a) = int^a a'/Q da' (so T[u] = a)
    # the Kick gives int (a/ac)/Q da -- the coefficients of eq. KDKALCstd.
    ai, af, ac = 0.23, 0.41, 0.3

    def u_std(a):
        val, _ = scipy.integrate.quad(lambda x: x / float(lcdm.Q(x)), 0.05, a, epsrel=1e-13)
        return val

    one = lambda a: np.ones_like(np.asarray(a, dtype=np.float64))
    assert lcdm.drift_general(one, ai, af, ac) == pytest.approx(lcdm.drift_std(ai, af), rel=1e-13)
    kick = Cosmology.kick_general(u_std, lambda a: a, ai, af, ac)
    assert kick == pytest.approx(lcdm.kick_std(ai, af, ac), rel=1e-10)


@pytest.mark.parametrize("n_lpt", [-2.5, -1.0, 1.0, 3.0])
def test_toy_kdk_exact_for_the_ansatz(eds, n_lpt):
    # eq. toyKDK: if v_res / u and f / T[u] are constant in time the Kick and Drift are exact.
    # In EdS, s_res = a^(n - 1/2) has v_res = T[s_res] = (n - 1/2) a^n = (n - 1/2) u and
    # f = T^2[s_res] = (n - 1/2) T[u]; one K-D-K step of any size must reproduce it exactly.
    _, Tu = eds.u_lpt(n_lpt)
    p = n_lpt - 0.5
    force = lambda a: p * float(Tu(a))
    for ai, af in ((0.1, 1.0), (0.3, 0.31), (0.02, 0.5)):
        am = 0.5 * (ai + af)
        s, v = ai**p, p * ai**n_lpt
        v += eds.kick_cola(ai, am, ai, n_lpt) * force(ai)
        s += eds.drift_cola(ai, af, am, n_lpt) * v
        v += eds.kick_cola(am, af, af, n_lpt) * force(af)
        # relative to the largest term, since s and v may cancel from ai^p down to af^p
        assert abs(s - af**p) <= 1e-13 * max(ai**p, af**p)
        assert abs(v - p * af**n_lpt) <= 1e-13 * abs(p) * max(ai**n_lpt, af**n_lpt)
    # the standard discretisation is not exact for the same problem (the test has teeth)
    ai, af = 0.1, 1.0
    am = 0.5 * (ai + af)
    s, v = ai**p, p * ai**n_lpt
    v += eds.kick_std(ai, am, ai) * force(ai) / ai * ai  # same force, standard coefficient
    s += eds.drift_std(ai, af) * v
    assert abs(s / af**p - 1.0) > 1e-3


def test_sigma8_normalisation(lcdm):
    # independent integral (adaptive quadrature in k) of the normalised spectrum
    def integrand(lnk):
        k = math.exp(lnk)
        x = 8.0 * k
        w = 3.0 * (math.sin(x) - x * math.cos(x)) / x**3 if x > 1e-3 else 1.0 - x * x / 10.0
        return k**3 * float(lcdm.pk_linear(k)) * w * w / (2 * math.pi**2)

    val, _ = scipy.integrate.quad(integrand, math.log(1e-6), math.log(1e3), limit=500, epsrel=1e-10)
    assert math.sqrt(val) == pytest.approx(0.8, rel=1e-7)


def test_bbks_limits(lcdm):
    assert float(lcdm.transfer_bbks(1e-9)) == pytest.approx(1.0, abs=1e-7)
    # large-q asymptote: T -> ln(2.34 q) / (2.34 q) / (6.71 q)
    q = 1e7
    k = q * lcdm.omega_m * lcdm.h
    asym = math.log(2.34 * q) / (2.34 * q) / (6.71 * q)
    assert float(lcdm.transfer_bbks(k)) == pytest.approx(asym, rel=1e-5)


def _bbks_of_q(lcdm, q):
    return np.asarray(lcdm.transfer_bbks(np.asarray(q, dtype=np.float64) * lcdm.omega_m * lcdm.h))


def test_bbks_small_q_taylor_coefficients(lcdm):
    # The limits above fix only 2.34 and 6.71.  The interior coefficients of the BBKS fit
    # (Bardeen, Bond, Kaiser & Szalay 1986, eq. G3), T = ln(1 + 2.34 q)/(2.34 q) (1 + u)^(-1/4)
    # with u = 3.89 q + (16.1 q)^2 + (5.46 q)^3 + (6.71 q)^4, enter the Taylor series at q = 0:
    #   ln(1 + x)/x = 1 - x/2 + x^2/3 - ...,   (1 + u)^(-1/4) = 1 - u/4 + (5/32) u^2 - ...
    # so T = 1 + c1 q + c2 q^2 + O(q^3) with
    #   c1 = -2.34/2 - 3.89/4
    #   c2 = 2.34^2/3 + (2.34/2)(3.89/4) - 16.1^2/4 + (5/32) 3.89^2
    # c1 pins 3.89 and c2 pins 16.1.  The coefficients are read off the oracle by a least
    # squares fit of (T - 1)/q on q in [1e-5, 2e-3] (a quartic, so that the higher orders do
    # not leak into c1, c2).
    c1 = -2.34 / 2.0 - 3.89 / 4.0
    c2 = 2.34**2 / 3.0 + (2.34 / 2.0) * (3.89 / 4.0) - 16.1**2 / 4.0 + 5.0 / 32.0 * 3.89**2
    q = np.linspace(1e-5, 2e-3, 400)
    y = (_bbks_of_q(lcdm, q) - 1.0) / q
    fit = np.polynomial.polynomial.polyfit(q, y, 4)
    assert fit[0] == pytest.approx(c1, rel=1e-7)
    assert fit[1] == pytest.approx(c2, rel=1e-4)


def test_bbks_large_q_correction(lcdm):
    # For q -> oo, T (6.71 q) (2.34 q) / ln(1 + 2.34 q) = (1 + u / (6.71 q)^4)^(-1/4)
    #   = 1 - 5.46^3 / (4 * 6.71^4 q) + O(q^-2):  the 1/q term pins 5.46 (given 6.71).
    expect = -(5.46**3) / (4.0 * 6.71**4)
    for q in (1e5, 1e6):
        x = 2.34 * q
        r = float(_bbks_of_q(lcdm, q)) * 6.71 * q * x / math.log1p(x)
        assert (r - 1.0) * q == pytest.approx(expect, rel=2e-3)


def test_bbks_interior_values_and_ratio(lcdm):
    # An independent transcription of eq. G3 of BBKS, term by term in plain floats, at
    # q = 0.1, 1 and 10, and the ratio T(0.3)/T(3), which weighs the 3.89 and 16.1 terms
    # against the 5.46 and 6.71 terms.
    def t_bbks(q):
        lead = math.log(1.0 + 2.34 * q) / (2.34 * q)
        s = 1.0
        s += 3.89 * q
        s += (16.1 * q) * (16.1 * q)
        s += (5.46 * q) * (5.46 * q) * (5.46 * q)
        s += (6.71 * q) * (6.71 * q) * (6.71 * q) * (6.71 * q)
        return lead / math.sqrt(math.sqrt(s))

    for q in (0.1, 1.0, 10.0):
        assert float(_bbks_of_q(lcdm, q)) == pytest.approx(t_bbks(q), rel=1e-13)
    ratio = float(_bbks_of_q(lcdm, 0.3)) / float(_bbks_of_q(lcdm, 3.0))
    assert ratio == pytest.approx(t_bbks(0.3) / t_bbks(3.0), rel=1e-13)
    # the transfer function falls monotonically through the interior
    q = np.logspace(-3, 3, 200)
    assert np.all(np.diff(_bbks_of_q(lcdm, q)) < 0)


def test_time_grid_uniform_in_a():
    a, mid = time_grid(0.1, 1.0, 10)
    assert a[0] == 0.1 and a[-1] == 1.0 and len(a) == 11
    assert np.allclose(np.diff(a), 0.09, rtol=1e-12)
    assert np.allclose(mid, a[:-1] + 0.045, rtol=1e-12)


def test_time_grid_uniform_in_log_a():
    a, mid = time_grid(0.02, 1.0, 8, "loga")
    assert a[0] == 0.02 and a[-1] == 1.0 and len(a) == 9
    assert np.allclose(a[1:] / a[:-1], 50.0 ** (1.0 / 8.0), rtol=1e-12)
    assert np.allclose(mid, 0.5 * (a[:-1] + a[1:]), rtol=1e-15)
    with pytest.raises(ValueError):
        time_grid(0.1, 1.0, 4, "linear")
