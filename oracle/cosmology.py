"""Background cosmology, growth factors, COLA time coefficients and the linear power spectrum.

Oracle (test infrastructure only; never imported by the product path).  Float64 throughout.

Paper passages followed (arXiv:1301.0322):
  * App. A.1, eq. eom: T = Q(a) d/da with Q(a) = a^3 H(a)/H0; the displacement obeys
    T^2[s] = -(3/2) Om a d_x d_x^-2 delta.
  * App. A.3: s_res = s - D1 s1 - D2 s2 with D1(1) = D2(1) = 1; T[D], T^2[D] are needed at the
    step times ("a straightforward exercise").
  * App. A.3.2, eqs. toyKDK and KDKALC: u(a) = a^nLPT; Drift coefficient
    int_{ai}^{af} u/Q da / u(ac); Kick coefficient (u(af) - u(ai)) / T[u](ac).
  * App. A.2, eq. KDKStd and App. A.3.1, eq. KDKALCstd: the standard coefficients
    int da/Q and int (a/ac)/Q da.
  * eq. ALCtimestep: K(a_i, a_{i+1/2}; a_i), D(a_i, a_{i+1}; a_{i+1/2}), K(a_{i+1/2}, a_{i+1}; a_{i+1}),
    with a_{i+1/2} = (a_i + a_{i+1})/2 (App. A.2) and steps uniform in a (App. A.3.2).

Readings where the paper is silent:
  * H(a)/H0 = sqrt(Om a^-3 + Ok a^-2 + OL), Ok = 1 - Om - OL (no radiation).
  * Growth ODEs follow from eq. eom expanded to second order in Lagrangian perturbation
    theory (delta = -div s at first order, J = det(1 + grad s)):
        T^2[D1] = (3/2) Om a D1,        T^2[D2u] = (3/2) Om a (D2u - D1^2),
    growing modes D1 ~ a, D2u ~ -(3/7) a^2 at early times.  D1 is normalised to 1 at a = 1,
    D2 = D2u / D2u(1); the 2LPT field is then s2 = D2u(1) psi2 where div psi2 = mu2(psi1).
  * Linear P(k): BBKS no-wiggle transfer function with Gamma = Om h, P = A k^ns T^2,
    A fixed by sigma8 with a real-space top hat of radius 8 Mpc/h.
"""
import math

import numpy as np


class Cosmology:
    """Flat-or-curved LCDM background (no radiation); all quantities float64."""

    def __init__(self, omega_m=0.27, omega_l=0.73, h=0.7, sigma8=0.8, n_s=0.96):
        self.omega_m = float(omega_m)
        self.omega_l = float(omega_l)
        self.omega_k = 1.0 - self.omega_m - self.omega_l
        self.h = float(h)
        self.sigma8 = float(sigma8)
        self.n_s = float(n_s)
        self._growth_cache = {}
        self._amp = None

    # ---- background (eq. eom) -------------------------------------------------------------
    def hubble(self, a):
        """H(a)/H0."""
        a = np.asarray(a, dtype=np.float64)
        return np.sqrt(self.omega_m / a**3 + self.omega_k / a**2 + self.omega_l)

    def Q(self, a):
        """Q(a) = a^3 H(a)/H0, so that T = Q d/da (eq. eom)."""
        a = np.asarray(a, dtype=np.float64)
        return a**3 * self.hubble(a)

    # ---- growth factors (App. A.3) ---------------------------------------------------------
    def _rhs(self, a, y):
        # y = (D1, T[D1], D2u, T[D2u]); derivative with respect to x = ln a, i.e. a d/da.
        d1, v1, d2, v2 = y
        q = float(self.Q(a))
        om = self.omega_m
        return np.array([
            a * v1 / q,
            a * 1.5 * om * a * d1 / q,
            a * v2 / q,
            a * 1.5 * om * a * (d2 - d1 * d1) / q,
        ])

    def _integrate_raw(self, targets, a_start=1e-8, dlna=1e-3):
        """Classic RK4 in ln a from the matter-era growing mode to each target scale factor.

        Returns raw (unnormalised) (D1, T[D1], D2u, T[D2u]) at each target."""
        targets = sorted(set(float(t) for t in targets))
        q0 = float(self.Q(a_start))
        y = np.array([a_start, q0, -3.0 / 7.0 * a_start**2, -6.0 / 7.0 * a_start * q0])
        x = math.log(a_start)
        out = {}
        for t in targets:
            xt = math.log(t)
            nstep = max(1, int(math.ceil((xt - x) / dlna)))
            hstep = (xt - x) / nstep
            for _ in range(nstep):
                a = math.exp(x)
                k1 = self._rhs(a, y)
                am = math.exp(x + 0.5 * hstep)
                k2 = self._rhs(am, y + 0.5 * hstep * k1)
                k3 = self._rhs(am, y + 0.5 * hstep * k2)
                k4 = self._rhs(math.exp(x + hstep), y + hstep * k3)
                y = y + hstep / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
                x += hstep
            x = xt
            out[t] = y.copy()
        return out

    def growth(self, a):
        """Normalised growth quantities at scale factors ``a`` (App. A.3).

        Returns a dict of float64 arrays: D1, D2 (both 1 at a=1), TD1 = T[D1], TD2 = T[D2],
        T2D1 = T^2[D1], T2D2 = T^2[D2], and the scalar d2u1 = D2u(1) (with D1(1) = 1) that
        converts the standard 2LPT field psi2 into the paper's s2 = d2u1 * psi2."""
        a = np.atleast_1d(np.asarray(a, dtype=np.float64))
        need = [float(x) for x in a if float(x) not in self._growth_cache]
        if 1.0 not in self._growth_cache:
            need.append(1.0)
        if need:
            self._growth_cache.update(self._integrate_raw(need + list(self._growth_cache)))
        d1_1, _, d2_1, _ = self._growth_cache[1.0]
        d2u1 = d2_1 / d1_1**2
        om = self.omega_m
        rows = np.array([self._growth_cache[float(x)] for x in a])
        D1 = rows[:, 0] / d1_1
        TD1 = rows[:, 1] / d1_1
        D2un = rows[:, 2] / d1_1**2
        TD2un = rows[:, 3] / d1_1**2
        return {
            "D1": D1,
            "TD1": TD1,
            "T2D1": 1.5 * om * a * D1,
            "D2": D2un / d2u1,
            "TD2": TD2un / d2u1,
            "T2D2": 1.5 * om * a * (D2un - D1 * D1) / d2u1,
            "d2u1": d2u1,
        }

    # ---- COLA time coefficients (eqs. toyKDK, KDKALC) ------------------------------------
    @staticmethod
    def _gauss_legendre(f, lo, hi, n=32, pieces=16):
        """Composite Gauss-Legendre quadrature on geometrically spaced sub-intervals
        (integrands here are smooth powers of a, so this is exact to rounding)."""
        if lo == hi:
            return 0.0
        x, w = np.polynomial.legendre.leggauss(n)
        if lo > 0 and hi > 0:
            edges = np.geomspace(lo, hi, pieces + 1)
        else:
            edges = np.linspace(lo, hi, pieces + 1)
        total = 0.0
        for a0, a1 in zip(edges[:-1], edges[1:]):
            mid, half = 0.5 * (a1 + a0), 0.5 * (a1 - a0)
            total += half * float(np.sum(w * f(mid + half * x)))
        return total

    def drift_general(self, u, ai, af, ac):
        """Drift coefficient of the modified scheme for a general u(a):
        int_{ai}^{af} u(a)/Q(a) da / u(ac)   (eq. KDKALC, from eq. toyKDK)."""
        return self._gauss_legendre(lambda x: u(x) / self.Q(x), ai, af) / u(ac)

    @staticmethod
    def kick_general(u, Tu, ai, af, ac):
        """Kick coefficient of the modified scheme for a general u(a):
        (u(af) - u(ai)) / T[u](ac)   (eq. KDKALC, from eq. toyKDK)."""
        return (u(af) - u(ai)) / Tu(ac)

    def u_lpt(self, n_lpt):
        """The ansatz u(a) = a^nLPT and T[u] = Q n a^(n-1) (App. A.3.2)."""
        return (lambda a: np.asarray(a, dtype=np.float64) ** n_lpt,
                lambda a: self.Q(a) * n_lpt * np.asarray(a, dtype=np.float64) ** (n_lpt - 1.0))

    def drift_cola(self, ai, af, ac, n_lpt):
        u, _ = self.u_lpt(n_lpt)
        return self.drift_general(u, ai, af, ac)

    def kick_cola(self, ai, af, ac, n_lpt):
        if abs(n_lpt) < 1e-12:
            # limit n -> 0 of (af^n - ai^n) / (Q n ac^(n-1))
            return math.log(af / ai) * ac / float(self.Q(ac))
        u, Tu = self.u_lpt(n_lpt)
        return float(self.kick_general(u, Tu, ai, af, ac))

    def drift_std(self, ai, af):
        """Standard drift coefficient int_{ai}^{af} da/Q (eq. KDKStd / KDKALCstd)."""
        return self._gauss_legendre(lambda x: 1.0 / self.Q(x), ai, af)

    def kick_std(self, ai, af, ac):
        """Standard COLA kick coefficient int_{ai}^{af} (a/ac)/Q da (eq. KDKALCstd)."""
        return self._gauss_legendre(lambda x: x / ac / self.Q(x), ai, af)

    # ---- linear power spectrum ----------------------------------------------------------
    def transfer_bbks(self, k):
        """BBKS no-wiggle transfer function, q = k / (Om h), k in h/Mpc."""
        k = np.asarray(k, dtype=np.float64)
        q = k / (self.omega_m * self.h)
        x = 2.34 * q
        lead = np.where(x > 1e-12, np.log1p(x) / np.where(x > 0, x, 1.0), 1.0)
        poly = 1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4
        return lead * poly ** -0.25

    @staticmethod
    def tophat(x):
        x = np.asarray(x, dtype=np.float64)
        small = x < 1e-2
        xs = np.where(small, 1.0, x)
        full = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs**3
        series = 1.0 - x * x / 10.0 + x**4 / 280.0
        return np.where(small, series, full)

    def sigma_r_unnormalised(self, radius=8.0):
        """sigma^2(R) of k^ns T^2(k): (1/2pi^2) int k^3 P W^2 dln k, Simpson on a ln-k grid."""
        lnk = np.linspace(math.log(1e-7), math.log(1e4), 2**16 + 1)
        k = np.exp(lnk)
        f = k**3 * k**self.n_s * self.transfer_bbks(k) ** 2 * self.tophat(k * radius) ** 2
        hstep = lnk[1] - lnk[0]
        simpson = hstep / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum())
        return simpson / (2.0 * math.pi**2)

    @property
    def amplitude(self):
        """A in P(k) = A k^ns T^2(k), fixed by sigma8 (z = 0 linear power)."""
        if self._amp is None:
            self._amp = self.sigma8**2 / self.sigma_r_unnormalised(8.0)
        return self._amp

    def pk_linear(self, k):
        """Linear P(k) at a = 1 in (Mpc/h)^3, k in h/Mpc."""
        k = np.asarray(k, dtype=np.float64)
        return self.amplitude * k**self.n_s * self.transfer_bbks(k) ** 2


def time_grid(a_init, a_final, nsteps, spacing="a"):
    """Scale factors a_0..a_n and midpoints a_{i+1/2} = (a_i + a_{i+1}) / 2 (App. A.2).

    spacing "a": uniform in a, the grid of the optimal COLA variant (App. A.3.2);
    spacing "loga": uniform in ln a, the grid App. A.2 finds better for the standard leapfrog.
    The midpoint rule is the one App. A.2 states for small steps; it is kept for both grids."""
    i = np.arange(nsteps + 1, dtype=np.float64) / nsteps
    if spacing == "a":
        a = a_init + (a_final - a_init) * i
    elif spacing == "loga":
        a = a_init * (a_final / a_init) ** i
    else:
        raise ValueError(f"unknown spacing {spacing!r}")
    a[0], a[-1] = a_init, a_final
    return a, 0.5 * (a[:-1] + a[1:])
