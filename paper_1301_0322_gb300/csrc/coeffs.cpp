// Host float64 background cosmology and COLA time coefficients (App. A.1, A.3 of
// arXiv:1301.0322).  Computed once per plan; the kernels receive float32 copies.
//
//  Q(a) = a^3 H(a)/H0 = sqrt(Om a^3 + Ok a^4 + OL a^6),  T = Q d/da                 (eq. eom)
//  T^2[D1] = (3/2) Om a D1,  T^2[D2u] = (3/2) Om a (D2u - D1^2)  (second-order Lagrangian
//  perturbation theory of eq. eom), growing modes D1 ~ a, D2u ~ -(3/7) a^2 in matter domination;
//  D1(1) = 1, D2 = D2u / D2u(1)                                                     (App. A.3)
//  Kick:  c_K = (u(kb) - u(ka)) / T[u](a_c),  Drift: c_D = int_{ai}^{af} u/Q da / u(a_c),
//  u = a^nLPT                                                                      (eq. KDKALC)
//  standard coefficients: c_K = int (a/a_c)/Q da, c_D = int da/Q           (eqs. KDKStd, KDKALCstd)
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "cola_internal.cuh"

namespace cola {
namespace {

struct Background {
  double om, ol, ok;
  double Q(double a) const { return std::sqrt(om * a * a * a + ok * a * a * a * a + ol * a * a * a * a * a * a); }
};

struct GrowthState {
  double d1, t1, d2, t2;  // D1, T[D1], D2u, T[D2u] (unnormalised)
};

// d/d(ln a) of the growth state
GrowthState growth_rhs(const Background& bg, double a, const GrowthState& y) {
  const double q = bg.Q(a);
  const double src = 1.5 * bg.om * a;
  return {a * y.t1 / q, a * src * y.d1 / q, a * y.t2 / q, a * src * (y.d2 - y.d1 * y.d1) / q};
}

GrowthState axpy(const GrowthState& y, double h, const GrowthState& k) {
  return {y.d1 + h * k.d1, y.t1 + h * k.t1, y.d2 + h * k.d2, y.t2 + h * k.t2};
}

// Growth state at each (sorted ascending) target scale factor.
std::vector<GrowthState> integrate_growth(const Background& bg, const std::vector<double>& targets) {
  const double a0 = 1e-8;
  const double q0 = bg.Q(a0);
  GrowthState y{a0, q0, -3.0 / 7.0 * a0 * a0, -6.0 / 7.0 * a0 * q0};
  double x = std::log(a0);
  std::vector<GrowthState> out;
  out.reserve(targets.size());
  for (double t : targets) {
    const double xt = std::log(t);
    const int n = std::max(1, (int)std::ceil((xt - x) / 5e-4));
    const double h = (xt - x) / n;
    for (int i = 0; i < n; ++i) {
      const double a = std::exp(x), am = std::exp(x + 0.5 * h), a1 = std::exp(x + h);
      const GrowthState k1 = growth_rhs(bg, a, y);
      const GrowthState k2 = growth_rhs(bg, am, axpy(y, 0.5 * h, k1));
      const GrowthState k3 = growth_rhs(bg, am, axpy(y, 0.5 * h, k2));
      const GrowthState k4 = growth_rhs(bg, a1, axpy(y, h, k3));
      y.d1 += h / 6.0 * (k1.d1 + 2 * k2.d1 + 2 * k3.d1 + k4.d1);
      y.t1 += h / 6.0 * (k1.t1 + 2 * k2.t1 + 2 * k3.t1 + k4.t1);
      y.d2 += h / 6.0 * (k1.d2 + 2 * k2.d2 + 2 * k3.d2 + k4.d2);
      y.t2 += h / 6.0 * (k1.t2 + 2 * k2.t2 + 2 * k3.t2 + k4.t2);
      x += h;
    }
    x = xt;
    out.push_back(y);
  }
  return out;
}

// composite Simpson in ln a of int_{ai}^{af} a^n / Q(a) da
double drift_integral(const Background& bg, double ai, double af, double n) {
  const int m = 4096;
  const double x0 = std::log(ai), x1 = std::log(af), h = (x1 - x0) / m;
  auto f = [&](double x) {
    const double a = std::exp(x);
    return std::pow(a, n) * a / bg.Q(a);
  };
  double s = f(x0) + f(x1);
  for (int i = 1; i < m; ++i) s += f(x0 + i * h) * ((i & 1) ? 4.0 : 2.0);
  return s * h / 3.0;
}

double bbks(double k, double gamma) {
  const double q = k / gamma;
  const double x = 2.34 * q;
  const double lead = x > 1e-12 ? std::log1p(x) / x : 1.0;
  const double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
  return lead * std::pow(poly, -0.25);
}

double tophat(double x) {
  if (x < 1e-2) return 1.0 - x * x / 10.0 + x * x * x * x / 280.0;
  return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

// A such that sigma(8 Mpc/h) = sigma8 for P = A k^ns T^2
double power_amplitude(const cola_cosmo& c) {
  const double gamma = c.omega_m * c.h;
  const int m = 1 << 17;
  const double x0 = std::log(1e-7), x1 = std::log(1e4), h = (x1 - x0) / m;
  auto f = [&](double x) {
    const double k = std::exp(x);
    const double t = bbks(k, gamma), w = tophat(8.0 * k);
    return k * k * k * std::pow(k, c.n_s) * t * t * w * w;
  };
  double s = f(x0) + f(x1);
  for (int i = 1; i < m; ++i) s += f(x0 + i * h) * ((i & 1) ? 4.0 : 2.0);
  const double sigma2 = s * h / 3.0 / (2.0 * M_PI * M_PI);
  return c.sigma8 * c.sigma8 / sigma2;
}

}  // namespace

int build_coefficients(const cola_config& cfg, std::vector<double>& table, double& pk_amp, double& d2u1,
                       std::string& why) {
  const Background bg{cfg.cosmo.omega_m, cfg.cosmo.omega_l, 1.0 - cfg.cosmo.omega_m - cfg.cosmo.omega_l};
  const int n = cfg.nsteps;
  std::vector<double> a(n + 1), mid(n);
  for (int i = 0; i <= n; ++i)
    a[i] = cfg.log_a ? cfg.a_init * std::pow(cfg.a_final / cfg.a_init, (double)i / n)
                     : cfg.a_init + (cfg.a_final - cfg.a_init) * i / n;
  a[0] = cfg.a_init;
  a[n] = cfg.a_final;
  for (int i = 0; i < n; ++i) mid[i] = 0.5 * (a[i] + a[i + 1]);

  std::vector<double> targets(a);
  targets.push_back(1.0);
  std::sort(targets.begin(), targets.end());
  targets.erase(std::unique(targets.begin(), targets.end()), targets.end());
  const std::vector<GrowthState> gs = integrate_growth(bg, targets);
  auto at = [&](double x) -> const GrowthState& {
    const size_t i = std::lower_bound(targets.begin(), targets.end(), x) - targets.begin();
    return gs[i];
  };
  const GrowthState& g1 = at(1.0);
  d2u1 = g1.d2 / (g1.d1 * g1.d1);
  if (!(std::isfinite(d2u1)) || d2u1 == 0.0) {
    why = "growth factors are not finite";
    return COLA_EINVAL;
  }
  const double nl = cfg.n_lpt;
  auto u = [&](double x) { return std::pow(x, nl); };
  auto Tu = [&](double x) { return bg.Q(x) * nl * std::pow(x, nl - 1.0); };
  const bool modified_kick = cfg.scheme == COLA_SCHEME_COLA || cfg.scheme == COLA_SCHEME_COLA_U1;
  const bool modified_drift = cfg.scheme == COLA_SCHEME_COLA;
  auto kick = [&](double ka, double kb, double ac) {
    if (!modified_kick) return drift_integral(bg, ka, kb, 1.0) / ac;  // int (a/a_c)/Q da
    if (std::fabs(nl) < 1e-12) return std::log(kb / ka) * ac / bg.Q(ac);
    return (u(kb) - u(ka)) / Tu(ac);
  };

  table.assign((size_t)(n + 1) * COLA_NCOEF, 0.0);
  for (int i = 0; i <= n; ++i) {
    const GrowthState& g = at(a[i]);
    const double D1 = g.d1 / g1.d1, TD1 = g.t1 / g1.d1;
    const double D2un = g.d2 / (g1.d1 * g1.d1), TD2un = g.t2 / (g1.d1 * g1.d1);
    const double om = cfg.cosmo.omega_m;
    double* row = &table[(size_t)i * COLA_NCOEF];
    const double ka = i == 0 ? a[0] : mid[i - 1];
    const double kb = i == n ? a[n] : mid[i];
    row[0] = a[i];
    row[1] = 1.5 * om * a[i];
    row[2] = kick(ka, kb, a[i]);
    row[3] = 1.5 * om * a[i] * D1;
    row[4] = 1.5 * om * a[i] * (D2un - D1 * D1) / d2u1;
    if (i < n) {
      const GrowthState& h = at(a[i + 1]);
      row[5] = modified_drift ? drift_integral(bg, a[i], a[i + 1], nl) / u(mid[i])
                              : drift_integral(bg, a[i], a[i + 1], 0.0);  // int da/Q
      row[6] = h.d1 / g1.d1 - D1;
      row[7] = h.d2 / (g1.d1 * g1.d1) / d2u1 - D2un / d2u1;
      row[14] = a[i + 1];
    }
    row[8] = TD1;
    row[9] = TD2un / d2u1;
    row[10] = D1;
    row[11] = D2un / d2u1;
    row[12] = ka;
    row[13] = kb;
    row[15] = d2u1;
  }
  for (double x : table)
    if (!std::isfinite(x)) {
      why = "a time coefficient is not finite";
      return COLA_EINVAL;
    }
  pk_amp = power_amplitude(cfg.cosmo);
  if (!std::isfinite(pk_amp) || pk_amp <= 0) {
    why = "power spectrum normalisation failed";
    return COLA_EINVAL;
  }
  return COLA_OK;
}

void twiddle_table(int n, std::vector<float2>& out) {
  out.resize(n);
  for (int m = 0; m < n; ++m) {
    const double ang = -2.0 * M_PI * (double)m / (double)n;
    out[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
}

}  // namespace cola
