// Minimax relative rational approximation of x^gamma on [lo, hi] (host code).
//
// The action and heatbath of the rational HMC need (M^dag M)^-1/4 and
// (M^dag M)^1/8 as alpha_0 + sum_i alpha_i / (x + beta_i) (Eqs. jkjk, hbeq) with
// coefficients minimising the error over the spectrum of the free operator
// (Sec. 7.4); the paper prints none, so they are computed here.  Reading: the
// largest relative error max |r(x) / x^gamma - 1| is minimised (type (d, d)).
//
// Method (double precision, product form r = C prod (x + z_i) / (x + p_i) with
// log-parametrised z_i, p_i, which keeps the Newton systems well scaled):
//   1. Zolotarev's closed-form optimum for gamma = -1/2 (Jacobi elliptic
//      functions by the arithmetic-geometric mean, Abramowitz & Stegun 16.4);
//   2. homotopy gamma: -1/2 -> -|gamma| in small steps, each a Remez exchange:
//      Newton on ln r(t_j) - gamma ln t_j = ln(1 + s_j h) at 2d + 2 alternating
//      extrema t_j, then new extrema of the error;
//   3. gamma > 0: 1/r approximates x^|gamma| (poles and zeros swap), refined by
//      one more exchange at +gamma;
//   4. partial fractions alpha_i = C prod_k (z_k - p_i) / prod_{k != i} (p_k - p_i).
// Where the optimum on [lo, hi] lies below what double precision resolves
// (relative error near 1e-14) the exchange cannot level the extrema; the
// interval is then widened until it can, which only lowers the error on the
// requested interval.  The error reported is measured on [lo, hi] from the
// partial fractions, the form the solver evaluates.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/wz.h"

namespace {

// ---------------------------------------------------------------- elliptic functions
// K(m) = pi / (2 AGM(1, sqrt(1 - m)))
double ellip_K(double m) {
  double a = 1.0, b = std::sqrt(1.0 - m);
  for (int i = 0; i < 60 && std::fabs(a - b) > 1e-16 * a; ++i) {
    const double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = an;
  }
  return 3.14159265358979323846 / (2.0 * a);
}

// sn(u | m), cn(u | m) by the descending AGM sequence (A&S 16.4.1-16.4.3)
void ellip_sncn(double u, double m, double* sn, double* cn) {
  double a[64], c[64];
  a[0] = 1.0;
  double b = std::sqrt(1.0 - m);
  c[0] = std::sqrt(m);
  int N = 0;
  while (N < 62 && std::fabs(c[N]) > 1e-17) {
    a[N + 1] = 0.5 * (a[N] + b);
    c[N + 1] = 0.5 * (a[N] - b);
    b = std::sqrt(a[N] * b);
    ++N;
  }
  double phi = std::ldexp(a[N] * u, N);
  for (int n = N; n >= 1; --n) phi = 0.5 * (phi + std::asin(c[n] * std::sin(phi) / a[n]));
  *sn = std::sin(phi);
  *cn = std::cos(phi);
}

// ---------------------------------------------------------------- product form
struct Approx {
  int d = 0;
  double gamma = 0.0;
  double c = 0.0;          // ln C
  std::vector<double> lz;  // ln z_i
  std::vector<double> lp;  // ln p_i
};

// ln r(t) - gamma ln t, each factor as log1p((z - p) / (t + p)) so that the
// rounding error of the sum stays relative to the (small) result
double log_err(const Approx& r, double t) {
  double s = r.c - r.gamma * std::log(t);
  for (int i = 0; i < r.d; ++i) {
    const double z = std::exp(r.lz[i]), p = std::exp(r.lp[i]);
    s += std::log1p((z - p) / (t + p));
  }
  return s;
}

double rel_err(const Approx& r, double t) { return std::expm1(log_err(r, t)); }

// Solve J x = f in place (n x n, row-major), partial pivoting; false if singular.
bool gauss(std::vector<double>& J, std::vector<double>& f, int n) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(J[i * n + k]) > std::fabs(J[piv * n + k])) piv = i;
    if (!(std::fabs(J[piv * n + k]) > 1e-300)) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(J[k * n + j], J[piv * n + j]);
      std::swap(f[k], f[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double l = J[i * n + k] / J[k * n + k];
      if (l == 0.0) continue;
      for (int j = k; j < n; ++j) J[i * n + j] -= l * J[k * n + j];
      f[i] -= l * f[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = f[k];
    for (int j = k + 1; j < n; ++j) s -= J[k * n + j] * f[j];
    f[k] = s / J[k * n + k];
    if (!std::isfinite(f[k])) return false;
  }
  return true;
}

// Alternating extrema of the relative error on [tl, th] (log grid, refined by
// golden section); exactly n of them or false.
bool extrema(const Approx& r, double tl, double th, int n, std::vector<double>& t, std::vector<double>& e) {
  const int G = 60 * n;
  const double L0 = std::log(tl), L1 = std::log(th);
  std::vector<double> s(G), v(G);
  for (int k = 0; k < G; ++k) {
    s[k] = L0 + (L1 - L0) * k / (G - 1);
    v[k] = rel_err(r, std::exp(s[k]));
    if (!std::isfinite(v[k])) return false;
  }
  std::vector<double> P, V;
  auto push = [&](double u, double val) {
    if (!P.empty() && ((val > 0) == (V.back() > 0))) {
      if (std::fabs(val) > std::fabs(V.back())) {
        P.back() = u;
        V.back() = val;
      }
    } else {
      P.push_back(u);
      V.push_back(val);
    }
  };
  const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
  for (int k = 0; k < G; ++k) {
    if (k == 0 || k == G - 1) {
      push(s[k], v[k]);
      continue;
    }
    if ((v[k] - v[k - 1]) * (v[k + 1] - v[k]) > 0) continue;
    const double sg = v[k] > 0 ? 1.0 : -1.0;
    double a = s[k - 1], b = s[k + 1];
    double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
    double f1 = sg * rel_err(r, std::exp(x1)), f2 = sg * rel_err(r, std::exp(x2));
    for (int it = 0; it < 50; ++it) {
      if (f1 > f2) {
        b = x2;
        x2 = x1;
        f2 = f1;
        x1 = b - gr * (b - a);
        f1 = sg * rel_err(r, std::exp(x1));
      } else {
        a = x1;
        x1 = x2;
        f1 = f2;
        x2 = a + gr * (b - a);
        f2 = sg * rel_err(r, std::exp(x2));
      }
    }
    const double u = 0.5 * (a + b);
    push(u, rel_err(r, std::exp(u)));
  }
  while ((int)P.size() > n) {  // drop the smaller end
    if (std::fabs(V.front()) < std::fabs(V.back())) {
      P.erase(P.begin());
      V.erase(V.begin());
    } else {
      P.pop_back();
      V.pop_back();
    }
  }
  if ((int)P.size() != n) return false;
  t.resize(n);
  e = V;
  for (int j = 0; j < n; ++j) t[j] = std::exp(P[j]);
  return true;
}

// Newton on the levelled-error equations at the reference t (sign of e at t_0
// given by s0); h is the level (>= 0) on input and output.
bool newton(Approx& r, const std::vector<double>& t, double s0, double& h) {
  const int d = r.d, n = 2 * d + 2;
  std::vector<double> sig(n);
  for (int j = 0; j < n; ++j) sig[j] = (j % 2 == 0) ? s0 : -s0;
  auto resid = [&](const Approx& a, double hh, std::vector<double>& F) -> double {
    double mx = 0.0;
    for (int j = 0; j < n; ++j) {
      if (!(1.0 + sig[j] * hh > 0.0)) return HUGE_VAL;
      F[j] = log_err(a, t[j]) - std::log1p(sig[j] * hh);
      mx = std::max(mx, std::fabs(F[j]));
    }
    return std::isfinite(mx) ? mx : HUGE_VAL;
  };
  std::vector<double> F(n), F2(n), J(n * n), dx(n);
  double nf = resid(r, h, F);
  if (!std::isfinite(nf)) return false;
  for (int it = 0; it < 40; ++it) {
    for (int j = 0; j < n; ++j) {
      J[j * n + 0] = 1.0;
      for (int i = 0; i < d; ++i) {
        const double z = std::exp(r.lz[i]), p = std::exp(r.lp[i]);
        J[j * n + 1 + i] = z / (t[j] + z);
        J[j * n + 1 + d + i] = -p / (t[j] + p);
      }
      J[j * n + n - 1] = -sig[j] / (1.0 + sig[j] * h);
      dx[j] = -F[j];
    }
    if (!gauss(J, dx, n)) return false;
    double lam = 1.0, nf2 = INFINITY, h2 = h;
    Approx a = r;
    for (int k = 0; k < 30; ++k) {
      a.c = r.c + lam * dx[0];
      for (int i = 0; i < d; ++i) {
        a.lz[i] = r.lz[i] + lam * dx[1 + i];
        a.lp[i] = r.lp[i] + lam * dx[1 + d + i];
      }
      h2 = h + lam * dx[n - 1];
      nf2 = resid(a, h2, F2);
      if (nf2 <= nf) break;
      lam *= 0.5;
    }
    if (!std::isfinite(nf2)) return false;
    double step = 0.0;
    for (int j = 0; j < n; ++j) step = std::max(step, std::fabs(lam * dx[j]));
    r = a;
    h = h2;
    F.swap(F2);
    nf = nf2;
    if (nf < 1e-15 || step < 1e-14) break;
  }
  return true;
}

// Remez exchange at fixed gamma from the current approximation and reference.
// Levelled when the extrema agree to 1e-6 or to the rounding noise of the
// error (~1e-13 absolute); after the iteration budget a spread below 1e-2 is
// accepted (by de la Vallee Poussin the optimum is then within 1% of the level).
bool remez(Approx& r, double tl, double th, std::vector<double>& t, double* level) {
  const int n = 2 * r.d + 2;
  std::vector<double> e;
  double h = 0.0;
  double s0 = rel_err(r, t[0]) > 0 ? 1.0 : -1.0;
  double spread = 1.0;
  for (int it = 0; it < 30; ++it) {
    h = std::fabs(h);
    if (!newton(r, t, s0, h)) return false;
    if (!extrema(r, tl, th, n, t, e)) return false;
    s0 = e[0] > 0 ? 1.0 : -1.0;
    double mx = 0.0, mn = HUGE_VAL;
    for (double v : e) {
      mx = std::max(mx, std::fabs(v));
      mn = std::min(mn, std::fabs(v));
    }
    *level = mx;
    spread = (mx - mn) / mx;
    if (spread < std::max(1e-6, 1e-13 / mx)) return true;
  }
  return spread < 1e-2;
}

// Minimax of t^gamma on [1/sqrt(kappa), sqrt(kappa)] in product form.
bool minimax_scaled(double gamma, double kappa, int d, Approx& out) {
  const double tl = 1.0 / std::sqrt(kappa), th = std::sqrt(kappa);
  const int n = 2 * d + 2;
  Approx r;
  r.d = d;
  r.gamma = -0.5;
  r.lz.resize(d);
  r.lp.resize(d);
  // 1. Zolotarev: c_l = tl sn^2 / cn^2 (l K / (2d + 1) | 1 - 1/kappa), poles at odd l
  const double m = 1.0 - 1.0 / kappa;
  const double K = ellip_K(m);
  for (int l = 1; l <= 2 * d; ++l) {
    double sn, cn;
    ellip_sncn(l * K / (2 * d + 1), m, &sn, &cn);
    const double cl = std::log(tl) + 2.0 * std::log(std::fabs(sn)) - 2.0 * std::log(std::fabs(cn));
    if (l % 2) r.lp[(l - 1) / 2] = cl;
    else r.lz[l / 2 - 1] = cl;
  }
  {  // level the constant, then take the extrema as the first reference
    double mx = -INFINITY, mn = INFINITY;
    for (int k = 0; k < 2001; ++k) {
      const double v = log_err(r, std::exp(std::log(tl) + (std::log(th) - std::log(tl)) * k / 2000.0));
      mx = std::max(mx, v);
      mn = std::min(mn, v);
    }
    r.c = -0.5 * (mx + mn);
  }
  std::vector<double> t, e;
  if (!extrema(r, tl, th, n, t, e)) return false;
  double level = 0.0;
  // 2. homotopy in gamma
  const double g1 = -std::fabs(gamma);
  const int steps = std::fabs(g1 + 0.5) < 1e-15 ? 1 : 8;
  for (int s = 1; s <= steps; ++s) {
    r.gamma = -0.5 + (g1 + 0.5) * s / steps;
    if (!remez(r, tl, th, t, &level)) return false;
  }
  // 3. positive powers: the reciprocal, refined at +gamma
  if (gamma > 0) {
    std::swap(r.lz, r.lp);
    r.c = -r.c;
    r.gamma = gamma;
    if (!remez(r, tl, th, t, &level)) return false;
  }
  out = r;
  return true;
}

// partial fractions of s^gamma C prod (x + s z_i) / (x + s p_i); false on cancellation
bool to_partial_fractions(const Approx& r, double s, wz_rational* o) {
  const int d = r.d;
  std::vector<double> Z(d), P(d);
  for (int i = 0; i < d; ++i) {
    Z[i] = s * std::exp(r.lz[i]);
    P[i] = s * std::exp(r.lp[i]);
  }
  std::vector<int> ord(d);
  for (int i = 0; i < d; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return P[a] < P[b]; });
  const double a0 = std::pow(s, r.gamma) * std::exp(r.c);
  o->d = d;
  o->a0 = a0;
  for (int q = 0; q < d; ++q) {
    const int i = ord[q];
    double res = a0;
    for (int k = 0; k < d; ++k) {
      res *= (Z[k] - P[i]);
      if (k != i) res /= (P[k] - P[i]);
    }
    if (!std::isfinite(res)) return false;
    o->alpha[q] = res;
    o->beta[q] = P[i];
  }
  for (int q = d; q < WZ_RATIONAL_MAX; ++q) o->alpha[q] = o->beta[q] = 0.0;
  return true;
}

double measured_error(const wz_rational* o, double gamma, double lo, double hi) {
  double mx = 0.0;
  const int N = 100001;
  for (int k = 0; k < N; ++k) {
    const double x = std::exp(std::log(lo) + (std::log(hi) - std::log(lo)) * k / (N - 1));
    double r = o->a0;
    for (int i = 0; i < o->d; ++i) r += o->alpha[i] / (x + o->beta[i]);
    mx = std::max(mx, std::fabs(r / std::pow(x, gamma) - 1.0));
  }
  return mx;
}

}  // namespace

extern "C" int wz_rational_minimax(double power, double lo, double hi, int d, wz_rational* out) {
  if (!out || !(lo > 0.0) || !(hi > lo) || d < 0 || d > WZ_RATIONAL_MAX || !(std::fabs(power) < 1.0) ||
      power == 0.0)
    return WZ_EINVAL;
  wz_rational o{};
  o.power = power;
  o.lo = lo;
  o.hi = hi;
  if (d == 0) {  // best constant: C = 2 / (lo^-gamma + hi^-gamma)
    o.d = 0;
    o.a0 = 2.0 / (std::pow(lo, -power) + std::pow(hi, -power));
    o.err = measured_error(&o, power, lo, hi);
    o.build_lo = lo;
    o.build_hi = hi;
    *out = o;
    return WZ_OK;
  }
  // widen the interval (geometrically about its centre) until the exchange levels
  double blo = lo, bhi = hi;
  for (int attempt = 0; attempt < 16; ++attempt) {
    Approx r;
    const double s = std::sqrt(blo * bhi);
    if (minimax_scaled(power, bhi / blo, d, r) && to_partial_fractions(r, s, &o)) {
      o.power = power;
      o.lo = lo;
      o.hi = hi;
      o.build_lo = blo;
      o.build_hi = bhi;
      o.err = measured_error(&o, power, lo, hi);
      *out = o;
      return WZ_OK;
    }
    blo *= 0.5;
    bhi *= 2.0;
  }
  return WZ_NOT_CONVERGED;
}
