// Upper quantile of the chi-square distribution, for eps of Lemma 3 (Eq. 2).
//
// The survival function of chi2(K) at x is the regularised upper incomplete
// gamma function Q(K/2, x/2). It is evaluated from its power series
// P(a,x) = x^a e^{-x} / Gamma(a+1) * sum_n x^n / ((a+1)...(a+n)) below
// x = a + 1, and from the Legendre continued fraction of Q(a,x) above it
// (evaluated with the modified Lentz method); the quantile is found by
// bisection, the survival function being decreasing in x.
#include <cmath>

namespace detlsh {

namespace {

double gamma_p_series(double a, double x) {
  double term = 1.0 / a, sum = term;
  for (int n = 1; n < 10000; ++n) {
    term *= x / (a + n);
    sum += term;
    if (std::fabs(term) < std::fabs(sum) * 1e-17) break;
  }
  return sum * std::exp(-x + a * std::log(x) - std::lgamma(a));
}

double gamma_q_cfrac(double a, double x) {
  const double tiny = 1e-300;
  double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 10000; ++i) {
    const double an = -i * (i - a);
    b += 2.0;
    d = an * d + b;
    if (std::fabs(d) < tiny) d = tiny;
    c = b + an / c;
    if (std::fabs(c) < tiny) c = tiny;
    d = 1.0 / d;
    const double del = d * c;
    h *= del;
    if (std::fabs(del - 1.0) < 1e-17) break;
  }
  return std::exp(-x + a * std::log(x) - std::lgamma(a)) * h;
}

double chi2_sf(double x, int K) {
  if (x <= 0.0) return 1.0;
  const double a = 0.5 * K, hx = 0.5 * x;
  if (hx < a + 1.0) return 1.0 - gamma_p_series(a, hx);
  return gamma_q_cfrac(a, hx);
}

}  // namespace

double chi2_upper_quantile(double alpha, int K) {
  if (!(alpha > 0.0 && alpha < 1.0) || K < 1) return std::nan("");
  double lo = 0.0, hi = 1.0;
  while (chi2_sf(hi, K) > alpha) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (chi2_sf(mid, K) > alpha) lo = mid;
    else hi = mid;
    if (hi - lo <= 1e-15 * hi) break;
  }
  return 0.5 * (lo + hi);
}

}  // namespace detlsh
