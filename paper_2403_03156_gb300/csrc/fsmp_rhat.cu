// fsmp_rhat.cu -- the convergence check of Sec. 3.2 (host code): the Gelman-Rubin potential
// scale reduction R of a scalar over several chains of one waveform, from the chains'
// summaries, as the point estimate of Gelman and Rubin (1992) and as the degrees-of-freedom
// corrected estimate with its upper confidence limit (Gelman and Rubin 1992, Sec. 3; Brooks
// and Gelman 1998, Sec. 3.2). The scalars are N, t0, the charge summary and the Wasserstein
// scalars of the PE sequences {t_i} and {e_i} (a dummy PE at t = 0, e = 0 joins every
// sequence; the scalar is the sequence's 1-Wasserstein distance to the dummy alone).
//
// The upper limit needs a quantile of the F distribution. It is found by bisection on the
// regularized incomplete beta function I_x(a, b) (P(F <= f) = I_{d1 f / (d1 f + d2)}(d1 / 2,
// d2 / 2)), evaluated by its continued fraction with the modified Lentz algorithm; for an
// infinite d2 (the within-chain variance known exactly) by bisection on the regularized
// incomplete gamma function P(k / 2, y / 2) of the chi-square distribution (series below
// a + 1, continued fraction above). log Gamma(b + a) - log Gamma(b) uses Stirling's series
// for large b, where the difference of two lgamma values would lose its digits.
#include <math.h>

#include "fsmp_internal.h"

namespace fsmp {
namespace {

// Stirling's correction log Gamma(x) - [(x - 1/2) log x - x + log(2 pi) / 2], x >= 10
double stirling_tail(double x) {
  const double r = 1.0 / x, r2 = r * r;
  return r * (1.0 / 12.0 - r2 * (1.0 / 360.0 - r2 * (1.0 / 1260.0 - r2 / 1680.0)));
}

// log Gamma(b + a) - log Gamma(b), a > 0, b > 0
double lgamma_ratio(double b, double a) {
  if (b < 100.0) return lgamma(b + a) - lgamma(b);
  return (b - 0.5) * log1p(a / b) + a * log(b + a) - a + stirling_tail(b + a) - stirling_tail(b);
}

// continued fraction of I_x(a, b) (modified Lentz), for x < (a + 1) / (a + b + 2)
double beta_cf(double a, double b, double x) {
  const double tiny = 1e-300;
  double c = 1.0, d = 1.0 - (a + b) * x / (a + 1.0);
  if (fabs(d) < tiny) d = tiny;
  d = 1.0 / d;
  double h = d;
  for (int k = 1; k <= 1000000; ++k) {
    const double k2 = 2.0 * k;
    double num = k * (b - k) * x / ((a + k2 - 1.0) * (a + k2));  // even step
    d = 1.0 + num * d;
    if (fabs(d) < tiny) d = tiny;
    c = 1.0 + num / c;
    if (fabs(c) < tiny) c = tiny;
    d = 1.0 / d;
    h *= d * c;
    num = -(a + k) * (a + b + k) * x / ((a + k2) * (a + k2 + 1.0));  // odd step
    d = 1.0 + num * d;
    if (fabs(d) < tiny) d = tiny;
    c = 1.0 + num / c;
    if (fabs(c) < tiny) c = tiny;
    d = 1.0 / d;
    const double del = d * c;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return h;
}

// regularized incomplete beta I_x(a, b)
double ibeta(double a, double b, double x) {
  if (x <= 0.0) return 0.0;
  if (x >= 1.0) return 1.0;
  // log of x^a (1 - x)^b / B(a, b), B(a, b) = Gamma(a) Gamma(b) / Gamma(a + b); the ratio of
  // Gammas taken with the larger argument in lgamma_ratio
  const double lb = a >= b ? lgamma_ratio(a, b) - lgamma(b) : lgamma_ratio(b, a) - lgamma(a);
  const double lf = lb + a * log(x) + b * log1p(-x);
  if (x < (a + 1.0) / (a + b + 2.0)) return exp(lf) * beta_cf(a, b, x) / a;
  return 1.0 - exp(lf) * beta_cf(b, a, 1.0 - x) / b;
}

// regularized lower incomplete gamma P(a, x)
double igamma_p(double a, double x) {
  if (x <= 0.0) return 0.0;
  const double lf = a * log(x) - x - lgamma(a);
  if (x < a + 1.0) {  // series: x^a e^-x / Gamma(a + 1) sum_n x^n / ((a + 1) .. (a + n))
    double term = 1.0 / a, sum = term, ap = a;
    for (int n = 1; n < 1000000; ++n) {
      ap += 1.0;
      term *= x / ap;
      sum += term;
      if (fabs(term) < fabs(sum) * 1e-17) break;
    }
    return sum * exp(lf);
  }
  // continued fraction of Q(a, x) (modified Lentz)
  const double tiny = 1e-300;
  double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 1000000; ++i) {
    const double an = -i * (i - a);
    b += 2.0;
    d = an * d + b;
    if (fabs(d) < tiny) d = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    d = 1.0 / d;
    const double del = d * c;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return 1.0 - exp(lf) * h;
}

// the p quantile of F(d1, d2); d2 = inf gives chi2(d1) / d1. Above d2 = 1e7 the limit is taken
// as well: the quantile differs from it by a relative O(1 / d2) there, while the beta function's
// complementary fraction would need 1 - x (x ~ d1 f / d2) to more digits than a double holds.
double f_quantile(double p, double d1, double d2) {
  if (d2 > 1e7) {
    double lo = 0.0, hi = d1 + 10.0;
    while (igamma_p(0.5 * d1, 0.5 * hi) < p && hi < 1e12) hi *= 2.0;
    for (int it = 0; it < 2000 && hi - lo > 1e-15 * hi; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (igamma_p(0.5 * d1, 0.5 * mid) < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi) / d1;
  }
  double lo = 0.0, hi = 1.0;  // on x = d1 f / (d1 f + d2), where P(F <= f) = I_x(d1/2, d2/2)
  for (int it = 0; it < 5000 && hi - lo > 1e-16 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (ibeta(0.5 * d1, 0.5 * d2, mid) < p) lo = mid; else hi = mid;
  }
  const double x = 0.5 * (lo + hi);
  return d2 * x / (d1 * (1.0 - x));
}

double field_mean(const fsmp_summary& c, int field) {
  switch (field) {
    case FSMP_RHAT_N: return c.mean_N;
    case FSMP_RHAT_T0: return c.mean_t0;
    case FSMP_RHAT_Q: return c.mean_Q;
    case FSMP_RHAT_WT: return c.mean_wt;
    default: return c.mean_we;
  }
}
double field_var(const fsmp_summary& c, int field) {
  switch (field) {
    case FSMP_RHAT_N: return c.var_N;
    case FSMP_RHAT_T0: return c.var_t0;
    case FSMP_RHAT_Q: return c.var_Q;
    case FSMP_RHAT_WT: return c.var_wt;
    default: return c.var_we;
  }
}

}  // namespace
}  // namespace fsmp

using namespace fsmp;

extern "C" int fsmp_gelman_rubin(const fsmp_summary* chains, int m, int field, double* rhat) {
  record_error(nullptr, nullptr);
  if (!chains || !rhat || m < 2 || field < FSMP_RHAT_N || field > FSMP_RHAT_WE) {
    record_error("fsmp_gelman_rubin", "bad arguments");
    return FSMP_ERR_INVALID;
  }
  const int n = chains[0].n_samples;
  if (n < 2) {
    record_error("fsmp_gelman_rubin", "fewer than two samples per chain");
    return FSMP_ERR_INVALID;
  }
  double sx = 0.0;
  for (int j = 0; j < m; ++j) {
    if (chains[j].n_samples != n) {
      record_error("fsmp_gelman_rubin", "chains of different lengths");
      return FSMP_ERR_INVALID;
    }
    sx += field_mean(chains[j], field);
  }
  const double xbar = sx / m;
  double w = 0.0, b = 0.0;
  for (int j = 0; j < m; ++j) {
    const double x = field_mean(chains[j], field);
    w += field_var(chains[j], field) * n / (n - 1.0);
    b += (x - xbar) * (x - xbar);
  }
  w /= m;
  const double b_over_n = b / (m - 1.0);
  if (!(w > 0.0)) {
    *rhat = b_over_n > 0.0 ? INFINITY : 1.0;
    return FSMP_OK;
  }
  *rhat = sqrt(((n - 1.0) / n * w + b_over_n) / w);
  return FSMP_OK;
}

extern "C" int fsmp_gelman_diag(const fsmp_summary* chains, int m, int field, double confidence, double* rhat,
                                double* upper) {
  record_error(nullptr, nullptr);
  if (!chains || !rhat || !upper || m < 2 || field < FSMP_RHAT_N || field > FSMP_RHAT_WE || !(confidence > 0.0) ||
      !(confidence < 1.0)) {
    record_error("fsmp_gelman_diag", "bad arguments");
    return FSMP_ERR_INVALID;
  }
  const int n = chains[0].n_samples;
  if (n < 2) {
    record_error("fsmp_gelman_diag", "fewer than two samples per chain");
    return FSMP_ERR_INVALID;
  }
  // chain means xbar_j and within-chain variances s2_j (n - 1 denominators) from the
  // summaries' population variances
  double mx = 0.0, ms2 = 0.0;
  for (int j = 0; j < m; ++j) {
    if (chains[j].n_samples != n) {
      record_error("fsmp_gelman_diag", "chains of different lengths");
      return FSMP_ERR_INVALID;
    }
    mx += field_mean(chains[j], field);
    ms2 += field_var(chains[j], field) * n / (n - 1.0);
  }
  mx /= m;
  const double W = ms2 / m;
  // across chains (m - 1 denominators): var(xbar), var(s2), cov(s2, xbar^2), cov(s2, xbar)
  double mx2 = 0.0;
  for (int j = 0; j < m; ++j) {
    const double x = field_mean(chains[j], field);
    mx2 += x * x;
  }
  mx2 /= m;
  double vx = 0.0, vs2 = 0.0, cs2x2 = 0.0, cs2x = 0.0;
  for (int j = 0; j < m; ++j) {
    const double x = field_mean(chains[j], field), s2 = field_var(chains[j], field) * n / (n - 1.0);
    vx += (x - mx) * (x - mx);
    vs2 += (s2 - W) * (s2 - W);
    cs2x2 += (s2 - W) * (x * x - mx2);
    cs2x += (s2 - W) * (x - mx);
  }
  vx /= (m - 1.0); vs2 /= (m - 1.0); cs2x2 /= (m - 1.0); cs2x /= (m - 1.0);
  const double B = n * vx;
  if (!(W > 0.0)) {
    *rhat = *upper = B == 0.0 ? 1.0 : INFINITY;
    return FSMP_OK;
  }
  const double k = 1.0 + 1.0 / m;
  const double V = (n - 1.0) / n * W + k * B / n;
  const double varV = ((n - 1.0) * (n - 1.0) * vs2 / m + k * k * 2.0 * B * B / (m - 1.0) +
                       2.0 * (n - 1.0) * k * ((double)n / m) * (cs2x2 - 2.0 * mx * cs2x)) /
                      ((double)n * n);
  double dadj = 1.0;
  if (varV > 0.0) {
    const double d = 2.0 * V * V / varV;
    dadj = (d + 3.0) / (d + 1.0);
  }
  const double r_fixed = (n - 1.0) / n, r_random = k * (B / W) / n;
  const double d2 = vs2 > 0.0 ? 2.0 * W * W * m / vs2 : INFINITY;
  const double fq = f_quantile(0.5 * (1.0 + confidence), m - 1.0, d2);
  *rhat = sqrt(dadj * (r_fixed + r_random));
  *upper = sqrt(dadj * (r_fixed + fq * r_random));
  return FSMP_OK;
}
