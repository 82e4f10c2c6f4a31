// param_tails.cuh -- FP64 tails of the F and Student t laws for the parametric
// comparison statistics (one-way ANOVA F, dosage-regression t), shared by the
// host (thresholds) and the finalisation kernel.
//
// Both tails are regularised incomplete beta functions I_x(a, b):
//   P(F(d1, d2) > f) = I_{d2 / (d2 + d1 f)}(d2 / 2, d1 / 2),
//   P(|T(nu)| > t)   = I_{nu / (nu + t^2)}(nu / 2, 1 / 2),
// evaluated by the continued fraction of I_x(a, b) (the even / odd convergent
// pair of the classical expansion) with the modified Lentz method, on the side
// x < (a + 1) / (a + b + 2) where it converges fast, and by the reflection
// I_x(a, b) = 1 - I_{1-x}(b, a) otherwise.  Small tails are on the direct side, so
// they keep full relative precision.
#pragma once
#include <cmath>

namespace krux {

#ifdef __CUDACC__
#define KRUX_HD __host__ __device__
#else
#define KRUX_HD
#endif

// Continued fraction of I_x(a, b) / (x^a (1-x)^b / (a B(a, b))).
KRUX_HD inline double ibeta_cf(double a, double b, double x) {
  const double tiny = 1e-300;
  double f = 1.0, C = 1.0, Dn = 1.0 - (a + b) * x / (a + 1.0);
  if (std::fabs(Dn) < tiny) Dn = tiny;
  Dn = 1.0 / Dn;
  f = Dn;
  for (int m = 1; m <= 400; ++m) {
    const double dm = (double)m;
    // even step: d_{2m} = m (b - m) x / ((a + 2m - 1)(a + 2m))
    double c = dm * (b - dm) * x / ((a + 2.0 * dm - 1.0) * (a + 2.0 * dm));
    Dn = 1.0 + c * Dn;
    if (std::fabs(Dn) < tiny) Dn = tiny;
    C = 1.0 + c / C;
    if (std::fabs(C) < tiny) C = tiny;
    Dn = 1.0 / Dn;
    f *= Dn * C;
    // odd step: d_{2m+1} = -(a + m)(a + b + m) x / ((a + 2m)(a + 2m + 1))
    c = -(a + dm) * (a + b + dm) * x / ((a + 2.0 * dm) * (a + 2.0 * dm + 1.0));
    Dn = 1.0 + c * Dn;
    if (std::fabs(Dn) < tiny) Dn = tiny;
    C = 1.0 + c / C;
    if (std::fabs(C) < tiny) C = tiny;
    Dn = 1.0 / Dn;
    const double delta = Dn * C;
    f *= delta;
    if (std::fabs(delta - 1.0) < 1e-15) break;
  }
  return f;
}

// Regularised incomplete beta I_x(a, b), a, b > 0.
KRUX_HD inline double ibeta(double a, double b, double x) {
  if (!(x > 0.0)) return 0.0;
  if (!(x < 1.0)) return 1.0;
  const double lfront = std::lgamma(a + b) - std::lgamma(a) - std::lgamma(b) + a * std::log(x) +
                        b * std::log1p(-x);
  if (x < (a + 1.0) / (a + b + 2.0)) return std::exp(lfront) * ibeta_cf(a, b, x) / a;
  return 1.0 - std::exp(lfront) * ibeta_cf(b, a, 1.0 - x) / b;
}

// Upper tail of F(d1, d2) at f >= 0.  With two numerator degrees of freedom (three
// genotype groups) I_x(d2/2, 1) = x^(d2/2), i.e. the tail is (1 + 2f/d2)^(-d2/2) in
// closed form; other d1 take the continued fraction.
KRUX_HD inline double f_tail(double f, double d1, double d2) {
  if (!(f > 0.0)) return 1.0;
  if (d1 == 2.0) return std::exp(-0.5 * d2 * std::log1p(2.0 * f / d2));
  return ibeta(0.5 * d2, 0.5 * d1, d2 / (d2 + d1 * f));
}

// Two-sided tail of Student's t(nu) at |t|.
KRUX_HD inline double t_tail2(double t, double nu) {
  if (!(t * t > 0.0)) return 1.0;
  return ibeta(0.5 * nu, 0.5, nu / (nu + t * t));
}

}  // namespace krux
