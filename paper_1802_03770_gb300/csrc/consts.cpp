// Host-side constants of the quadrature (paper Sec. 2.5-2.7), in grid units.
//
// With lattice offsets m (y_j - y_i = h m), rho = delta / h and s = d + alpha,
// the entries of M (eq. linearelliptic) are c k(m) with c = C_{alpha,d} h^{-alpha}:
//   k(0) = Z - 2d a,   k(m) = -|m|^{-s} + a [|m|_1 = 1]   (m != 0),
// where Z = h^{d+alpha} A_1 = sum_{m != 0} |m|^{-s} and
// a = h^{d+alpha-2} (A_2 + A_3) = S2 - T3 with
//   S2 = (1/2) sum_{m != 0} W(|m|/rho) m_1^2 / |m|^s          (A_2, eq. int1constants)
//   T3 = |S^{d-1}| / (2d) rho^{2-alpha} P(alpha)            (-A_3, eq. a3)
//   P(alpha) = int_0^1 W_1(t) t^{1-alpha} dt  for the window of eq. window.
// Z is evaluated by the Ewald (theta-function) split of the lattice sum,
// which converges exponentially; the paper's own route is Chebyshev far-field
// compression (end of Sec. 2.7), which targets the same number.
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace fl {

double c_alpha_d(double alpha, int d) {
  return std::pow(2.0, alpha) * std::tgamma(0.5 * (d + alpha)) /
         (std::pow(M_PI, 0.5 * d) * std::fabs(std::tgamma(-0.5 * alpha)));
}

// Regularised lower incomplete gamma by its power series
// gamma(a,x) = x^a e^{-x} sum_k x^k / (a (a+1) ... (a+k)), valid for x < a + 1.
static double lower_gamma_series(double a, double x) {
  double term = 1.0 / a, sum = term;
  for (int k = 1; k < 500; ++k) {
    term *= x / (a + k);
    sum += term;
    if (std::fabs(term) < 1e-17 * std::fabs(sum)) break;
  }
  return sum * std::exp(-x + a * std::log(x));
}

// Upper incomplete gamma by Legendre's continued fraction
// Gamma(a,x) = x^a e^{-x} / (x + 1 - a - 1(1-a)/(x + 3 - a - 2(2-a)/(x + 5 - a - ...))),
// evaluated with the modified Lentz method; valid for x >= a + 1.
static double upper_gamma_cf(double a, double x) {
  const double tiny = 1e-300;
  double b = x + 1.0 - a, c = 1.0 / tiny, dd = 1.0 / b, f = dd;
  for (int k = 1; k < 500; ++k) {
    const double an = -k * (k - a);
    b += 2.0;
    dd = an * dd + b;
    if (std::fabs(dd) < tiny) dd = tiny;
    c = b + an / c;
    if (std::fabs(c) < tiny) c = tiny;
    dd = 1.0 / dd;
    const double delta = dd * c;
    f *= delta;
    if (std::fabs(delta - 1.0) < 1e-16) break;
  }
  return f * std::exp(-x + a * std::log(x));
}

// Non-normalised upper incomplete gamma for a > -1, a != 0, x > 0.
double upper_gamma(double a, double x) {
  if (a < 0.0) return (upper_gamma(a + 1.0, x) - std::exp(a * std::log(x) - x)) / a;
  if (x < a + 1.0) return std::tgamma(a) - lower_gamma_series(a, x);
  return upper_gamma_cf(a, x);
}

// Z_d(alpha) = sum over Z^d minus 0 of |m|^{-(d+alpha)}.  From
// |m|^{-s} = pi^{s/2} / Gamma(s/2) int_0^inf t^{s/2-1} e^{-pi t |m|^2} dt,
// split at t = 1 and theta(t) = t^{-d/2} theta(1/t):
//   pi^{-s/2} Gamma(s/2) Z = sum_{m != 0} [ (pi|m|^2)^{-s/2} Gamma(s/2, pi|m|^2)
//       + (pi|m|^2)^{(s-d)/2} Gamma((d-s)/2, pi|m|^2) ] + 2/(s-d) - 2/s.
double lattice_zeta(int d, double alpha) {
  const double s = d + alpha;
  const int R = 7;  // e^{-pi |m|^2} < 1e-66 beyond
  double sum = 0.0;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int i = 0; i < d; ++i) { lo[i] = -R; hi[i] = R; }
  for (int i = lo[0]; i <= hi[0]; ++i)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int k = lo[2]; k <= hi[2]; ++k) {
        const int m2 = i * i + j * j + k * k;
        if (m2 == 0) continue;
        const double x = M_PI * m2;
        sum += std::pow(x, -0.5 * s) * upper_gamma(0.5 * s, x) +
               std::pow(x, 0.5 * (s - d)) * upper_gamma(0.5 * (d - s), x);
      }
  sum += 2.0 / (s - d) - 2.0 / s;
  return sum * std::pow(M_PI, 0.5 * s) / std::tgamma(0.5 * s);
}

static double window1(double t) {
  if (t >= 1.0) return 0.0;
  const double t2 = t * t, t4 = t2 * t2;
  return 1.0 + t4 * (-35.0 + t * (84.0 + t * (-70.0 + 20.0 * t)));
}

double window_corr(int d, double alpha, double rho) {
  const double s = d + alpha;
  const int R = (int)std::ceil(rho);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int i = 0; i < d; ++i) { lo[i] = -R; hi[i] = R; }
  double s2 = 0.0;
  for (int i = lo[0]; i <= hi[0]; ++i)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int k = lo[2]; k <= hi[2]; ++k) {
        const double m2 = (double)i * i + (double)j * j + (double)k * k;
        if (m2 == 0.0) continue;
        const double r = std::sqrt(m2);
        const double w = window1(r / rho);
        if (w == 0.0) continue;
        s2 += w * (double)i * i * std::pow(r, -s);
      }
  s2 *= 0.5;
  const double P = 1.0 / (2.0 - alpha) - 35.0 / (6.0 - alpha) + 84.0 / (7.0 - alpha) -
                   70.0 / (8.0 - alpha) + 20.0 / (9.0 - alpha);
  const double area = 2.0 * std::pow(M_PI, 0.5 * d) / std::tgamma(0.5 * d);
  const double t3 = area / (2.0 * d) * std::pow(rho, 2.0 - alpha) * P;
  return s2 - t3;
}

// In-place iterative radix-2 FFT (forward, e^{-2 pi i jk/L}) in long double,
// for the plan-time chirp tables.
void host_fft(std::vector<std::complex<long double>>& a) {
  const size_t L = a.size();
  for (size_t i = 1, j = 0; i < L; ++i) {
    size_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  const long double pi = 3.141592653589793238462643383279502884L;
  for (size_t len = 2; len <= L; len <<= 1) {
    const long double ang = -2.0L * pi / (long double)len;
    for (size_t i = 0; i < L; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const std::complex<long double> w(cosl(ang * k), sinl(ang * k));
        const std::complex<long double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

}  // namespace fl
