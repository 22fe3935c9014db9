// Host-side constants of the CUDA path: Daubechies filters and the NUFFT kernel.
//
// Daubechies db1..db8 (the SARA bases of Section 4.1) are built here from their
// defining spectral factorisation, |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)),
// P(y) = sum_{k<p} C(p-1+k, k) y^k (Daubechies 1988), keeping the zeros inside
// the unit circle (extremal phase). The roots of P are found with the
// Weierstrass (Durand-Kerner) iteration in long double.
//
// The NUFFT interpolation kernel is the "exponential of semicircle"
// phi(t) = exp(beta (sqrt(1 - (2t/W)^2) - 1)), |t| < W/2 (Barnett, Magland &
// af Klinteberg 2019), with beta = 2.30 W for 2x oversampling. Its Fourier
// transform, which sets the de-apodisation of the Z operator in Phi = G F Z
// (Section 5.1, Eq. meas_op), is evaluated by Gauss-Legendre quadrature.
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace ps {

using cld = std::complex<long double>;

static std::vector<cld> poly_roots(const std::vector<long double>& a) {
  // a[k] multiplies y^k; returns the deg roots by Durand-Kerner.
  int deg = (int)a.size() - 1;
  std::vector<cld> r(deg);
  if (deg <= 0) return r;
  std::vector<cld> c(deg + 1);
  for (int k = 0; k <= deg; ++k) c[k] = cld(a[k] / a[deg], 0);
  cld seed(0.4L, 0.9L);
  for (int i = 0; i < deg; ++i) r[i] = std::pow(seed, (long double)i);
  for (int it = 0; it < 2000; ++it) {
    long double delta = 0;
    for (int i = 0; i < deg; ++i) {
      cld num = c[deg];
      for (int k = deg - 1; k >= 0; --k) num = num * r[i] + c[k];
      cld den(1, 0);
      for (int j = 0; j < deg; ++j)
        if (j != i) den *= (r[i] - r[j]);
      cld step = num / den;
      r[i] -= step;
      delta = std::max(delta, std::abs(step));
    }
    if (delta < 1e-30L) break;
  }
  return r;
}

void daubechies_filters(double h[kDb][kMaxTaps]) {
  for (int p = 1; p <= kDb; ++p) {
    for (int j = 0; j < kMaxTaps; ++j) h[p - 1][j] = 0.0;
    std::vector<long double> P(p);
    for (int k = 0; k < p; ++k) {           // binomial C(p-1+k, k)
      long double b = 1;
      for (int i = 1; i <= k; ++i) b = b * (long double)(p - 1 + i) / (long double)i;
      P[k] = b;
    }
    // Polynomial in z, stored by descending power: start with (z + 1)^p.
    std::vector<cld> poly{cld(1, 0)};
    auto mul = [&](cld a0, cld a1) {         // poly *= (a0 z + a1)
      std::vector<cld> out(poly.size() + 1, cld(0, 0));
      for (size_t i = 0; i < poly.size(); ++i) {
        out[i] += poly[i] * a0;
        out[i + 1] += poly[i] * a1;
      }
      poly.swap(out);
    };
    for (int k = 0; k < p; ++k) mul(cld(1, 0), cld(1, 0));
    for (const cld& y : poly_roots(P)) {
      // (2 - z - 1/z) / 4 = y  <=>  z^2 - (2 - 4y) z + 1 = 0; keep |z| < 1.
      cld b = cld(2, 0) - cld(4, 0) * y;
      cld d = std::sqrt(b * b - cld(4, 0));
      cld z1 = (b + d) / cld(2, 0), z2 = (b - d) / cld(2, 0);
      cld z = std::abs(z1) < 1.0L ? z1 : z2;
      mul(cld(1, 0), -z);
    }
    long double s = 0;
    for (const cld& c : poly) s += c.real();
    long double norm = std::sqrt(2.0L) / s;
    for (int j = 0; j < 2 * p; ++j) h[p - 1][j] = (double)(poly[j].real() * norm);
  }
}

double es_beta(int W) { return 2.30 * W; }

double es_kernel(double t, int W, double beta) {
  double z = 2.0 * t / W;
  if (std::fabs(z) >= 1.0) return 0.0;
  return std::exp(beta * (std::sqrt(1.0 - z * z) - 1.0));
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

double es_fourier(double xi, int W, double beta) {
  // phihat(xi) = int_{-W/2}^{W/2} phi(t) cos(xi t) dt; phi is even. The quadrature rule is
  // built once (thread-safe static initialisation: handles may be prepared concurrently).
  struct Rule {
    std::vector<double> x, w;
    Rule() { gauss_legendre(400, x, w); }
  };
  static const Rule rule;
  const double half = 0.5 * W;
  double s = 0.0;
  for (size_t i = 0; i < rule.x.size(); ++i) {
    const double t = half * rule.x[i];
    s += rule.w[i] * es_kernel(t, W, beta) * std::cos(xi * t);
  }
  return s * half;
}

}  // namespace ps
