// Scale-discretised tiling of the harmonic and radial lines (App. A, Eqs. A2-A5) on the
// host, shared by the sphere plan and the ball wavelet plan.
#pragma once
#include <algorithm>
#include <cmath>

namespace s2w {
namespace tiling {

constexpr double kPi = 3.14159265358979323846264338327950288;

// 20-point Gauss-Legendre rule on [-1, 1] by Newton iteration on P_20.
struct GaussLegendre {
  static constexpr int n = 20;
  double x[n], w[n];
  GaussLegendre() {
    for (int i = 0; i < n; ++i) {
      double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-17) break;
      }
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

// Smooth bump s(t) = exp(-1/(1-t^2)) (Eq. A3) and its dilation s_lambda (Eq. A2).
inline double bump(double t) { return (t <= -1.0 || t >= 1.0) ? 0.0 : std::exp(-1.0 / (1.0 - t * t)); }

struct Tiling {
  double lam;
  double norm;
  GaussLegendre gl;
  explicit Tiling(double lam_) : lam(lam_) { norm = integral(1.0 / lam); }
  double integrand(double u) const {
    double s = bump(2.0 * lam / (lam - 1.0) * (u - 1.0 / lam) - 1.0);
    return s * s / u;
  }
  // int_a^b s_lambda(u)^2/u du over [a, b] clipped to the support [1/lambda, 1],
  // composite Gauss-Legendre (64 panels x 20 nodes).
  double integral(double a, double b = 1.0) const {
    a = std::max(a, 1.0 / lam);
    b = std::min(b, 1.0);
    if (a >= b) return 0.0;
    const int panels = 64;
    double h = (b - a) / panels, tot = 0.0;
    for (int p = 0; p < panels; ++p) {
      double lo = a + p * h, mid = lo + 0.5 * h, acc = 0.0;
      for (int i = 0; i < GaussLegendre::n; ++i) acc += gl.w[i] * integrand(mid + 0.5 * h * gl.x[i]);
      tot += 0.5 * h * acc;
    }
    return tot;
  }
  // k_lambda(t) (Eq. A4).
  double k(double t) const {
    if (t <= 1.0 / lam) return 1.0;
    if (t >= 1.0) return 0.0;
    return integral(t) / norm;
  }
  // kappa_lambda(t) = sqrt(k(t/lambda) - k(t)) (Eq. A5).  By Eq. A4 the difference is the
  // single integral of s_lambda^2/u over [t/lambda, t]; evaluating it that way keeps full
  // relative precision at the support edges, where two values of k near 1 would cancel.
  double kappa(double t) const {
    double d = integral(t / lam, t) / norm;
    return d > 0.0 ? std::sqrt(d) : 0.0;
  }
};

// ceil(lambda^e) robust to rounding of exact integer powers.
inline int ceil_pow(double lam, int e) {
  double v = std::pow(lam, e);
  double r = std::nearbyint(v);
  if (std::fabs(v - r) < 1e-9 * std::max(1.0, v)) return (int)r;
  return (int)std::ceil(v);
}

}  // namespace tiling
}  // namespace s2w
