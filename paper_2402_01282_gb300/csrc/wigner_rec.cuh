// Wigner-d recursion in float64 shared by the contraction kernels: closed-form seeds at
// l0 = max(|m|, |n|) with an extended exponent, and the coefficients of the three-term
// recursion in l with the pole-accurate form of A (cos beta - B).
#pragma once
#include <math.h>

#include <cuda_runtime.h>
#include <stdint.h>

namespace s2w {

// ------------------------------------------------------------- Wigner-d recursion
struct RecTables {
  const double* wpole;   // -2 sin^2(beta/2) (northern half) or 2 cos^2(beta/2) (southern half)
  const double* cpow_m;
  const int* cpow_e;
  const double* spow_m;
  const int* spow_e;
  const double* sqrtC;
  int n;    // row stride (2L-1)
  int den;  // ring b sits at beta_b = pi (2b+1)/den; it is on the northern half when 2 (2b+1) < den
};

// Values below 2^-100 of the true d^l_mn never reach the sums; while a column's value
// is smaller than that it is carried scaled by 2^(600 q), q > 0, and skipped.
inline constexpr int kSkipExp = -100;
inline constexpr int kStepExp = 600;
inline constexpr double kRescaleAt = 3.273390607896142e+150;   // 2^500
inline constexpr double kRescaleBy = 2.409919865102884e-181;   // 2^-600

// d^{l0}_{mn}(beta_b) at l0 = max(|m|, |n|) from the closed form
//   d^l_{l n} = sqrt(binom(2l, l+n)) cos^{l+n}(b/2) (-sin(b/2))^{l-n}
// and the symmetries d_{mn} = (-1)^{m-n} d_{nm} = d_{-n,-m}.
__device__ __forceinline__ void wigner_seed(const RecTables& T, int b, int l0, int m, int n, double& v,
                                            int& q) {
  int kb, ac, as;
  double sign = 1.0;
  if (m == l0) {
    kb = l0 + n; ac = l0 + n; as = l0 - n;
    if ((l0 - n) & 1) sign = -1.0;
  } else if (m == -l0) {
    kb = l0 - n; ac = l0 - n; as = l0 + n;
  } else if (n == l0) {
    kb = l0 + m; ac = l0 + m; as = l0 - m;
  } else {
    kb = l0 - m; ac = l0 - m; as = l0 + m;
    if ((l0 + m) & 1) sign = -1.0;
  }
  const int64_t row = (int64_t)b * T.n;
  const double prod = sign * T.sqrtC[(int64_t)l0 * T.n + kb] * T.cpow_m[row + ac] * T.spow_m[row + as];
  q = 0;
  if (prod == 0.0) {
    v = 0.0;
    return;
  }
  const int E = T.cpow_e[row + ac] + T.spow_e[row + as];
  const int tot = E + ilogb(prod);
  if (tot >= kSkipExp) {
    v = scalbn(prod, E);
  } else {
    q = (kSkipExp - tot + kStepExp - 1) / kStepExp;
    v = scalbn(prod, E + kStepExp * q);
  }
}

// Coefficients of the three-term recursion in l (Varshalovich),
//   d^{l+1} = A (cos b - B) d^l - C d^{l-1},
//   A = (l+1)(2l+1)/sqrt(((l+1)^2-m^2)((l+1)^2-n^2)),  B = m n/(l(l+1)),
//   C = A sqrt((l^2-m^2)(l^2-n^2))/(l(2l+1))            (B = C = 0 at l = 0).
// Near the poles cos b and B are both close to +-1, so A (cos b - B) is formed as
//   north: A (1 - B) - A (1 - cos b),   south: A (1 + cos b) - A (1 + B),
// with 1 -+ B = (l(l+1) -+ m n)/(l(l+1)) from exact integers and 1 -+ cos b = 2 sin^2, 2 cos^2
// of the half angle (the per-ring weight `wpole`).  Kn = A (1 - B), Ks = -A (1 + B).
__device__ __forceinline__ void rec_coeffs(int l, int m, int n, double& A, double& Kn, double& Ks, double& C) {
  const double l1 = l + 1.0, dl = l;
  const double den = sqrt((l1 * l1 - (double)m * m) * (l1 * l1 - (double)n * n));
  A = l1 * (2.0 * dl + 1.0) / den;
  if (l == 0) {
    Kn = A;
    Ks = -A;
    C = 0.0;
  } else {
    const double ll = dl * l1, mn = (double)m * (double)n;   // exact integers in float64
    Kn = A * ((ll - mn) / ll);
    Ks = -A * ((ll + mn) / ll);
    C = A * sqrt((dl * dl - (double)m * m) * (dl * dl - (double)n * n)) / (dl * (2.0 * dl + 1.0));
  }
}


}  // namespace s2w
